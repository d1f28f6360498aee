"""Batched flows (alb_batch_*): many flows of uneven size in one launch per
step must give, flow by flow, exactly what each flow gives alone through
alb_step: the per-node update is the same code and reads only its own flow,
so every kernel variant, tile shape and work distribution must agree bit for
bit, and so must the counters."""
import numpy as np
import pytest

from paper_2009_13426_gb300 import flows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FS = flows.FlowSpec
# small (nx < 128), medium (nx < 512) and large flows, both precisions
SPECS = [
    FS("vortex", 40, 24, 1.2, 2.0, 1e-3, 0, "fp32", seed=11),
    FS("shear", 64, 64, 2.0, 3.0, 1e-4, 0, "fp32", seed=12),
    FS("shear", 136, 20, 1.5, 2.0, 1e-5, 0, "fp32", seed=13),
    FS("shear", 520, 8, 2.2, 3.0, 1e-4, 0, "fp32", seed=16),
    FS("vortex", 49, 41, 1.0, 1.5, 1e-3, 0, "fp64", seed=14),
    FS("shear", 96, 40, 2.5, 3.0, 1e-4, 0, "fp64", seed=15),
]
STEPS = 7  # three graph replays of two steps, then one single step


@pytest.fixture(scope="module")
def alb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13426_gb300 import alb as A
    A.lib()
    return A


def cfg_of(alb, sp):
    prec = alb.ALB_FP32_FORM if sp.precision == "fp32" else alb.ALB_FP64_PLAIN
    return dict(nx=sp.nx, ny=sp.ny, nu=sp.nu, precision=prec)


def state(fl):
    return fl.moments(), fl.shifts()


# Work counters of the equilibrium solves depend on the tile shape: the
# rebuilt pulls of one sender in one receiver lattice share a solve within a
# tile. The state and the per-node and per-pull counters do not.
SOLVE_WORK = ("newton_calls", "newton_iterations", "fp64_evaluations", "fp32_iterations",
              "fp64_updates")


def per_pull(st):
    return {k: v for k, v in st.items() if k not in SOLVE_WORK}


def alone(alb, sp, steps):
    fl = alb.Flow(**cfg_of(alb, sp))
    assert fl.init(*sp.fields()) == alb.ALB_OK
    fl.step(steps)
    fl.sync()
    out = state(fl), fl.stats()
    fl.close()
    return out


@pytest.fixture(scope="module")
def reference(alb):
    return {k: {n: alone(alb, sp, n) for n in (2, 3, STEPS)} for k, sp in enumerate(SPECS)}


def init_all(batch):
    for sp, fl in zip(SPECS, batch.flows):
        fl.init(*sp.fields())


def assert_same(got, ref, what):
    (m, s), (M, S) = got, ref
    for a, b in zip(m, M):
        assert np.array_equal(a, b), what
    for a, b in zip(s, S):
        assert np.array_equal(a, b), what


def test_batch_equals_alone_bit_for_bit(alb, reference):
    b = alb.Batch([cfg_of(alb, sp) for sp in SPECS])
    try:
        init_all(b)
        b.step(STEPS)
        b.sync()
        for k, fl in enumerate(b.flows):
            assert_same(state(fl), reference[k][STEPS][0], "flow %d" % k)
            st, ref = fl.stats(), reference[k][STEPS][1]
            assert per_pull(st) == per_pull(ref), (k, st, ref)
    finally:
        b.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_every_variant_and_tile_shape_agrees(alb, reference, prec):
    P = alb.ALB_FP32_FORM if prec == "fp32" else alb.ALB_FP64_PLAIN
    b = alb.Batch([cfg_of(alb, sp) for sp in SPECS])
    try:
        for v, (block, _) in enumerate(alb.alb_batch_variants(P)):
            for tw, dyn in ((8, 0), (min(32, block), 1), (block, 1)):
                b.set_tuning(P, variant=v, tile_w=(tw, tw, tw), dynamic=dyn)
                assert b.tuning(P)["variant"] == v
                init_all(b)
                b.step(STEPS)
                b.sync()
                for k, (sp, fl) in enumerate(zip(SPECS, b.flows)):
                    if sp.precision == prec:
                        assert_same(state(fl), reference[k][STEPS][0],
                                    "flow %d variant %d tile %d dynamic %d" % (k, v, tw, dyn))
    finally:
        b.close()


def test_tuner_leaves_state_and_counters_alone(alb, reference):
    b = alb.Batch([cfg_of(alb, sp) for sp in SPECS])
    try:
        init_all(b)
        b.step(3)
        b.sync()
        before = [(state(fl), fl.stats()) for fl in b.flows]
        b.tune(trials=1)
        for k, fl in enumerate(b.flows):
            assert_same(state(fl), before[k][0], "flow %d after tuning" % k)
            assert fl.stats() == before[k][1]
            assert_same(state(fl), reference[k][3][0], "flow %d" % k)
        for P in (alb.ALB_FP32_FORM, alb.ALB_FP64_PLAIN):
            t = b.tuning(P)
            block = alb.alb_batch_variants(P)[t["variant"]][0]
            assert all(8 <= w <= block for w in t["tile_w"])
        b.step(STEPS - 3)
        b.sync()
        for k, fl in enumerate(b.flows):
            assert_same(state(fl), reference[k][STEPS][0], "flow %d tuned" % k)
    finally:
        b.close()


def test_flow_stepped_alone_inside_a_batch(alb, reference):
    """A batch flow's own handle steps it alone; the batch picks up its
    buffer parity at the next batched step."""
    b = alb.Batch([cfg_of(alb, sp) for sp in SPECS])
    try:
        init_all(b)
        b.flows[0].step(1)
        b.step(2)
        b.sync()
        assert_same(state(b.flows[0]), reference[0][3][0], "flow 0")
        for k in range(1, len(SPECS)):
            assert_same(state(b.flows[k]), reference[k][2][0], "flow %d" % k)
    finally:
        b.close()


def test_batch_errors(alb):
    b = alb.Batch([cfg_of(alb, sp) for sp in SPECS[:2]])
    try:
        with pytest.raises(alb.AlbError) as ei:
            b.step(1)  # not initialised
        assert ei.value.code == alb.ALB_EINVAL
        with pytest.raises(alb.AlbError) as ei:
            alb.alb_destroy(b.flows[0].h)  # owned by the batch
        assert ei.value.code == alb.ALB_EINVAL
        with pytest.raises(alb.AlbError):
            b.set_tuning(alb.ALB_FP32_FORM, variant=99)
        with pytest.raises(alb.AlbError):
            b.set_tuning(alb.ALB_FP32_FORM, variant=0, tile_w=(12, 64, 64))
        with pytest.raises(alb.AlbError):
            alb.alb_batch_flow(b.b, 5)
    finally:
        b.close()


def test_prandtl_flows_in_a_batch(alb):
    """Flows with Pr != 1 (App. E) in a batch, next to BGK flows: bit-identical
    to each flow run alone."""
    specs = [(SPECS[0], 0.71), (SPECS[1], 1.0), (SPECS[4], 2.0), (SPECS[5], 0.5)]
    cfgs = [dict(cfg_of(alb, sp), prandtl=pr) for sp, pr in specs]
    ref = []
    for (sp, _), c in zip(specs, cfgs):
        fl = alb.Flow(**c)
        fl.init(*sp.fields())
        fl.step(STEPS)
        fl.sync()
        ref.append(state(fl))
        fl.close()
    b = alb.Batch(cfgs)
    try:
        for (sp, _), fl in zip(specs, b.flows):
            fl.init(*sp.fields())
        b.step(STEPS)
        b.sync()
        for k, fl in enumerate(b.flows):
            assert_same(state(fl), ref[k], "flow %d" % k)
    finally:
        b.close()


def _sync_flagged(alb, obj):
    """Wait; a flagged root-finder failure (ALB_ENEWTON) is part of the state
    being compared, not an error here."""
    try:
        obj.sync()
    except alb.AlbError as e:
        if e.code != alb.ALB_ENEWTON:
            raise


def test_mixed_configurations_in_one_batch(alb):
    """Flows that differ in every per-flow option - overlap rules, sensor,
    zero-gradient ends, the reduced model, Maxwellian or previous starts, u_max,
    n0 - share one launch and each stays bit-identical to its own run, its
    per-node and per-pull counters (including any flagged rebuild failures)
    included."""
    ZG = alb.ALB_ZERO_GRADIENT
    specs = [
        (SPECS[0], dict(shift_overlap=0.5, shift_rule=alb.ALB_RULE_HISTORY)),
        (SPECS[1], dict(shift_overlap=0.4, shift_rule=alb.ALB_RULE_NEIGHBOURS, bc_x=ZG)),
        (SPECS[2], dict(sensor=1, bc_y=ZG, n0=0.51)),
        (SPECS[3], dict(moments=4)),
        (SPECS[4], dict(newton_start=alb.ALB_START_PREVIOUS, u_max=3)),
        (SPECS[5], dict(shift_overlap=0.3, shift_rule=alb.ALB_RULE_NEIGHBOURS, sensor=1,
                        prandtl=0.8)),
    ]
    cfgs = [dict(cfg_of(alb, sp), **extra) for sp, extra in specs]
    ref = []
    for (sp, _), c in zip(specs, cfgs):
        fl = alb.Flow(**c)
        assert fl.init(*sp.fields()) == alb.ALB_OK
        fl.step(STEPS)
        _sync_flagged(alb, fl)
        ref.append((state(fl), fl.stats()))
        fl.close()
    b = alb.Batch(cfgs)
    try:
        for (sp, _), fl in zip(specs, b.flows):
            fl.init(*sp.fields())
        b.step(STEPS)
        _sync_flagged(alb, b)
        for k, fl in enumerate(b.flows):
            assert_same(state(fl), ref[k][0], "flow %d" % k)
            got, want = fl.stats(), ref[k][1]
            assert per_pull(got) == per_pull(want), k
    finally:
        b.close()

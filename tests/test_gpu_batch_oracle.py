"""Batched flows and served requests against the CPU oracle.

The result a batched or served flow must reproduce is the paper's time step
(Sec. IV.A.3; Eqs. stream, coll): the oracle's, not only the single-flow
kernel's. One batch holds four uneven flows: an FP64 plain vortex with
lattice changes and rebuilt pulls, an FP64 plain Sod tube with zero-gradient
ends and the kinetic sensor, an FP32-form shear layer and an FP32-form
vortex. FP64 flows are compared with the free-running oracle (1e-11, shifts
and rebuild counts equal), FP32 flows with the oracle replaying the batch's
lattice decisions (1e-5). The batch is stepped one launch per step for the
replay, and a second copy is stepped by the two-step CUDA graph; the two must
agree bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2009_13426_gb300 import flows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5
STEPS = 60


@pytest.fixture(scope="module")
def alb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13426_gb300 import alb as A
    A.lib()
    return A


def rel_errors(got, ref):
    r, a, b, e = got
    R, A, B, E = ref
    mom = np.sqrt((a - A) ** 2 + (b - B) ** 2).max() / np.sqrt(A ** 2 + B ** 2).max()
    return max(np.abs(r - R).max() / np.abs(R).max(), mom, np.abs(e - E).max() / np.abs(E).max())


def _flows(alb):
    """(name, GPU config, oracle config keywords, fields) of the batch's flows."""
    zg = alb.ALB_ZERO_GRADIENT
    shear = flows.FlowSpec("shear", 96, 64, 2.5, 3.0, 1e-4, STEPS, "fp32", seed=41)
    vort = flows.FlowSpec("vortex", 40, 24, 1.2, 2.0, 1e-3, STEPS, "fp32", seed=42)
    return [
        ("vortex fp64", dict(nx=64, ny=64, nu=1e-3, precision=alb.ALB_FP64_PLAIN),
         dict(nu=1e-3), flows.isentropic_vortex()),
        ("sod fp64", dict(nx=512, ny=4, nu=1e-4, precision=alb.ALB_FP64_PLAIN, bc_x=zg,
                          sensor=1),
         dict(nu=1e-4, bc_x=O.ZERO_GRADIENT, sensor=True), flows.riemann_1d(512, 4)),
        ("shear fp32", dict(nx=96, ny=64, nu=1e-4, precision=alb.ALB_FP32_FORM, sensor=1),
         dict(nu=1e-4, sensor=True), shear.fields()),
        ("vortex fp32", dict(nx=40, ny=24, nu=1e-3, precision=alb.ALB_FP32_FORM),
         dict(nu=1e-3), vort.fields()),
    ]


def test_batched_flows_match_the_oracle(alb):
    specs = _flows(alb)
    b = alb.Batch([c for _, c, _, _ in specs])
    g = alb.Batch([c for _, c, _, _ in specs])
    try:
        for (_, c, _, fld), fa, fg in zip(specs, b.flows, g.flows):
            assert fa.init(*fld) == alb.ALB_OK and fg.init(*fld) == alb.ALB_OK
        fp32 = [k for k, (_, c, _, _) in enumerate(specs) if c["precision"] == alb.ALB_FP32_FORM]
        replay = {}
        for k in fp32:
            _, c, okw, fld = specs[k]
            s = O.Simulation(O.make_config(c["nx"], c["ny"], **okw))
            assert s.init(*fld) == O.OK
            replay[k] = s
        for _ in range(STEPS):
            b.step(1)
            for k in fp32:
                ux, uy = b.flows[k].shifts()
                assert replay[k].step_forced(ux, uy) == O.OK
        b.sync()
        g.step(STEPS)  # two-step graph replays
        g.sync()
        for k, (name, c, okw, fld) in enumerate(specs):
            fa, fg = b.flows[k], g.flows[k]
            for x, y in zip(fa.moments() + list(fa.shifts()), fg.moments() + list(fg.shifts())):
                assert np.array_equal(x, y), name
            st = fa.stats()
            assert st["newton_failures"] == 0 and st["reconstruction_failures"] == 0, name
            if k in replay:
                err = rel_errors(fa.moments(), replay[k].moments())
                assert err <= FP32_TOL, (name, err)
                continue
            s = O.Simulation(O.make_config(c["nx"], c["ny"], **okw))
            assert s.init(*fld) == O.OK
            assert s.step(STEPS) == O.OK
            err = rel_errors(fa.moments(), s.moments())
            assert err <= FP64_TOL, (name, err)
            sx, sy = fa.shifts()
            rx, ry = s.shifts()
            assert (sx == rx).all() and (sy == ry).all(), name
            assert st["reconstructions"] == s.stats()["reconstructions"], name
        # the vortex and the shear layer changed lattices on the way
        assert b.flows[0].stats()["reconstructions"] > 0
        assert b.flows[2].stats()["reconstructions"] > 0
    finally:
        b.close()
        g.close()


def test_served_requests_match_the_oracle(alb):
    """Two requests served among others: an FP64 plain vortex against the
    free-running oracle (1e-11, the same number of rebuilt pulls), and an
    FP32-form shear layer against the oracle replaying the lattice decisions
    of the same request stepped alone (1e-5)."""
    import time

    v64 = ("vortex fp64", dict(nx=64, ny=64, nu=1e-3, precision=alb.ALB_FP64_PLAIN),
           dict(nu=1e-3), flows.isentropic_vortex(), 45)
    sh = flows.FlowSpec("shear", 96, 64, 2.5, 3.0, 1e-4, 33, "fp32", seed=43)
    s32 = ("shear fp32", dict(nx=96, ny=64, nu=1e-4, precision=alb.ALB_FP32_FORM, sensor=1),
           dict(nu=1e-4, sensor=True), sh.fields(), 33)
    others = [flows.FlowSpec("vortex", 40, 40, 1.2, 2.0, 1e-3, 20, "fp32", seed=44),
              flows.FlowSpec("shear", 136, 24, 1.5, 2.0, 1e-5, 50, "fp32", seed=45),
              flows.FlowSpec("vortex", 49, 41, 1.0, 1.5, 1e-3, 15, "fp64", seed=46)]
    srv = alb.Server(chunk_ms=2.0, max_chunk=5)
    try:
        ids = [srv.submit(sp.steps, fields=sp.fields(), nx=sp.nx, ny=sp.ny, nu=sp.nu,
                          precision=alb.ALB_FP32_FORM if sp.precision == "fp32"
                          else alb.ALB_FP64_PLAIN)
               for sp in others[:2]]
        rv = srv.submit(v64[4], fields=v64[3], **v64[1])
        rs = srv.submit(s32[4], fields=s32[3], **s32[1])
        ids.append(srv.submit(others[2].steps, fields=others[2].fields(), nx=others[2].nx,
                              ny=others[2].ny, nu=others[2].nu, precision=alb.ALB_FP64_PLAIN))
        srv.drain(120000)
        results = {}
        for rid in [rv, rs] + ids:
            st, res = srv.poll(rid)
            assert st == alb.ALB_DONE and res["status"] == alb.ALB_OK, (rid, st, res)
            results[rid] = res
    finally:
        srv.close()
    # FP64 request: the free-running oracle
    name, c, okw, fld, steps = v64
    s = O.Simulation(O.make_config(c["nx"], c["ny"], **okw))
    assert s.init(*fld) == O.OK and s.step(steps) == O.OK
    res = results[rv]
    assert res["steps"] == steps
    assert rel_errors(res["moments"], s.moments()) <= FP64_TOL
    assert res["stats"]["reconstructions"] == s.stats()["reconstructions"] > 0
    # FP32 request: the oracle replays the lattice decisions of the request
    # stepped alone (served and alone are the same computation)
    name, c, okw, fld, steps = s32
    fl = alb.Flow(**c)
    fl.init(*fld)
    r = O.Simulation(O.make_config(c["nx"], c["ny"], **okw))
    assert r.init(*fld) == O.OK
    for _ in range(steps):
        fl.step(1)
        ux, uy = fl.shifts()
        assert r.step_forced(ux, uy) == O.OK
    fl.close()
    res = results[rs]
    assert res["steps"] == steps
    assert rel_errors(res["moments"], r.moments()) <= FP32_TOL

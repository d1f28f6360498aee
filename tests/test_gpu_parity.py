"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances: FP64 plain path 1e-11 relative on rho, rho*u and rho*E; FP32
form 1e-5 relative; lattice shifts bit-exact. The relative error of a field
is max_x |m - m_oracle| / max_x |m_oracle| (momentum as a vector norm).
"""
import numpy as np
import pytest

import oracle as O
from paper_2009_13426_gb300 import flows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5


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
    return {"rho": np.abs(r - R).max() / np.abs(R).max(), "mom": mom,
            "E": np.abs(e - E).max() / np.abs(E).max()}


def run_oracle(nx, ny, fields, steps, **kw):
    s = O.Simulation(O.make_config(nx, ny, **kw))
    assert s.init(*fields) == O.OK
    st = s.step(steps) if steps else O.OK
    return s, st


def run_replay(alb, nx, ny, fields, steps, precision, **kw):
    """GPU run step by step; the oracle replays the GPU's lattice decisions.

    In the FP32 form a node whose velocity lies within FP32 round-off of a
    shift threshold can pick the other lattice than the FP64 oracle would, and a
    lattice change moves that node by O(1e-4..1e-2) (every pull is rebuilt).
    Feeding the oracle the same decisions isolates the arithmetic; the decisions
    themselves are checked bit-exactly on identical moments elsewhere."""
    fl = run_gpu(alb, nx, ny, fields, 0, precision, **kw)
    okw = {k: v for k, v in kw.items() if k != "newton_start"}  # GPU-only option
    s = O.Simulation(O.make_config(nx, ny, **okw))
    assert s.init(*fields) == O.OK
    free = O.Simulation(O.make_config(nx, ny, **okw))
    assert free.init(*fields) == O.OK
    differs = 0
    for _ in range(steps):
        fl.step(1)
        ux, uy = fl.shifts()
        assert s.step_forced(ux, uy) == O.OK
        free.step(1)
        fx, fy = free.shifts()
        differs += int((fx != ux).sum() + (fy != uy).sum())
    fl.sync()
    return fl, s, differs


def run_gpu(alb, nx, ny, fields, steps, precision, **kw):
    okw = dict(kw)
    bc = {O.PERIODIC: alb.ALB_PERIODIC, O.ZERO_GRADIENT: alb.ALB_ZERO_GRADIENT}
    cfg = {"u_max": okw.pop("umax", 2), "precision": precision}
    if "bc_x" in okw:
        cfg["bc_x"] = bc[okw.pop("bc_x")]
    if "bc_y" in okw:
        cfg["bc_y"] = bc[okw.pop("bc_y")]
    if "sensor" in okw:
        cfg["sensor"] = int(okw.pop("sensor"))
    if "overlap" in okw:
        cfg["shift_overlap"] = okw.pop("overlap")
    if "overlap_rule" in okw:
        cfg["shift_rule"] = okw.pop("overlap_rule")
    cfg.update(okw)
    fl = alb.Flow(nx, ny, **cfg)
    fl.init(*fields)
    fl.step(steps)
    fl.sync()
    return fl


# --------------------------------------------------------------- equilibrium

def test_equilibrium_sweep_matches_oracle(alb):
    rng = np.random.default_rng(21)
    n = 10000
    rho = rng.uniform(0.05, 4.0, n)
    ang = rng.uniform(0, 2 * np.pi, n)
    mag = rng.uniform(0, 1.2, n)
    T = rng.uniform(0.4, 1.4, n)
    ubx, uby = mag * np.cos(ang), mag * np.sin(ang)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    feq = torch.empty(n * 21, dtype=torch.float64, device="cuda")
    lam = torch.empty(n * 8, dtype=torch.float64, device="cuda")
    its = torch.empty(n, dtype=torch.int32, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    alb.alb_equilibrium(dev(rho), dev(ubx), dev(uby), dev(T), n, 1e-12, 50, feq, lam, its, st)
    torch.cuda.synchronize()
    feq = feq.cpu().numpy().reshape(n, 21)
    st = st.cpu().numpy()
    its = its.cpu().numpy()
    mism = 0
    for k in range(n):
        ost, olam, ofeq, oit = O.equilibrium(rho[k], ubx[k], uby[k], T[k])
        assert (ost == O.OK) == (st[k] == 0), (k, ost, st[k])
        if ost == O.OK:
            np.testing.assert_allclose(feq[k], ofeq, rtol=1e-11, atol=1e-14 * rho[k])
            mism += int(oit != its[k])
    assert mism <= n // 100  # same Newton path almost everywhere


def test_shift_selection_bit_exact_including_ties(alb):
    rng = np.random.default_rng(3)
    base = np.concatenate([np.arange(-3.5, 3.51, 0.5), np.arange(-3.49, 3.5, 0.5),
                           np.arange(-3.51, 3.5, 0.5), rng.uniform(-4, 4, 5000)])
    eps = np.concatenate([base, np.nextafter(base, 10), np.nextafter(base, -10)])
    rho = rng.uniform(0.1, 3.0, eps.size)
    # rho*u chosen so that the FP64 division reproduces u exactly or lands next to it
    rhou = rho * eps
    for n0 in (0.5, 0.51):
        for umax in (2, 3):
            out = torch.empty(eps.size, dtype=torch.int8, device="cuda")
            alb.alb_select_shift(torch.tensor(rho, device="cuda", dtype=torch.float64),
                                 torch.tensor(rhou, device="cuda", dtype=torch.float64),
                                 eps.size, n0, umax, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            ref = np.array([O.select_shift(rhou[k] / rho[k], n0, umax) for k in range(eps.size)])
            assert (got == ref).all()


# --------------------------------------------------------------- whole flows

@pytest.fixture(scope="module")
def vortex_oracle():
    fields = flows.isentropic_vortex()
    s, st = run_oracle(64, 64, fields, 100, umax=2, nu=1e-3)
    assert st == O.OK
    return fields, s.moments(), s.shifts(), s.stats()


def test_vortex_fp64_plain_matches_oracle(alb, vortex_oracle):
    """64x64 periodic vortex at Mach 1.2, 100 steps, FP64 plain."""
    fields, ref, (rx, ry), ostats = vortex_oracle
    fl = run_gpu(alb, 64, 64, fields, 100, alb.ALB_FP64_PLAIN, umax=2, nu=1e-3)
    err = rel_errors(fl.moments(), ref)
    assert max(err.values()) <= FP64_TOL, err
    sx, sy = fl.shifts()
    assert (sx == rx).all() and (sy == ry).all()
    st = fl.stats()
    assert st["newton_failures"] == 0 and st["reconstruction_failures"] == 0
    assert st["reconstructions"] == ostats["reconstructions"]


def test_vortex_fp64_previous_start_matches_oracle(alb, vortex_oracle):
    """FP64 plain with every solve started from the previous step's
    multipliers (ALB_START_PREVIOUS): a different Newton path to the same
    unique root, fewer iterations, the same 1e-11 on the vortex."""
    fields, ref, (rx, ry), ostats = vortex_oracle
    cold = run_gpu(alb, 64, 64, fields, 100, alb.ALB_FP64_PLAIN, umax=2, nu=1e-3)
    fl = run_gpu(alb, 64, 64, fields, 100, alb.ALB_FP64_PLAIN, umax=2, nu=1e-3,
                 newton_start=alb.ALB_START_PREVIOUS)
    err = rel_errors(fl.moments(), ref)
    assert max(err.values()) <= FP64_TOL, err
    sx, sy = fl.shifts()
    assert (sx == rx).all() and (sy == ry).all()
    assert fl.stats()["newton_iterations"] < 0.7 * cold.stats()["newton_iterations"]


def test_vortex_fp32_maxwellian_start_matches_oracle(alb, vortex_oracle):
    fields = vortex_oracle[0]
    fl, s, _ = run_replay(alb, 64, 64, fields, 20, alb.ALB_FP32_FORM, umax=2, nu=1e-3,
                          newton_start=alb.ALB_START_MAXWELLIAN)
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= FP32_TOL, err


@pytest.mark.parametrize("rule", [O.RULE_HISTORY, O.RULE_NEIGHBOURS])
@pytest.mark.parametrize("precision", [0, 1])
def test_vortex_overlapping_ranges_match_oracle(alb, precision, rule):
    """Shift ranges widened by 0.5 (Sec. III.A.2), chosen by history or by the
    neighbourhood: FP64 plain against the free-running oracle (1e-11, shifts
    and rebuild counts equal), FP32 form with replayed decisions (1e-5)."""
    fields = flows.isentropic_vortex()
    kw = dict(umax=2, nu=1e-3, overlap=0.5, overlap_rule=rule)
    if precision == 0:
        s, st = run_oracle(64, 64, fields, 60, **kw)
        assert st == O.OK
        fl = run_gpu(alb, 64, 64, fields, 60, alb.ALB_FP64_PLAIN, **kw)
        sx, sy = fl.shifts()
        rx, ry = s.shifts()
        assert (sx == rx).all() and (sy == ry).all()
        tol = FP64_TOL
        assert fl.stats()["reconstructions"] == s.stats()["reconstructions"]
    else:
        fl, s, _ = run_replay(alb, 64, 64, fields, 60, alb.ALB_FP32_FORM, **kw)
        tol = FP32_TOL
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= tol, err


@pytest.mark.parametrize("precision", [0, 1])
def test_vortex_reduced_model_matches_oracle(alb, precision):
    """The reduced 4-moment equilibrium (App. C.2): FP64 plain against the
    free-running oracle (1e-11, shifts equal), FP32 form with replayed
    decisions (1e-5); 64^2 vortex, 60 steps."""
    fields = flows.isentropic_vortex()
    kw = dict(umax=2, nu=1e-3, moments=4)
    if precision == 0:
        s, st = run_oracle(64, 64, fields, 60, **kw)
        assert st == O.OK
        fl = run_gpu(alb, 64, 64, fields, 60, alb.ALB_FP64_PLAIN, **kw)
        sx, sy = fl.shifts()
        rx, ry = s.shifts()
        assert (sx == rx).all() and (sy == ry).all()
        assert fl.stats()["reconstructions"] == s.stats()["reconstructions"]
        tol = FP64_TOL
    else:
        fl, s, _ = run_replay(alb, 64, 64, fields, 60, alb.ALB_FP32_FORM, **kw)
        tol = FP32_TOL
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= tol, err


@pytest.mark.parametrize("precision", [0, 1])
def test_vortex_prandtl_matches_oracle(alb, precision):
    """Pr = 0.71 (App. E): the heat-flux term in every collision, kappa =
    rho Cp nu / Pr in the initial state and in Grad rebuilds, which carry the
    term too. 64^2 vortex at Mach 1.2, nu = 0.02, 60 steps: FP64 plain against
    the free-running oracle (1e-11, shifts and rebuild counts equal), FP32
    form with replayed decisions (1e-5). The flow differs from the Pr = 1 one
    by about 2 %."""
    fields = flows.isentropic_vortex()
    kw = dict(umax=2, nu=0.02, prandtl=0.71)
    if precision == 0:
        s, st = run_oracle(64, 64, fields, 60, **kw)
        assert st == O.OK
        fl = run_gpu(alb, 64, 64, fields, 60, alb.ALB_FP64_PLAIN, **kw)
        sx, sy = fl.shifts()
        rx, ry = s.shifts()
        assert (sx == rx).all() and (sy == ry).all()
        assert fl.stats()["reconstructions"] == s.stats()["reconstructions"]
        tol = FP64_TOL
    else:
        fl, s, _ = run_replay(alb, 64, 64, fields, 60, alb.ALB_FP32_FORM, **kw)
        tol = FP32_TOL
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= tol, err
    bgk = run_gpu(alb, 64, 64, fields, 60, precision, umax=2, nu=0.02)
    assert max(rel_errors(bgk.moments(), s.moments()).values()) > 1e-3


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_sod_prandtl_with_sensor_matches_oracle(alb, precision, tol):
    """Pr = 0.5 with the kinetic sensor (both relaxation times scaled by its
    factor) on a 512 x 4 Sod tube, zero-gradient x ends, 150 steps."""
    nx, ny, steps = 512, 4, 150
    fields = flows.riemann_1d(nx, ny)
    kw = dict(umax=2, nu=1e-3, bc_x=O.ZERO_GRADIENT, sensor=True, prandtl=0.5)
    if precision == 0:
        s, st = run_oracle(nx, ny, fields, steps, **kw)
        assert st == O.OK
        fl = run_gpu(alb, nx, ny, fields, steps, precision, **kw)
        sx, sy = fl.shifts()
        rx, ry = s.shifts()
        assert (sx == rx).all() and (sy == ry).all()
    else:
        fl, s, _ = run_replay(alb, nx, ny, fields, steps, precision, **kw)
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= tol, err


def test_neighbourhood_rule_at_zero_gradient_ends(alb):
    """The neighbourhood rule reads ghost neighbours through the boundary
    rule: a ragged grid with zero-gradient ends in x and y, FP64 plain."""
    nx, ny = 45, 29
    fields = flows.isentropic_vortex(nx, ny, strength=3.0, radius=5.0, mach=0.9, seed=7)
    kw = dict(umax=2, nu=1e-3, overlap=0.4, overlap_rule=O.RULE_NEIGHBOURS,
              bc_x=O.ZERO_GRADIENT, bc_y=O.ZERO_GRADIENT)
    s, st = run_oracle(nx, ny, fields, 30, **kw)
    fl = run_gpu(alb, nx, ny, fields, 30, alb.ALB_FP64_PLAIN, **kw)
    sx, sy = fl.shifts()
    rx, ry = s.shifts()
    assert (sx == rx).all() and (sy == ry).all()
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= FP64_TOL, err


def test_vortex_fp32_form_matches_oracle(alb, vortex_oracle):
    fields = vortex_oracle[0]
    fl, s, differs = run_replay(alb, 64, 64, fields, 100, alb.ALB_FP32_FORM, umax=2, nu=1e-3)
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= FP32_TOL, err
    # decisions that differ from a free FP64 run are rare (round-off at a threshold)
    assert differs <= 64 * 64 * 100 * 1e-4


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, FP32_TOL)])
def test_sod_tube_matches_oracle(alb, precision, tol):
    """Sod tube 2048x4, periodic in y, zero-gradient x ends, nu = 1e-4, sensor
    on, 1000 steps: FP32 form and FP64 plain against the oracle."""
    nx, ny, steps = 2048, 4, 1000
    fields = flows.riemann_1d(nx, ny)
    kw = dict(umax=2, nu=1e-4, bc_x=O.ZERO_GRADIENT, sensor=True)
    if precision == 0:
        s, st = run_oracle(nx, ny, fields, steps, **kw)
        assert st == O.OK
        fl = run_gpu(alb, nx, ny, fields, steps, precision, **kw)
        sx, sy = fl.shifts()
        rx, ry = s.shifts()
        assert (sx == rx).all() and (sy == ry).all()
    else:
        fl, s, differs = run_replay(alb, nx, ny, fields, steps, precision, **kw)
        # lattice decisions that differ from the free-running FP64 oracle's
        # (FP32 round-off at a threshold, then the runs part) stay rare
        print("\nSod FP32 form: %d differing lattice decisions in %d node-steps"
              % (differs, nx * ny * steps))
        assert differs <= nx * ny * steps * 1e-4
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= tol, err


@pytest.mark.parametrize("nx,ny,bcx,bcy,umax", [
    (37, 5, O.PERIODIC, O.PERIODIC, 2),          # ragged: not a multiple of the block
    (4, 4, O.PERIODIC, O.PERIODIC, 2),           # streams wrap several times around
    (130, 3, O.ZERO_GRADIENT, O.PERIODIC, 3),    # two blocks, ragged tail, u_max 3
    (20, 24, O.ZERO_GRADIENT, O.ZERO_GRADIENT, 1),
    (1, 1, O.PERIODIC, O.PERIODIC, 2),           # a single node
])
@pytest.mark.parametrize("precision", [0, 1])
def test_small_and_ragged_grids(alb, nx, ny, bcx, bcy, umax, precision):
    r, a, b, e = flows.isentropic_vortex(nx, ny, strength=3.0, radius=max(1.5, min(nx, ny) / 6),
                                         mach=0.9, seed=7)
    fields = (r, a, b, e)
    kw = dict(umax=umax, nu=2e-3, bc_x=bcx, bc_y=bcy)
    if precision == 0:
        s, st = run_oracle(nx, ny, fields, 12, **kw)
        assert st == O.OK
        fl = run_gpu(alb, nx, ny, fields, 12, precision, **kw)
    else:
        fl, s, _ = run_replay(alb, nx, ny, fields, 12, precision, **kw)
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= (FP64_TOL if precision == 0 else FP32_TOL), err


def test_zero_steps_returns_initial_moments(alb):
    fields = flows.isentropic_vortex(16, 16, radius=3.0)
    s, _ = run_oracle(16, 16, fields, 0)
    fl = run_gpu(alb, 16, 16, fields, 0, alb.ALB_FP64_PLAIN)
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= 1e-13, err


def test_unrealizable_initial_state_is_reported(alb):
    r, a, b, e = flows.uniform(8, 8)
    r = r.copy()
    r[3, 3] = -1.0
    fl = alb.Flow(8, 8)
    with pytest.raises(alb.AlbError) as ei:
        fl.init(r, a, b, e)
    assert ei.value.code == alb.ALB_EUNREALIZABLE
    e2 = e.copy()
    e2[2, 2] = 0.0  # T < 0
    with pytest.raises(alb.AlbError) as ei:
        fl.init(flows.uniform(8, 8)[0], a, b, e2)
    assert ei.value.code == alb.ALB_EUNREALIZABLE
    # the context is still usable afterwards
    fl.init(*flows.uniform(8, 8))
    fl.step(2)
    fl.sync()


def test_device_pointer_init_and_moments(alb):
    fields = flows.isentropic_vortex(32, 32, radius=4.0)
    host = run_gpu(alb, 32, 32, fields, 7, alb.ALB_FP64_PLAIN)
    dev = [torch.tensor(f, dtype=torch.float64, device="cuda").contiguous() for f in fields]
    fl = alb.Flow(32, 32)
    fl.init(*dev)
    fl.step(7)
    out = [torch.empty(32 * 32, dtype=torch.float64, device="cuda") for _ in range(4)]
    alb.alb_moments(fl.h, out)
    torch.cuda.synchronize()
    for a, b in zip(out, host.moments()):
        assert np.array_equal(a.cpu().numpy().reshape(32, 32), b)


# --------------------------------------------------------------- global totals

@pytest.mark.parametrize("precision", [0, 1])
def test_totals_match_host_sums(alb, precision):
    """alb_totals equals the sums of the exported fields; two chunks plus a
    ragged tail (300 x 300 = 90000 nodes, chunks of 65536)."""
    fields = flows.isentropic_vortex(300, 300, radius=20.0, mach=0.8)
    fl = run_gpu(alb, 300, 300, fields, 5, precision)
    tot = fl.totals()
    ref = np.array([m.sum() for m in fl.moments()])
    np.testing.assert_allclose(tot, ref, rtol=1e-12)
    assert np.array_equal(tot, fl.totals())  # deterministic


def test_totals_conserved_without_lattice_changes(alb):
    """Collision and plain streaming conserve mass, momentum and energy: with
    no lattice change (no rebuild) the totals drift only by the Newton
    tolerance per node and step."""
    n = 96
    fields = flows.isentropic_vortex(n, n, strength=1.0, radius=8.0, mach=0.0, noise=0.0)
    fl = alb.Flow(n, n, nu=1e-2)
    fl.init(*fields)
    t0 = fl.totals()
    fl.step(30)
    fl.sync()
    assert fl.stats()["reconstructions"] == 0
    t1 = fl.totals()
    assert abs(t1[0] - t0[0]) <= 30 * 1e-12 * t0[0]
    assert abs(t1[3] - t0[3]) <= 30 * 1e-12 * t0[3]
    assert abs(t1[1] - t0[1]) <= 30 * 1e-12 * t0[0]

"""The reference solver on the GPU (App. C.1): D2Q49 with the 13-moment
equilibrium, through the C ABI, against the oracle. FP64 throughout;
tolerance 1e-11 relative on rho, rho*u and rho*E, lattice shifts equal."""
import numpy as np
import pytest

import oracle as O
from paper_2009_13426_gb300 import flows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11


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


def both(alb, nx, ny, fields, steps, **kw):
    okw = dict(kw)
    s = O.Simulation(O.make_config(nx, ny, stencil=O.D2Q49, **okw))
    assert s.init(*fields) == O.OK
    assert s.step(steps) == O.OK
    bc = {O.PERIODIC: alb.ALB_PERIODIC, O.ZERO_GRADIENT: alb.ALB_ZERO_GRADIENT}
    cfg = dict(stencil=alb.ALB_D2Q49, moments=13, precision=alb.ALB_FP64_PLAIN,
               u_max=okw.pop("umax", 2))
    for k in ("bc_x", "bc_y"):
        if k in okw:
            cfg[k] = bc[okw.pop(k)]
    if "sensor" in okw:
        cfg["sensor"] = int(okw.pop("sensor"))
    if "overlap" in okw:
        cfg["shift_overlap"] = okw.pop("overlap")
    if "overlap_rule" in okw:
        cfg["shift_rule"] = okw.pop("overlap_rule")
    cfg.update(okw)
    fl = alb.Flow(nx, ny, **cfg)
    assert fl.init(*fields) == alb.ALB_OK
    fl.step(steps)
    fl.sync()
    return fl, s


def check(fl, s, rebuilds=True):
    err = rel_errors(fl.moments(), s.moments())
    assert max(err.values()) <= TOL, err
    sx, sy = fl.shifts()
    rx, ry = s.shifts()
    assert (sx == rx).all() and (sy == ry).all()
    st, ost = fl.stats(), s.stats()
    assert st["newton_failures"] == 0 and st["reconstruction_failures"] == 0
    assert st["reconstructions"] == ost["reconstructions"]
    if rebuilds:
        assert st["reconstructions"] > 0


def test_equilibrium13_sweep_matches_oracle(alb):
    rng = np.random.default_rng(31)
    n = 3000
    rho = rng.uniform(0.05, 4.0, n)
    ang = rng.uniform(0, 2 * np.pi, n)
    mag = rng.uniform(0, 1.0, n)
    T = rng.uniform(0.5, 1.2, n)
    ubx, uby = mag * np.cos(ang), mag * np.sin(ang)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    feq = torch.empty(n * 49, dtype=torch.float64, device="cuda")
    lam = torch.empty(n * 13, dtype=torch.float64, device="cuda")
    its = torch.empty(n, dtype=torch.int32, device="cuda")
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    alb.alb_equilibrium13(dev(rho), dev(ubx), dev(uby), dev(T), n, 1e-12, 50, feq, lam, its, st)
    torch.cuda.synchronize()
    feq = feq.cpu().numpy().reshape(n, 49)
    st = st.cpu().numpy()
    lam = lam.cpu().numpy().reshape(n, 13)
    converged = 0
    for k in range(n):
        ost, olam, ofeq, oit = O.equilibrium13(rho[k], ubx[k], uby[k], T[k])
        assert (ost == O.OK) == (st[k] == 0), (k, ost, st[k])
        if ost == O.OK:
            converged += 1
            np.testing.assert_allclose(feq[k], ofeq, rtol=1e-11, atol=1e-14 * rho[k])
            # the multipliers are less well conditioned than the populations
            np.testing.assert_allclose(lam[k], olam, rtol=1e-6, atol=1e-7)
    assert converged > 0.9 * n


def test_velocity_table(alb):
    x, y = alb.alb_stencil_velocities(alb.ALB_D2Q49)
    ox, oy = O.velocities(O.D2Q49)
    assert (x == ox).all() and (y == oy).all()


def test_vortex_matches_oracle(alb):
    """48^2 periodic vortex carried at Mach 1.2, 40 steps: lattice changes
    and Grad rebuilds on D2Q49."""
    fields = flows.isentropic_vortex(48, 48, radius=5.0, mach=1.2, seed=2)
    fl, s = both(alb, 48, 48, fields, 40, umax=2, nu=1e-3)
    check(fl, s)


def test_sod_with_sensor_and_zero_gradient_ends(alb):
    fields = flows.riemann_1d(256, 4)
    fl, s = both(alb, 256, 4, fields, 100, umax=2, nu=1e-4, bc_x=O.ZERO_GRADIENT, sensor=True)
    check(fl, s)


def test_prandtl_and_overlapping_ranges(alb):
    """App. E collision (Pr = 0.71) with shift ranges widened by 0.4 and
    chosen by history, on a ragged grid."""
    fields = flows.isentropic_vortex(37, 29, strength=3.0, radius=4.0, mach=1.0, seed=5)
    fl, s = both(alb, 37, 29, fields, 30, umax=2, nu=0.02, prandtl=0.71, overlap=0.4)
    check(fl, s)


def test_neighbourhood_rule_at_zero_gradient_ends(alb):
    fields = flows.isentropic_vortex(45, 29, strength=3.0, radius=5.0, mach=0.9, seed=7)
    fl, s = both(alb, 45, 29, fields, 25, umax=2, nu=1e-3, overlap=0.4,
                 overlap_rule=O.RULE_NEIGHBOURS, bc_x=O.ZERO_GRADIENT, bc_y=O.ZERO_GRADIENT)
    check(fl, s)


def test_exports_and_checkpoint(alb):
    nx, ny = 24, 16
    fields = flows.isentropic_vortex(nx, ny, radius=4.0, mach=1.1, seed=4)
    a = alb.Flow(nx, ny, stencil=alb.ALB_D2Q49, moments=13, nu=1e-3)
    a.init(*fields)
    a.step(3)
    f, g = a.populations()
    assert f.shape == (49, ny, nx) and g.shape == (49, ny, nx)
    # the exported populations carry the stored moments (the collision keeps
    # them to the Newton tolerance)
    x, y = alb.alb_stencil_velocities(alb.ALB_D2Q49)
    sx, sy = a.shifts()
    R, A, _, _ = a.moments()
    np.testing.assert_allclose(f.sum(0), R, rtol=5e-12)
    cx = x[:, None, None] + sx[None].astype(np.float64)
    np.testing.assert_allclose((f * cx).sum(0), A, rtol=1e-11, atol=1e-11)
    img = a.checkpoint()
    a.step(4)
    ref = a.moments()
    b = alb.Flow(nx, ny, stencil=alb.ALB_D2Q49, moments=13, nu=1e-3)
    b.restore(img)
    b.step(4)
    for u, v in zip(b.moments(), ref):
        assert np.array_equal(u, v)
    c = alb.Flow(nx, ny, nu=1e-3)  # D2Q21 flow of the same size
    with pytest.raises(alb.AlbError):
        c.restore(img)


def test_batches_and_server_refuse_d2q49(alb):
    with pytest.raises(alb.AlbError) as ei:
        alb.Batch([dict(nx=16, ny=16, stencil=alb.ALB_D2Q49, moments=13)])
    assert ei.value.code == alb.ALB_EUNSUPPORTED

"""The paper's validation cases (Sec. IV.B, IV.C) on the GPU: inviscid
(nu = 0) transport with shifts up to 3, compared with the oracle and with
what the paper prints or shows, and the 2D Riemann problem. The paper's figures
come from its own implementation; the bands below are loose (same order),
the oracle comparison is the gate.

Half-integer mean velocities sit on a criterion threshold; the runs use the
offset n0 = 0.51 the paper gives for such cases (Sec. III.A.2, Fig. 7)."""
import numpy as np
import pytest

import oracle as O
from paper_2009_13426_gb300 import flows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

A = 1e-3
T0 = 0.7


@pytest.fixture(scope="module")
def alb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13426_gb300 import alb as A_
    A_.lib()
    return A_


def run(alb, nx, ny, fields, steps, precision=0):
    fl = alb.Flow(nx, ny, precision=precision, u_max=3, nu=0.0, n0=0.51)
    assert fl.init(*fields) == alb.ALB_OK
    fl.step(steps)
    fl.sync()
    return fl


# u0, steps to t = 15 L / u0 with L = 100, the paper's dissipation
SHEAR = [(2.0, 750, 0.003), (2.5, 600, 0.009), (3.0, 500, 0.007)]


@pytest.mark.parametrize("u0,steps,paper", SHEAR)
def test_shear_wave(alb, u0, steps, paper):
    """Sec. IV.B.1: 100 x 1 shear wave, A = 1e-3, T0 = 0.7; numerical
    dissipation |max(u_y^ref) - max(u_y)| / max(u_y^ref) at t = 15 t_c."""
    fields = flows.shear_wave(100, 1, u0, amp=A, T0=T0)
    fl = run(alb, 100, 1, fields, steps)
    r, jx, jy, E = fl.moments()
    sx, _ = fl.shifts()
    assert (sx == sx.flat[0]).all()  # the lattice adjusts once and stays
    nu_num = abs(A - (jy / r).max()) / A
    assert nu_num < 5 * max(paper, 0.004), nu_num
    s = O.Simulation(O.make_config(100, 1, umax=3, nu=0.0, n0=0.51))
    assert s.init(*fields) == O.OK
    assert s.step(steps) == O.OK
    R, JX, JY, EE = s.moments()
    # the parity metric of the other tests: momentum as a vector
    mom = np.sqrt((jx - JX) ** 2 + (jy - JY) ** 2).max() / np.sqrt(JX ** 2 + JY ** 2).max()
    assert mom <= 1e-11
    for a, b in ((r, R), (E, EE)):
        assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max()


@pytest.mark.parametrize("u0,steps,paper", [(2.0, 750, 0.012), (2.5, 600, 0.009),
                                            (3.0, 500, 0.012)])
def test_entropy_spot(alb, u0, steps, paper):
    """Sec. IV.B.2: 100 x 100 Gaussian hot spot (R = L/10) at constant
    pressure, FP64 plain as in the paper; loss of the temperature peak at
    t = 15 t_c (paper: about 1 %), and the spot returns to its centre.

    The FP32 form is not run here: with nu = 0 the BGK relaxation reflects the
    non-equilibrium part (omega = 2) and nothing damps it, and at a relative
    velocity of 0.5 (u0 = 2.5 in lattice 3) a slowly growing mode seeded by
    FP32 round-off reaches the size of the 1e-3 perturbation within the 600
    steps; FP64 round-off keeps it invisible."""
    fields = flows.entropy_spot(100, u0, amp=A, T0=T0)
    fl = run(alb, 100, 100, fields, steps, 0)
    r, jx, jy, E = fl.moments()
    ux, uy = jx / r, jy / r
    T = (E / r - 0.5 * (ux ** 2 + uy ** 2)) / 2.5   # Cv = 1/(gamma - 1)
    dT = T - T0
    loss = abs(A * T0 - dT.max()) / (A * T0)
    assert loss < 3.0 * paper, loss
    iy, ix = np.unravel_index(np.argmax(dT), dT.shape)
    assert abs(ix - 50) <= 1 and abs(iy - 50) <= 1


def test_acoustic_pulse_is_galilean(alb):
    """Sec. IV.B.3: 100 x 100 isentropic pressure pulse (A = 1e-3, R = L/10)
    carried at u0 = 0.3, 1.6 and 2.9 (lattices 0, 2, 3). After 30 iterations
    the pressure field moved back by u0 x 30 nodes matches the one at rest
    (the paper shows the profiles overlapping; the oracle differs by 7e-4 of
    the amplitude), and the run at 2.9 matches the oracle."""
    ref = None
    for u0 in (0.0, 0.3, 1.6, 2.9):
        fields = flows.acoustic_pulse(100, u0, amp=A, T0=T0)
        fl = run(alb, 100, 100, fields, 30)
        r, jx, jy, E = fl.moments()
        T = (E / r - 0.5 * ((jx / r) ** 2 + (jy / r) ** 2)) / 2.5
        dP = np.roll((r * T - T0) / (A * T0), -int(round(u0 * 30)), axis=1)
        if ref is None:
            ref = dP
            assert dP.max() > 0.1
        else:
            assert np.abs(dP - ref).max() < 5e-3, (u0, np.abs(dP - ref).max())
    s = O.Simulation(O.make_config(100, 100, umax=3, nu=0.0, n0=0.51))
    assert s.init(*fields) == O.OK
    assert s.step(30) == O.OK
    R, JX, JY, EE = s.moments()
    mom = np.sqrt((jx - JX) ** 2 + (jy - JY) ** 2).max() / np.sqrt(JX ** 2 + JY ** 2).max()
    assert mom <= 1e-11
    for a, b in ((r, R), (E, EE)):
        assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max()


def test_riemann_2d(alb):
    """Sec. IV.C.2, Tab. 1: the four-quadrant Riemann problem on 200 x 200
    (zero-gradient ends, nu = 0, sensor on), 120 steps, FP64 plain: equal to
    the oracle (1e-11, shifts equal), symmetric about the diagonal x = y, and
    with the lattices the paper reports - (0,0), (1,0), (0,1), the (1,1) that
    appears upstream of the shocks' intersection, and the negative shifts
    (-1,0), (0,-1), (-1,-1) inside the dipole."""
    n = 200
    fields = flows.riemann_2d(n)
    fl = alb.Flow(n, n, precision=0, u_max=2, nu=0.0, sensor=1, bc_x=alb.ALB_ZERO_GRADIENT,
                  bc_y=alb.ALB_ZERO_GRADIENT)
    assert fl.init(*fields) == alb.ALB_OK
    fl.step(120)
    fl.sync()
    r, jx, jy, E = fl.moments()
    sx, sy = fl.shifts()
    assert np.abs(r - r.T).max() <= 1e-12 * np.abs(r).max()
    lattices = set(zip(sx.ravel().tolist(), sy.ravel().tolist()))
    assert {(0, 0), (1, 0), (0, 1), (1, 1), (-1, 0), (0, -1), (-1, -1)} <= lattices
    s = O.Simulation(O.make_config(n, n, umax=2, nu=0.0, sensor=True, bc_x=O.ZERO_GRADIENT,
                                   bc_y=O.ZERO_GRADIENT))
    assert s.init(*fields) == O.OK
    assert s.step(120) == O.OK
    rx, ry = s.shifts()
    assert (sx == rx).all() and (sy == ry).all()
    R, JX, JY, EE = s.moments()
    mom = np.sqrt((jx - JX) ** 2 + (jy - JY) ** 2).max() / np.sqrt(JX ** 2 + JY ** 2).max()
    assert mom <= 1e-11
    for a, b in ((r, R), (E, EE)):
        assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max()

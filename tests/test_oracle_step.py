"""Pins of the oracle's moments, shift criterion, collision, streaming and
Grad reconstruction against invariants, closed forms and printed examples."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from oracle import riemann
from paper_2009_13426_gb300 import flows

GAMMA = 1.4
CV = 1.0 / (GAMMA - 1.0)


def _xi():
    x, y = O.velocities()
    return x.astype(np.int64), y.astype(np.int64)


# ---------------------------------------------------------------- moments

def test_node_moments_exact_rational_bruteforce():
    """Eq. polyTemp evaluated in exact rational arithmetic with the absolute
    velocities c_i = xi_i + U, against the oracle's lattice-frame sums."""
    rng = np.random.default_rng(5)
    x, y = _xi()
    for _ in range(40):
        f = rng.uniform(0.01, 0.3, 21)
        g = rng.uniform(0.01, 0.5, 21)
        Ux, Uy = (int(v) for v in rng.integers(-2, 3, 2))
        F = [Fraction(v) for v in f]
        G = [Fraction(v) for v in g]
        cx = [int(a) + Ux for a in x]
        cy = [int(b) + Uy for b in y]
        rho = sum(F)
        jx = sum(fi * c for fi, c in zip(F, cx))
        jy = sum(fi * c for fi, c in zip(F, cy))
        e = sum((a * a + b * b) * fi + gi for fi, gi, a, b in zip(F, G, cx, cy))
        ux, uy = jx / rho, jy / rho
        T = (e - rho * (ux * ux + uy * uy)) / (2 * rho * Fraction(CV))
        got = O.node_moments(f, g, Ux, Uy, GAMMA)
        np.testing.assert_allclose(got, [float(rho), float(ux), float(uy), float(T)], rtol=1e-14,
                                   atol=1e-14)


# ---------------------------------------------------------------- criterion

@pytest.mark.parametrize("u,expect", [
    # Sec. III.A.2 examples: (-0.5,-0.5) < u <= (0.5,0.5) -> 0; (-1.5,-0.5) < u <= (-0.5, 0.5)
    # -> (-1, 0); (0.5, 0.5) < u <= (1.5, 1.5) -> (1, 1)
    (0.0, 0), (0.5, 0), (-0.4999999, 0), (-0.5, -1), (-1.5, -2), (-1.4999, -1),
    (0.5000001, 1), (1.5, 1), (1.5000001, 2), (2.5, 2), (7.0, 2), (-9.0, -2), (-2.5, -2),
])
def test_shift_criterion(u, expect):
    assert O.select_shift(u, 0.5, 2) == expect


@pytest.mark.parametrize("u,expect", [(0.49, 0), (0.4900001, 1), (-0.51, -1), (-0.5, 0),
                                      (1.49, 1), (1.4900001, 2)])
def test_shift_criterion_offset(u, expect):
    """n0 = 0.51 (Fig. 7 caption) read as U = n iff n - n0 < u <= n + 1 - n0."""
    assert O.select_shift(u, 0.51, 2) == expect


def test_shift_criterion_paper_figure_examples():
    for (ux, uy), (ex, ey) in [((0.5, 0.5), (0, 0)), ((-0.3, 0.2), (0, 0)),
                               ((-1.5 + 1e-9, 0.5), (-1, 0)), ((-0.5, -0.5 + 1e-9), (-1, 0)),
                               ((1.5, 1.5), (1, 1)), ((0.5 + 1e-9, 0.5 + 1e-9), (1, 1))]:
        assert (O.select_shift(ux), O.select_shift(uy)) == (ex, ey)


# ---------------------------------------------------------------- collision

@pytest.mark.parametrize("moments", [8, 4])
@pytest.mark.parametrize("sensor", [False, True])
def test_collision_conserves_mass_momentum_energy(sensor, moments):
    """Both constraint sets fix mass, momentum and the energy trace, so the
    collision conserves mass, momentum and total energy with either."""
    rng = np.random.default_rng(9)
    cfg = O.make_config(4, 4, nu=1e-3, sensor=sensor, moments=moments)
    x, y = _xi()
    for _ in range(25):
        Ux, Uy = (int(v) for v in rng.integers(-2, 3, 2))
        rho = rng.uniform(0.2, 2.0)
        T = rng.uniform(0.5, 1.2)
        ub = rng.uniform(-0.5, 0.5, 2)
        st, lam, feq, _ = O.equilibrium(rho, ub[0], ub[1], T)
        f = feq * (1 + 0.05 * rng.standard_normal(21))
        g = 3 * T * feq * (1 + 0.05 * rng.standard_normal(21))
        st, fs, gs = O.collide_node(cfg, f, g, Ux, Uy)
        assert st == O.OK
        cx, cy = x + Ux, y + Uy
        c2 = cx * cx + cy * cy
        for a, b in ((f, fs), (f * cx, fs * cx), (f * cy, fs * cy)):
            assert abs(a.sum() - b.sum()) <= 1e-13 * np.abs(f).sum() * 10
        e0 = (c2 * f + g).sum()
        e1 = (c2 * fs + gs).sum()
        assert abs(e0 - e1) <= 1e-13 * e0 * 10


def test_collision_relaxes_towards_equilibrium_at_rate_one_over_tau():
    cfg = O.make_config(4, 4, nu=0.05)
    st, lam, feq, _ = O.equilibrium(1.0, 0.1, -0.2, 0.8)
    rng = np.random.default_rng(2)
    f = feq * (1 + 0.01 * rng.standard_normal(21))
    # restore the moments of f to those of feq so that f^eq(f) = feq exactly in
    # the limit; instead compare with the definition using the oracle's own feq
    g = 3 * 0.8 * feq
    st, fs, gs = O.collide_node(cfg, f, g, 0, 0)
    mom = O.node_moments(f, g, 0, 0)
    st, lam2, feq2, _ = O.equilibrium(mom[0], mom[1], mom[2], mom[3])
    tau = 0.5 + 0.05 / mom[3]
    np.testing.assert_allclose(fs, f - (f - feq2) / tau, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(gs, g - (g - 3 * mom[3] * feq2) / tau, rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------- Grad

def test_grad_zero_gradient_is_equilibrium():
    cfg = O.make_config(4, 4, nu=1e-2)
    st, f, g = O.grad_populations(cfg, 1, 0, 0.8, 1.3, 0.1, 0.7, np.zeros((2, 2)), np.zeros(2), 1.0)
    st2, lam, feq, _ = O.equilibrium(0.8, 1.3 - 1, 0.1, 0.7)
    np.testing.assert_allclose(f, feq, rtol=1e-15)
    np.testing.assert_allclose(g, 3 * 0.7 * feq, rtol=1e-15)


def test_grad_correction_is_mass_neutral_and_linear():
    """sum f^eq phi_f = 0 (traceless sigma, zero third central trace moment of the
    8-moment equilibrium) and sum g^eq phi_g = 0 (zero first central moment)."""
    rng = np.random.default_rng(4)
    cfg = O.make_config(4, 4, nu=2e-2)
    for _ in range(10):
        du = rng.normal(0, 0.02, (2, 2))
        dT = rng.normal(0, 0.02, 2)
        rho, T = rng.uniform(0.5, 1.5), rng.uniform(0.5, 1.0)
        u = rng.uniform(-0.4, 0.4, 2) + np.array([1.0, 0.0])
        st, f1, g1 = O.grad_populations(cfg, 1, 0, rho, u[0], u[1], T, du, dT, 1.0)
        st, f0, g0 = O.grad_populations(cfg, 1, 0, rho, u[0], u[1], T, du * 0, dT * 0, 1.0)
        st, fh, gh = O.grad_populations(cfg, 1, 0, rho, u[0], u[1], T, du, dT, 0.5)
        assert abs((f1 - f0).sum()) < 1e-14 * rho * 10
        assert abs((g1 - g0).sum()) < 1e-14 * rho * 10
        np.testing.assert_allclose(fh - f0, 0.5 * (f1 - f0), rtol=1e-10, atol=1e-16)


def test_grad_stress_term_exact_at_rest():
    """At rest, with only d_x u_y != 0, Eq. GradGeneral_f reduces to
    phi_f = sigma_xy xi_x xi_y / (rho T^2) with sigma_xy = -rho nu d_x u_y, so the
    rebuilt shear stress is sigma_xy * sum f^eq xi_x^2 xi_y^2 / (rho T^2) exactly.
    This pins the sign of sigma, mu = rho nu and the 1/(2 rho T^2) factor."""
    nu, rho, T, s = 0.05, 1.0, 0.7, 0.01
    cfg = O.make_config(4, 4, nu=nu)
    du = np.array([[0.0, s], [0.0, 0.0]])  # du[a][b] = d_a u_b: d_x u_y = s
    st, f1, g1 = O.grad_populations(cfg, 0, 0, rho, 0.0, 0.0, T, du, np.zeros(2), 1.0)
    st, f0, g0 = O.grad_populations(cfg, 0, 0, rho, 0.0, 0.0, T, du * 0, np.zeros(2), 1.0)
    x, y = _xi()
    pixy = ((f1 - f0) * x * y).sum()
    sigma_xy = -rho * nu * s
    m22 = (f0 * x * x * y * y).sum()
    assert abs(pixy - sigma_xy * m22 / (rho * T * T)) < 1e-15
    # normal stresses vanish for a pure shear, g is untouched without heat flux
    assert abs(((f1 - f0) * x * x).sum()) < 1e-15 and abs((g1 - g0).sum()) < 1e-15


@pytest.mark.parametrize("gamma", [1.4, 2.0])
@pytest.mark.parametrize("T", [0.6, 1.0])
def test_grad_heat_flux_term_exact_at_rest(gamma, T):
    """At rest with only a temperature gradient, Eqs. GradGeneral_f/_g give
    f - f^eq = f^eq q.xi/(rho Cp T^2) (|xi|^2/(2T) - Cp) and g - g^eq =
    g^eq 2 q.xi/(rho Cp), q = -kappa grad T, kappa = rho Cp nu. Their
    momentum and heat flux are then fixed by the equilibrium's moments
    M2, M4, M6 = sum f^eq xi_x^2 |xi|^{0,2,4} (symmetric lattice at rest):
    momentum q (M4/(2T) - Cp M2) / (rho Cp T^2), heat flux
    q [(M6/(2T) - Cp M4) / (2 rho Cp T^2) + (2 Cv - 2) T M2 / (rho Cp)];
    no mass and no energy. This pins the sign of q, kappa, and every factor
    of the two heat-flux terms."""
    nu, rho = 0.05, 1.1
    cv = 1.0 / (gamma - 1.0)
    cp = gamma * cv
    cfg = O.make_config(4, 4, nu=nu, gamma=gamma)
    dT = np.array([0.02, -0.013])
    st, f1, g1 = O.grad_populations(cfg, 0, 0, rho, 0.0, 0.0, T, np.zeros((2, 2)), dT, 1.0)
    st, f0, g0 = O.grad_populations(cfg, 0, 0, rho, 0.0, 0.0, T, np.zeros((2, 2)), 0 * dT, 1.0)
    assert st == O.OK
    x, y = _xi()
    c2 = x * x + y * y
    M2, M4, M6 = (f0 * x * x).sum(), (f0 * x * x * c2).sum(), (f0 * x * x * c2 * c2).sum()
    q = -rho * cp * nu * dT
    df, dg = f1 - f0, g1 - g0
    k_mom = (M4 / (2 * T) - cp * M2) / (rho * cp * T * T)
    k_q = (M6 / (2 * T) - cp * M4) / (2 * rho * cp * T * T) + (2 * cv - 2) * T * M2 / (rho * cp)
    tol = 1e-13 * np.abs(q).max()
    assert abs(df.sum()) < tol and abs(dg.sum()) < tol
    assert abs(0.5 * (c2 * df + dg).sum()) < tol
    for a, xa in ((0, x), (1, y)):
        assert abs((df * xa).sum() - q[a] * k_mom) < tol
        assert abs(0.5 * (xa * (c2 * df + dg)).sum() - q[a] * k_q) < tol


# ---------------------------------------------------------------- streaming

def _smooth(n, ux0=0.0, uy0=0.0):
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    k = 2 * math.pi / n
    rho = 1.0 + 0.01 * np.sin(k * xx)
    ux = ux0 + 0.05 * np.sin(k * yy)
    uy = uy0 + 0.03 * np.cos(k * xx)
    T = 0.7 + 0.01 * np.cos(k * (xx + yy))
    return rho, ux, uy, T


def test_galilean_translation_by_integer_shift():
    """A flow carried by an integer velocity U, with every node in lattice U,
    equals the rest-frame flow translated by n U after n steps (Sec. A: the
    shifted lattice c = xi + U is a change of reference frame)."""
    n, steps, U = 16, 6, (1, -2)
    r, ux, uy, T = _smooth(n)
    cfg = O.make_config(n, n, nu=5e-3)
    a = O.Simulation(cfg)
    assert a.init(*flows.conserved(r, ux, uy, T)) == O.OK
    b = O.Simulation(cfg)
    assert b.init(*flows.conserved(r, ux + U[0], uy + U[1], T)) == O.OK
    assert a.step(steps) == O.OK and b.step(steps) == O.OK
    sa = a.shifts()
    sb = b.shifts()
    assert (sa[0] == 0).all() and (sa[1] == 0).all()
    assert (sb[0] == U[0]).all() and (sb[1] == U[1]).all()
    pa = a.primitives()
    pb = b.primitives()
    roll = lambda F: np.roll(F, (steps * U[1], steps * U[0]), axis=(0, 1))
    np.testing.assert_allclose(pb[0], roll(pa[0]), rtol=1e-12)
    np.testing.assert_allclose(pb[1] - U[0], roll(pa[1]), atol=1e-12)
    np.testing.assert_allclose(pb[2] - U[1], roll(pa[2]), atol=1e-12)
    np.testing.assert_allclose(pb[3], roll(pa[3]), rtol=1e-12)


def test_pull_direction_carries_a_density_bump_downstream():
    n = 40
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    rho = 1.0 + 1e-3 * np.exp(-((xx - 10) ** 2 + (yy - 20) ** 2) / 9.0)
    T = 0.7 / rho  # constant pressure: entropy spot, advected with the flow
    cfg = O.make_config(n, n, nu=1e-3)
    s = O.Simulation(cfg)
    assert s.init(*flows.conserved(rho, np.full_like(rho, 0.3), np.full_like(rho, -0.2), T)) == O.OK
    assert s.step(30) == O.OK
    r = s.primitives()[0] - 1.0
    cx = (r * xx).sum() / r.sum()
    cy = (r * yy).sum() / r.sum()
    assert abs(cx - (10 + 0.3 * 30)) < 0.5 and abs(cy - (20 - 0.2 * 30)) < 0.5


@pytest.mark.parametrize("U", [(0, 0), (2, 1)])
def test_uniform_state_is_steady(U):
    cfg = O.make_config(8, 8, nu=1e-3)
    s = O.Simulation(cfg)
    rho, ux, uy, T = 0.9, U[0] + 0.3, U[1] - 0.25, 0.8
    assert s.init(*flows.uniform(8, 8, rho, ux, uy, T)) == O.OK
    assert s.step(5) == O.OK
    p = s.primitives()
    np.testing.assert_allclose(p[0], rho, rtol=1e-13)
    np.testing.assert_allclose(p[1], ux, atol=1e-13)
    np.testing.assert_allclose(p[2], uy, atol=1e-13)
    np.testing.assert_allclose(p[3], T, rtol=1e-13)
    st = s.stats()
    assert st["reconstructions"] == 0


def test_uniform_flow_across_forced_lattice_change_stays_uniform():
    """Nodes initialised in a lattice that the criterion then leaves: every pull
    is rebuilt, and with zero gradients the rebuild is the equilibrium, so a
    uniform state stays uniform (to Newton tolerance)."""
    n = 8
    cfg = O.make_config(n, n, nu=1e-3)
    s = O.Simulation(cfg)
    rho, ux, uy, T = 1.0, 0.7, 0.0, 0.7
    assert s.init(*flows.uniform(n, n, rho, ux, uy, T)) == O.OK
    f, g = s.populations()
    # re-express a checkerboard of nodes in lattice U = 0 with the same moments
    st, lam, feq0, _ = O.equilibrium(rho, ux, uy, T)
    Ux, Uy = s.shifts()
    Ux = Ux.copy()
    mask = (np.add.outer(np.arange(n), np.arange(n)) % 2) == 0
    f[mask] = feq0
    g[mask] = 3 * T * feq0
    Ux[mask] = 0
    s.set_state(f, g, Ux, Uy)
    assert s.step(3) == O.OK
    assert s.stats()["reconstructions"] > 0
    p = s.primitives()
    np.testing.assert_allclose(p[0], rho, rtol=1e-11)
    np.testing.assert_allclose(p[1], ux, atol=1e-11)
    np.testing.assert_allclose(p[3], T, rtol=1e-11)
    assert (s.shifts()[0] == 1).all()


def test_periodic_vortex_conserves_mass_without_interfaces():
    """Collision and plain streaming conserve global mass, momentum and energy
    when no lattice changes (all nodes stay in lattice 0), up to the root
    finder's tolerance: each collision may leave |G_k| <= 1e-12 rho, so after
    n steps the totals agree to about n * 1e-12 relative."""
    n = 24
    r, a, b, e = flows.isentropic_vortex(n, n, strength=1.0, radius=4.0, mach=0.0, noise=0.0)
    cfg = O.make_config(n, n, nu=1e-2)
    s = O.Simulation(cfg)
    assert s.init(r, a, b, e) == O.OK
    m0 = [v.sum() for v in s.moments()]
    assert s.step(10) == O.OK
    assert s.stats()["reconstructions"] == 0
    m1 = [v.sum() for v in s.moments()]
    assert abs(m1[0] - m0[0]) < 10 * 1e-12 * m0[0]
    assert abs(m1[1] - m0[1]) < 10 * 1e-12 * m0[0]
    assert abs(m1[2] - m0[2]) < 10 * 1e-12 * m0[0]
    assert abs(m1[3] - m0[3]) < 10 * 1e-12 * m0[3]


# ---------------------------------------------------------------- exact Riemann solver

SOD_L, SOD_R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)


def test_exact_riemann_star_state_textbook_sod():
    p, u = riemann.star_state(SOD_L, SOD_R)
    assert abs(p - 0.30313) < 1e-5 and abs(u - 0.92745) < 1e-5


def test_exact_riemann_satisfies_jump_conditions():
    g = GAMMA
    p, u = riemann.star_state(SOD_L, SOD_R)
    S = riemann.shock_speed_right(SOD_L, SOD_R)
    rr, ur, pr = SOD_R
    # right shock: Rankine-Hugoniot for mass, momentum and energy in the shock frame
    r_s = riemann.sample(SOD_L, SOD_R, np.array([S - 1e-9]))[0][0]
    mflux = rr * (ur - S)
    assert abs(r_s * (u - S) - mflux) < 1e-10
    assert abs((r_s * (u - S) ** 2 + p) - (rr * (ur - S) ** 2 + pr)) < 1e-10
    H = lambda r, v, pp: 0.5 * v * v + g / (g - 1) * pp / r
    assert abs(H(r_s, u - S, p) - H(rr, ur - S, pr)) < 1e-10
    # left rarefaction: isentropic, Riemann invariant u + 2c/(g-1) constant
    xs = np.linspace(-1.18, -0.08, 7)
    rho, vel, pres = riemann.sample(SOD_L, SOD_R, xs)
    ent = pres / rho ** g
    np.testing.assert_allclose(ent, 1.0, rtol=1e-12)
    c = np.sqrt(g * pres / rho)
    np.testing.assert_allclose(vel + 2 * c / (g - 1), 2 * math.sqrt(g) / (g - 1), rtol=1e-12)


@pytest.mark.slow
def test_oracle_sod_tube_against_exact_solution():
    """Sec. IV.C.1 tube (here the benchmark's rho/p ratios, nu = 1e-4, sensor on,
    zero-gradient ends): density and pressure within 2% in L1 of the exact
    solution, and the star plateau within 2%."""
    nx, steps = 1024, 250
    cfg = O.make_config(nx, 1, nu=1e-4, bc_x=O.ZERO_GRADIENT, sensor=True)
    s = O.Simulation(cfg)
    assert s.init(*flows.riemann_1d(nx, 1)) == O.OK
    assert s.step(steps) == O.OK
    st = s.stats()
    assert st["newton_failures"] == 0 and st["reconstruction_failures"] == 0
    r, ux, uy, T = [a[0] for a in s.primitives()]
    p = r * T
    S = (np.arange(nx) - (nx // 2 - 0.5)) / steps
    re, ue, pe = riemann.sample(SOD_L, SOD_R, S)
    assert np.abs(r - re).sum() / np.abs(re).sum() < 0.02
    assert np.abs(p - pe).sum() / np.abs(pe).sum() < 0.02
    ps, us = riemann.star_state(SOD_L, SOD_R)
    sl = slice(nx // 2 + 10, nx // 2 + 200)  # between rarefaction tail and contact
    assert abs(p[sl].mean() - ps) < 0.02 * ps
    assert abs(ux[sl].mean() - us) < 0.02 * us
    # the post-shock region lives in lattice U_x = 1 (u* > 0.5)
    assert set(np.unique(s.shifts()[0])) == {0, 1}


def test_replayed_lattice_decisions_reproduce_the_free_run():
    """ora_step_forced with the decisions the criterion itself takes gives the
    same state bit for bit; other decisions change the state; shifts beyond
    u_max are refused."""
    n = 24
    fields = flows.isentropic_vortex(n, n, radius=4.0, mach=1.0)
    a = O.Simulation(O.make_config(n, n))
    b = O.Simulation(O.make_config(n, n))
    c = O.Simulation(O.make_config(n, n))
    for s in (a, b, c):
        assert s.init(*fields) == O.OK
    for _ in range(6):
        assert a.step(1) == O.OK
        ux, uy = a.shifts()
        assert b.step_forced(ux, uy) == O.OK
        assert c.step_forced(*c.shifts()) == O.OK  # never change lattice
    for x, y in zip(a.moments(), b.moments()):
        assert np.array_equal(x, y)
    assert not np.array_equal(a.moments()[1], c.moments()[1])
    bad = np.full((n, n), 5, np.int8)
    assert b.step_forced(bad, bad) != O.OK


# --------------------------------------------------------------- overlapping ranges

@pytest.mark.parametrize("u,current,expect", [
    # the paper's example: the range of U = 0 widened to [-1, 1] (w = 0.5)
    (0.3, 0, 0), (0.99, 0, 0), (1.0, 0, 0), (-0.99, 0, 0),
    (1.0 + 1e-12, 0, 1),        # leaves the widened range: the criterion's shift
    (-1.0, 0, -1),              # lower end open: criterion gives -1 (-1.5 < u <= -0.5)
    (0.01, 1, 1), (0.0, 1, 0),  # range of U = 1 is (0, 2]
    (1.7, 0, 2),                # far outside: the criterion decides
    (2.9, 2, 2), (-2.9, -2, -2),
])
def test_overlapping_ranges_keep_the_current_shift(u, current, expect):
    assert O.select_shift_kept(u, current, 0.5) == expect


def test_overlapping_ranges_with_zero_width_are_the_criterion():
    rng = np.random.default_rng(5)
    for u in rng.uniform(-3.2, 3.2, 2000):
        for cur in (-2, -1, 0, 1, 2):
            for n0 in (0.5, 0.51):
                assert O.select_shift_kept(u, cur, 0.0, n0) == O.select_shift(u, n0)


def test_overlapping_ranges_change_shift_only_outside_the_widened_range():
    """Step by step on the Mach-1.2 vortex with w = 0.5: a node's next shift U'
    always has u in (U' - 1, U' + 1]; it differs from its current shift U only
    when u has left (U - 1, U + 1]; fewer lattice changes than with the plain
    criterion (what the history rule is for; the number of interface nodes
    may grow or shrink)."""
    n = 48
    fields = flows.isentropic_vortex(n, n, radius=4.0, mach=1.2)
    runs = {}
    for w in (0.0, 0.5):
        s = O.Simulation(O.make_config(n, n, overlap=w))
        assert s.init(*fields) == O.OK
        changes = 0
        for _ in range(12):
            r, ux, uy, T = s.primitives()
            sx, sy = s.shifts()
            assert s.step(1) == O.OK
            nx_, ny_ = s.shifts()
            for u, cur, new in ((ux, sx, nx_), (uy, sy, ny_)):
                changes += int((new != cur).sum())
                if w > 0:
                    assert ((u > new - 1.0) & (u <= new + 1.0)).all()
                    moved = new != cur
                    assert not ((u[moved] > cur[moved] - 1.0) & (u[moved] <= cur[moved] + 1.0)).any()
        runs[w] = changes
    assert runs[0.5] < runs[0.0]


@pytest.mark.parametrize("u,nb,expect", [
    (0.6, [0] * 8, 0),                 # u = 0.6 lies in (-1, 1] (U = 0) and (0, 2] (U = 1)
    (0.6, [1] * 8, 1),
    (0.6, [0] * 4 + [1] * 4, 1),       # tie: the criterion's shift
    (0.6, [0] * 5 + [1] * 3, 0),
    (0.6, [2] * 8, 1),                 # 2 is not a candidate: (1, 3] does not hold 0.6
    (0.2, [1] * 8, 1),                 # (0, 2] holds 0.2
    (-0.2, [1] * 8, 0),                # ... but not -0.2
    (-0.7, [-1] * 3 + [0] * 5, 0),     # criterion -1; 0 is used by more neighbours
])
def test_overlapping_ranges_follow_the_neighbourhood(u, nb, expect):
    assert O.select_shift_neighbours(u, 0.5, nb) == expect


def test_neighbourhood_rule_with_zero_width_is_the_criterion():
    rng = np.random.default_rng(6)
    for u in rng.uniform(-3.2, 3.2, 1000):
        nb = rng.integers(-2, 3, 8)
        assert O.select_shift_neighbours(u, 0.0, nb) == O.select_shift(u)


def _interface_nodes(sx, sy):
    m = np.zeros(sx.shape, bool)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            m |= (np.roll(sx, (dy, dx), (0, 1)) != sx) | (np.roll(sy, (dy, dx), (0, 1)) != sy)
    return int(m.sum())


def test_neighbourhood_rule_reduces_interface_nodes():
    """Sec. III.A.2: choosing by the neighbourhood reduces the interface cells.
    On the 64^2 Mach-1.2 vortex over 40 steps with w = 0.5: every new shift's
    widened range holds the node's velocity, and the count of nodes with a
    neighbour in another lattice is lower than with Eq. criterion."""
    n = 64
    fields = flows.isentropic_vortex(n, n, radius=5.0, mach=1.2)
    total = {}
    for w, rule in ((0.0, O.RULE_HISTORY), (0.5, O.RULE_NEIGHBOURS)):
        s = O.Simulation(O.make_config(n, n, overlap=w, overlap_rule=rule))
        assert s.init(*fields) == O.OK
        total[w] = 0
        for _ in range(40):
            r, ux, uy, T = s.primitives()
            assert s.step(1) == O.OK
            sx, sy = s.shifts()
            for u, sh in ((ux, sx), (uy, sy)):
                assert ((u > sh - 0.5 - w) & (u <= sh + 0.5 + w)).all()
            total[w] += _interface_nodes(sx, sy)
    assert total[0.5] < 0.9 * total[0.0]

"""Pins of the oracle's flexible-Prandtl collision (App. E, Eqs. Shakhov and
prandtlPoly) and of Grad's populations with kappa = rho Cp nu / Pr.

The heat-flux term is checked through what it does to the moments, which
follow from the equilibrium's own moments by algebra: for a node at rest in
its lattice the term adds no mass, and it adds w q (M6/(2T) - Cp M4) /
(2 rho Cp T^2) + w q (2 Cv - 2) T M2 / (rho Cp) to the heat flux and
w q (M4/(2T) - Cp M2) / (rho Cp T^2) to the momentum, where w = 1/tau -
1/tau_Pr and M2, M4, M6 are sum_i f^eq_i xi_x^2 |xi|^{0,2,4}. A dropped or
misplaced factor anywhere in the term changes one of these."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2009_13426_gb300 import flows


def _xi():
    x, y = O.velocities()
    return x.astype(np.float64), y.astype(np.float64)


def _rates(nu, T, pr, alpha=1.0):
    tau = (0.5 + nu / T) * alpha
    tau_pr = (0.5 + (nu / pr) / T) * alpha
    return tau, 1.0 / tau - 1.0 / tau_pr


def _generic_state(seed, U=(1, 0), noise=1e-3):
    """Pre-collision populations with a heat flux: Grad populations of a state
    with gradients, perturbed."""
    rng = np.random.default_rng(seed)
    cfg = O.make_config(4, 4, nu=0.05)
    du = rng.normal(0, 0.05, (2, 2))
    dT = rng.normal(0, 0.05, 2)
    st, f, g = O.grad_populations(cfg, U[0], U[1], 0.9, U[0] + 0.2, U[1] - 0.15, 0.8, du, dT, 1.0)
    assert st == O.OK
    f = f * (1.0 + noise * rng.uniform(-1, 1, f.size))
    g = g * (1.0 + noise * rng.uniform(-1, 1, g.size))
    return f, g


def test_heat_flux_exact_rational():
    """q_a = 1/2 sum_i cbar_ia (|cbar_i|^2 f_i + g_i) with cbar_i = xi_i + U - u,
    in exact rational arithmetic with the absolute velocities."""
    rng = np.random.default_rng(2)
    x, y = O.velocities()
    for _ in range(30):
        f = rng.uniform(0.01, 0.3, 21)
        g = rng.uniform(0.01, 0.5, 21)
        Ux, Uy = (int(v) for v in rng.integers(-2, 3, 2))
        ux, uy = rng.uniform(-2.5, 2.5, 2)
        q = O.heat_flux(f, g, Ux, Uy, ux, uy)
        qx = qy = Fraction(0)
        scale = 0.0
        for i in range(21):
            cx = Fraction(int(x[i]) + Ux) - Fraction(ux)
            cy = Fraction(int(y[i]) + Uy) - Fraction(uy)
            e = (cx * cx + cy * cy) * Fraction(f[i]) + Fraction(g[i])
            qx += cx * e / 2
            qy += cy * e / 2
            scale += float(abs(cx) * e)
        assert abs(q[0] - float(qx)) <= 1e-15 * scale
        assert abs(q[1] - float(qy)) <= 1e-15 * scale


def test_unit_prandtl_is_bgk_bit_for_bit():
    f, g = _generic_state(3)
    a = O.collide_node(O.make_config(4, 4, nu=0.05), f, g, 1, 0)
    b = O.collide_node(O.make_config(4, 4, nu=0.05, prandtl=1.0), f, g, 1, 0)
    assert a[0] == b[0] == O.OK
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("sensor", [False, True])
def test_term_scales_with_rate_difference(sensor):
    """The change against BGK is w times a Pr-independent term, with
    w = 1/tau - 1/tau_Pr, tau_Pr = 1/2 + (nu/Pr)/T (App. E); with the sensor
    both times carry the same factor, so the ratio of the changes at two Pr
    is still the ratio of the w's."""
    nu = 0.05
    f, g = _generic_state(4, noise=5e-2 if sensor else 1e-3)
    mom = O.node_moments(f, g, 1, 0, 1.4)
    T = mom[3]
    base = O.collide_node(O.make_config(4, 4, nu=nu, sensor=sensor), f, g, 1, 0)
    if sensor:
        # the sensor is active on these populations: the BGK result differs
        plain = O.collide_node(O.make_config(4, 4, nu=nu), f, g, 1, 0)
        assert np.abs(plain[1] - base[1]).max() > 1e-6
    d = {}
    for pr in (0.5, 0.71, 2.0):
        st, fs, gs = O.collide_node(O.make_config(4, 4, nu=nu, sensor=sensor, prandtl=pr),
                                    f, g, 1, 0)
        assert st == O.OK
        d[pr] = (np.concatenate([fs - base[1], gs - base[2]]), _rates(nu, T, pr)[1])
    ref, w_ref = d[0.71]
    assert np.abs(ref).max() > 1e-6
    for pr in (0.5, 2.0):
        diff, w = d[pr]
        np.testing.assert_allclose(diff * (w_ref / w), ref, rtol=1e-9, atol=1e-12 * np.abs(ref).max())


def test_equilibrium_input_has_no_heat_flux_term():
    """Populations at equilibrium carry no heat flux (constraints G1, G3 in the
    node's frame), so the term vanishes for every Pr."""
    rho, ubx, uby, T = 1.1, 0.3, -0.2, 0.75
    st, lam, feq, it = O.equilibrium(rho, ubx, uby, T)
    geq = (2.0 / 0.4 - 2.0) * T * feq
    base = O.collide_node(O.make_config(4, 4, nu=0.05), feq, geq, 1, 1)
    for pr in (0.3, 3.0):
        st, fs, gs = O.collide_node(O.make_config(4, 4, nu=0.05, prandtl=pr), feq, geq, 1, 1)
        assert np.abs(fs - base[1]).max() <= 1e-11 * feq.max()
        assert np.abs(gs - base[2]).max() <= 1e-11 * geq.max()


@pytest.mark.parametrize("gamma", [1.4, 2.0])
@pytest.mark.parametrize("T", [0.6, 1.0])
@pytest.mark.parametrize("pr", [0.71, 2.0])
def test_term_moments_at_rest(gamma, T, pr):
    """A node at rest in lattice 0 with an odd perturbation that carries heat
    flux in f and in g and leaves rho, u, T unchanged: the term's mass, momentum,
    heat flux and energy against the closed forms of the module docstring."""
    x, y = _xi()
    nu, rho = 0.05, 1.2
    cv = 1.0 / (gamma - 1.0)
    cp = gamma * cv
    st, lam, feq, it = O.equilibrium(rho, 0.0, 0.0, T)
    assert st == O.OK
    c2 = x * x + y * y
    M2, M4, M6 = (feq * x * x).sum(), (feq * x * x * c2).sum(), (feq * x * x * c2 * c2).sum()
    geq = (2.0 * cv - 2.0) * T * feq
    h = feq * x * (c2 - M4 / M2)          # zero mass, momentum and energy
    f = feq + 0.02 * h + 0.01 * feq * y * (c2 - M4 / M2)
    g = geq * (1.0 + 0.03 * x - 0.02 * y)  # zero mass; internal heat flux
    mom = O.node_moments(f, g, 0, 0, gamma)
    # the equilibrium's constraints hold to the Newton tolerance
    assert abs(mom[0] - rho) < 1e-12 and abs(mom[1]) < 1e-14 and abs(mom[2]) < 1e-14
    assert abs(mom[3] - T) < 1e-12
    rho, T = mom[0], mom[3]
    q = O.heat_flux(f, g, 0, 0, 0.0, 0.0)
    assert np.abs(q).min() > 1e-3
    base = O.collide_node(O.make_config(4, 4, nu=nu, gamma=gamma), f, g, 0, 0)
    st, fs, gs = O.collide_node(O.make_config(4, 4, nu=nu, gamma=gamma, prandtl=pr), f, g, 0, 0)
    assert st == O.OK
    df, dg = fs - base[1], gs - base[2]
    w = _rates(nu, T, pr)[1]
    tol = 1e-10 * abs(w) * np.abs(q).max()
    assert abs(df.sum()) <= tol and abs(dg.sum()) <= tol
    k_mom = (M4 / (2 * T) - cp * M2) / (rho * cp * T * T)
    k_q = (M6 / (2 * T) - cp * M4) / (2 * rho * cp * T * T) + (2 * cv - 2) * T * M2 / (rho * cp)
    for a, xa in ((0, x), (1, y)):
        assert abs((df * xa).sum() - w * q[a] * k_mom) <= tol
        dq = 0.5 * (xa * (c2 * df + dg)).sum()
        assert abs(dq - w * q[a] * k_q) <= tol
    assert abs(0.5 * (c2 * df + dg).sum()) <= tol     # energy at rest


def test_monatomic_term_is_shakhov_within_lattice_error():
    """gamma = 2 (Cv = 1, Cp = (D + 2)/2, g^eq = 0): the term is Shakhov's,
    which with Maxwellian moments moves the post-collision heat flux from
    (1 - 1/tau) q to (1 - 1/tau_Pr) q and adds no momentum. At T = 1 the D2Q21
    equilibrium's fourth and sixth moments are within 1 % of the Maxwellian's,
    so the transfer is within 3 % and the momentum within 1 % of w q / T."""
    x, y = _xi()
    T, nu, pr, rho = 1.0, 0.05, 0.5, 1.0
    st, lam, feq, it = O.equilibrium(rho, 0.0, 0.0, T)
    c2 = x * x + y * y
    a = (feq * x * x * c2).sum() / (feq * x * x).sum()
    f = feq + 0.02 * feq * x * (c2 - a)
    g = np.zeros(21)
    q = O.heat_flux(f, g, 0, 0, 0.0, 0.0)
    tau, w = _rates(nu, T, pr)
    st, fs, gs = O.collide_node(O.make_config(4, 4, nu=nu, gamma=2.0, prandtl=pr), f, g, 0, 0)
    assert st == O.OK and np.abs(gs).max() == 0.0
    q_post = O.heat_flux(fs, gs, 0, 0, 0.0, 0.0)
    transfer = (q_post[0] - (1.0 - 1.0 / tau) * q[0]) / (w * q[0])
    assert abs(transfer - 1.0) < 0.03, transfer
    assert abs((fs * x).sum()) < 0.01 * abs(w * q[0]) / T


def test_grad_heat_part_and_prandtl():
    """Grad's populations: kappa = rho Cp nu / Pr scales the heat-flux part by
    1/Pr; w_pr multiplies only that part (and all of phi_g); without a
    temperature gradient w_pr has no effect."""
    du = np.array([[0.02, -0.01], [0.03, 0.015]])
    dT = np.array([0.04, -0.03])
    args = (1, 0, 0.9, 1.2, 0.1, 0.8)
    c1 = O.make_config(4, 4, nu=0.05)
    c2 = O.make_config(4, 4, nu=0.05, prandtl=0.5)
    _, f0, g0 = O.grad_populations(c1, *args, 0 * du, 0 * dT, 1.0)
    _, f1, g1 = O.grad_populations(c1, *args, 0 * du, dT, 1.0)
    _, f2, g2 = O.grad_populations(c2, *args, 0 * du, dT, 1.0)
    np.testing.assert_allclose(f2 - f0, (f1 - f0) / 0.5, rtol=1e-10, atol=1e-16)
    np.testing.assert_allclose(g2 - g0, (g1 - g0) / 0.5, rtol=1e-10, atol=1e-16)
    _, fa, ga = O.grad_populations(c1, *args, 0 * du, dT, 0.3, 0.2)
    _, fb, gb = O.grad_populations(c1, *args, 0 * du, dT, 0.5, 0.0)
    np.testing.assert_allclose(fa, fb, rtol=1e-14)
    np.testing.assert_allclose(ga, gb, rtol=1e-14)
    _, fa, ga = O.grad_populations(c1, *args, du, 0 * dT, 0.4, 0.3)
    _, fb, gb = O.grad_populations(c1, *args, du, 0 * dT, 0.4, 0.0)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_run_conserves_mass_and_differs_from_bgk():
    """A periodic flow without lattice changes (a slow vortex, lattice 0
    throughout): the term keeps the total mass to round-off at any Pr, and
    Pr changes the flow."""
    n = 24
    fields = flows.isentropic_vortex(n, n, strength=1.0, radius=4.0, mach=0.1, seed=3)
    out = {}
    for pr in (1.0, 0.71):
        s = O.Simulation(O.make_config(n, n, nu=0.02, prandtl=pr))
        assert s.init(*fields) == O.OK
        m0 = s.moments()[0].sum()
        assert s.step(20) == O.OK
        sx, sy = s.shifts()
        assert not sx.any() and not sy.any()
        assert s.stats()["reconstructions"] == 0
        m = s.moments()
        assert abs(m[0].sum() - m0) <= 1e-13 * m0
        out[pr] = m
    assert np.abs(out[1.0][3] - out[0.71][3]).max() > 1e-9


@pytest.mark.parametrize("pr", [0.0, -1.0, float("nan")])
def test_invalid_prandtl_is_refused(pr):
    with pytest.raises(ValueError):
        O.Simulation(O.make_config(4, 4, prandtl=pr))

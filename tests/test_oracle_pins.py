"""Pins of the oracle's kinetic sensor (Eq. DeltaAvg and the onset of
alpha, Sec. IV.A.2), of its second-order central differences (Sec. IV.A.1,
through the Grad initial state of Eqs. GradGeneral_f / GradGeneral_g), and
of the relaxation time of a rebuilt pull (Sec. III.B.2: the rebuilt
population is the sender's post-collision one, so it relaxes with the
sender's tau), and of the failure policy where the root finder fails (an
uncollided node; the normalised Maxwellian-guess exponential for a rebuild).

test_planted_mistakes_fail_their_pins plants each mistake these pins are
meant to catch in a copy of the oracle's source, builds it, and checks that
the pin fails on it."""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from oracle import build as obuild
from paper_2009_13426_gb300 import flows

GAMMA = 1.4
CV = 1.0 / (GAMMA - 1.0)
CP = GAMMA * CV
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _xi():
    x, y = O.velocities()
    return x.astype(np.float64), y.astype(np.float64)


# ---------------------------------------------------------------- sensor

def _sensor_state(eps, rho=1.1, ubx=0.3, uby=-0.2, T=0.7, seed=0, g_dev=0.3):
    """Populations f = f^eq (1 + d) and g = g^eq (1 + d_g) whose moments are
    those of f^eq, g^eq: d is orthogonal (weighted by f^eq) to 1, xi_x, xi_y
    and |xi|^2, d_g to 1 (weighted by g^eq), so rho, u and T (Eq. polyTemp)
    are unchanged. d is scaled so that (1/V) sum |d_i| = eps exactly; d_g has
    mean |d_g| = g_dev (the sensor reads f only)."""
    rng = np.random.default_rng(seed)
    st, lam, feq, _ = O.equilibrium(rho, ubx, uby, T)
    assert st == O.OK
    x, y = _xi()
    A = np.stack([feq, feq * x, feq * y, feq * (x * x + y * y)])
    r = rng.standard_normal(21)
    d = r - A.T @ np.linalg.solve(A @ A.T, A @ r)
    d *= eps / np.abs(d).mean()
    geq = (2 * CV - 2) * T * feq
    rg = rng.standard_normal(21)
    dg = rg - geq * (geq @ rg) / (geq @ geq)
    dg *= g_dev / np.abs(dg).mean()
    return feq, feq * (1 + d), geq * (1 + dg), d


def _alpha(eps, cfg_kw=None, **kw):
    """alpha(eps) as the oracle's collision applies it: f* = f - (f - f^eq) /
    (tau alpha), tau = 1/2 + nu/T, read back by least squares over the 21
    velocities."""
    nu, T = 0.01, kw.get("T", 0.7)
    feq, f, g, d = _sensor_state(eps, **kw)
    cfg = O.make_config(4, 4, nu=nu, sensor=True, **(cfg_kw or {}))
    st, fs, gs = O.collide_node(cfg, f, g, 1, 0)
    assert st == O.OK
    tau0 = 0.5 + nu / T
    a, b = f - feq, f - fs
    inv = (a @ b) / (a @ a)  # 1 / (tau alpha)
    return 1.0 / (inv * tau0)


@pytest.mark.parametrize("eps", [1e-5, 1e-3, 5e-3, 9.9e-3])
def test_sensor_is_off_below_the_onset(eps):
    """Sec. IV.A.2: dissipation is added only where eps_Kn > 0.01, so alpha = 1
    (plain BGK) below the onset."""
    assert abs(_alpha(eps) - 1.0) < 1e-9


def test_sensor_adds_dissipation_above_the_onset_and_grows_with_eps():
    """Sec. IV.A.2: above the onset dissipation is added (alpha > 1), and a
    larger departure from equilibrium never gets less of it."""
    for eps in (0.0102, 0.05, 0.3, 3.0, 30.0):
        assert _alpha(eps) > 1.0 + 1e-6, eps
    grid = np.geomspace(1e-3, 1e2, 41)
    al = np.array([_alpha(e) for e in grid])
    assert (np.diff(al) >= -1e-9).all()
    assert (al >= 1.0 - 1e-9).all()


def test_sensor_reading_knots_continuity_and_plateau():
    """The reading of alpha (the paper fixes its onset only): continuous,
    piecewise linear in log10(eps) through (0.01, 1), (0.1, a0), (1, a1),
    (10, a2), constant beyond 10, with the configured a = (1.05, 1.35, 1.6)."""
    for e, a in ((0.1, 1.05), (1.0, 1.35), (10.0, 1.6)):
        assert abs(_alpha(e) - a) < 1e-9
        for s in (1 - 1e-7, 1 + 1e-7):
            assert abs(_alpha(e * s) - a) < 1e-6
    assert abs(_alpha(0.01 * (1 + 1e-7)) - 1.0) < 1e-6
    assert abs(_alpha(50.0) - 1.6) < 1e-9 and abs(_alpha(1e3) - 1.6) < 1e-9
    # midway in log10 between two knots: the mean of their values
    assert abs(_alpha(math.sqrt(0.1 * 1.0)) - 0.5 * (1.05 + 1.35)) < 1e-9


@pytest.mark.parametrize("eps", [1.3e-3, 3.1e-3, 7.7e-3])
def test_sensor_measure_is_the_mean_relative_departure_of_f(eps):
    """Eq. DeltaAvg: eps_Kn = (1/V) sum_i |f_i - f_i^eq| / f_i^eq over the V = 21
    velocities, f only. With knots that make alpha = 1 + log10(eps / 1e-3) on
    [1e-3, 1e-2], the alpha applied gives back eps; the constructed state has
    (1/V) sum |d_i| = eps exactly and g far from g^eq."""
    kw = {"sensor_eps": (1e-3, 1e-2, 1e-1), "sensor_alpha": (2.0, 3.0, 4.0)}
    a = _alpha(eps, cfg_kw=kw)
    assert abs(1e-3 * 10 ** (a - 1.0) - eps) < 1e-9 * eps


# ---------------------------------------------------------------- central differences

def _init_state(nx, ny, rho, ux, uy, T, nu=0.05, bc_x=O.PERIODIC):
    cfg = O.make_config(nx, ny, nu=nu, bc_x=bc_x)
    sim = O.Simulation(cfg)
    assert sim.init(*flows.conserved(rho, ux, uy, T)) == O.OK
    f, g = sim.populations()
    sx, sy = sim.shifts()
    return cfg, f, g, sx, sy


def _pi_neq_xy(f, rho, ux, uy, T, Ux, Uy):
    """Pi^neq_xy = sum (f - f^eq) cbar_x cbar_y and M22 = sum f^eq cbar_x^2 cbar_y^2
    with f^eq the equilibrium of the node's own moments, cbar = xi + U - u."""
    x, y = _xi()
    st, lam, feq, _ = O.equilibrium(rho, ux - Ux, uy - Uy, T)
    assert st == O.OK
    cx, cy = x + Ux - ux, y + Uy - uy
    return ((f - feq) * cx * cy).sum(), (feq * cx * cx * cy * cy).sum()


@pytest.mark.parametrize("axis", ["y", "x"])
def test_initial_shear_stress_uses_second_order_central_differences(axis):
    """A pure shear u_x = A sin(2 pi k y / n) (or u_y = A sin(2 pi k x / n)) with
    uniform rho and T. The Grad initial state h = h^eq (1 + phi) has
    Pi^neq_xy = sigma_xy M22 / (rho T^2), sigma_xy = -rho nu d u (Eq.
    GradGeneral_f; the normal stresses and the heat flux vanish). The
    second-order central difference of the sinusoid is exactly
    A sin(2 pi k / n) cos(2 pi k y / n): sin(kh)/h times the analytic derivative."""
    n, k, A, nu, rho0, T0 = 24, 2, 0.02, 0.05, 1.0, 0.7
    nx, ny = (8, n) if axis == "y" else (n, 8)
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    s = yy if axis == "y" else xx
    w = 2 * math.pi * k / n
    rho = np.full((ny, nx), rho0)
    T = np.full((ny, nx), T0)
    ux = A * np.sin(w * s) if axis == "y" else np.zeros((ny, nx))
    uy = np.zeros((ny, nx)) if axis == "y" else A * np.sin(w * s)
    cfg, f, g, sx, sy = _init_state(nx, ny, rho, ux, uy, T, nu=nu)
    fd = A * math.sin(w) * np.cos(w * s)  # central difference, spacing 1
    err = 0.0
    scale = 0.0
    for j in range(ny):
        for i in range(nx):
            pi, m22 = _pi_neq_xy(f[j, i], rho0, ux[j, i], uy[j, i], T0, sx[j, i], sy[j, i])
            expect = -rho0 * nu * fd[j, i] * m22 / (rho0 * T0 * T0)
            err = max(err, abs(pi - expect))
            scale = max(scale, abs(expect))
    assert scale > 1e-5
    assert err <= 1e-12 * scale


@pytest.mark.parametrize("axis", ["x", "y"])
def test_initial_heat_flux_uses_second_order_central_differences(axis):
    """At rest with T = T0 + C sin(2 pi k s / n): the Grad initial state adds the
    momentum q k_mom, q = -kappa dT, kappa = rho Cp nu, k_mom = (M4/(2T) - Cp M2)
    / (rho Cp T^2) from the node's equilibrium moments (the closed form of the
    heat-flux terms at rest); dT is the central difference
    C sin(2 pi k / n) cos(2 pi k s / n)."""
    n, k, C, nu, rho0, T0 = 20, 3, 0.05, 0.05, 1.0, 0.7
    nx, ny = (n, 6) if axis == "x" else (6, n)
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    s = xx if axis == "x" else yy
    w = 2 * math.pi * k / n
    T = T0 + C * np.sin(w * s)
    rho = np.full((ny, nx), rho0)
    z = np.zeros((ny, nx))
    cfg, f, g, sx, sy = _init_state(nx, ny, rho, z, z, T, nu=nu)
    x, y = _xi()
    xa = x if axis == "x" else y
    c2 = x * x + y * y
    dT = C * math.sin(w) * np.cos(w * s)
    err = scale = 0.0
    for j in range(ny):
        for i in range(nx):
            assert sx[j, i] == 0 and sy[j, i] == 0
            st, lam, feq, _ = O.equilibrium(rho0, 0.0, 0.0, T[j, i])
            M2, M4 = (feq * xa * xa).sum(), (feq * xa * xa * c2).sum()
            Tn = T[j, i]
            k_mom = (M4 / (2 * Tn) - CP * M2) / (rho0 * CP * Tn * Tn)
            q = -rho0 * CP * nu * dT[j, i]
            mom = ((f[j, i] - feq) * xa).sum()
            err = max(err, abs(mom - q * k_mom))
            scale = max(scale, abs(q * k_mom))
    assert scale > 1e-5
    assert err <= 1e-12 * scale


def test_central_differences_at_zero_gradient_ends_use_the_ghost_copy():
    """At a zero-gradient end the ghost node carries the nearest interior
    moments (reading of Sec. IV.A.1 / IV.C.1), so the central difference at the
    last node is (F[n-1] - F[n-2]) / 2 and at the first (F[1] - F[0]) / 2."""
    nx, ny, A, nu, rho0, T0 = 10, 4, 0.01, 0.05, 1.0, 0.7
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    uy = A * (xx - 4.5) ** 2 / 10.0
    z = np.zeros((ny, nx))
    rho = np.full((ny, nx), rho0)
    T = np.full((ny, nx), T0)
    cfg, f, g, sx, sy = _init_state(nx, ny, rho, z, uy, T, nu=nu, bc_x=O.ZERO_GRADIENT)
    F = uy[0]
    fd = np.empty(nx)
    fd[1:-1] = 0.5 * (F[2:] - F[:-2])
    fd[0] = 0.5 * (F[1] - F[0])
    fd[-1] = 0.5 * (F[-1] - F[-2])
    for i in range(nx):
        pi, m22 = _pi_neq_xy(f[1, i], rho0, 0.0, uy[1, i], T0, sx[1, i], sy[1, i])
        expect = -rho0 * nu * fd[i] * m22 / (rho0 * T0 * T0)
        assert abs(pi - expect) <= 1e-12 * 1e-3, (i, pi, expect)


# ---------------------------------------------------------------- relaxation time of a rebuild

@pytest.mark.parametrize("prandtl", [1.0, 0.7])
def test_rebuilt_pull_relaxes_with_the_sender_tau(prandtl):
    """Every node is forced from lattice (0, 0) into (1, 0), so every pull is
    rebuilt. The rebuilt population must be h^eq (1 + (1 - 1/tau_s) phi_h +
    (1/tau_s - 1/tau_Pr,s) phi_h,q) of the sender s, with tau_s = 1/2 + nu/T_s,
    the sender's gradients by central differences and its equilibrium in the
    receiver's lattice (Sec. III.B.2, reading 7). The temperature varies
    strongly, so the receiver's tau would give visibly different values."""
    nx, ny, nu = 12, 10, 0.2
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    rho = 1.0 + 0.05 * np.sin(2 * math.pi * xx / nx)
    T = 0.8 + 0.3 * np.sin(2 * math.pi * xx / nx + 1.0)
    ux = 0.1 * np.sin(2 * math.pi * yy / ny)
    uy = 0.08 * np.cos(2 * math.pi * xx / nx)
    cfg = O.make_config(nx, ny, nu=nu, prandtl=prandtl)
    sim = O.Simulation(cfg)
    assert sim.init(*flows.conserved(rho, ux, uy, T)) == O.OK
    sx, sy = sim.shifts()
    assert (sx == 0).all() and (sy == 0).all()
    r0, u0, v0, T0 = sim.primitives()  # the moments the step's first pass computes
    d = lambda F, ax: 0.5 * (np.roll(F, -1, axis=ax) - np.roll(F, 1, axis=ax))
    dudx, dudy, dvdx, dvdy = d(u0, 1), d(u0, 0), d(v0, 1), d(v0, 0)
    dTdx, dTdy = d(T0, 1), d(T0, 0)
    assert sim.step_forced(np.ones((ny, nx)), np.zeros((ny, nx))) == O.OK
    f, g = sim.populations()
    xi_x, xi_y = O.velocities()
    err = 0.0
    alt = 0.0
    for j in range(ny):
        for i in range(nx):
            for q in range(21):
                a = (i - (xi_x[q] + 1)) % nx
                b = (j - xi_y[q]) % ny
                du = np.array([[dudx[b, a], dvdx[b, a]], [dudy[b, a], dvdy[b, a]]])
                dT = np.array([dTdx[b, a], dTdy[b, a]])

                def rebuilt(Tt):
                    tau = 0.5 + nu / Tt
                    tau_pr = 0.5 + (nu / prandtl) / Tt
                    st, fr, gr = O.grad_populations(cfg, 1, 0, r0[b, a], u0[b, a], v0[b, a],
                                                    T0[b, a], du, dT, 1 - 1 / tau,
                                                    1 / tau - 1 / tau_pr)
                    assert st == O.OK
                    return fr[q], gr[q]

                fe, ge = rebuilt(T0[b, a])
                err = max(err, abs(f[j, i, q] - fe) / abs(fe), abs(g[j, i, q] - ge) / abs(ge))
                fr_, gr_ = rebuilt(T0[j, i])  # with the receiver's tau
                alt = max(alt, abs(fr_ - fe) / abs(fe))
    assert err <= 1e-12
    assert alt > 1e-3


# ---------------------------------------------------------------- planted mistakes

SRC = os.path.join(ROOT, "oracle", "alb_oracle.c")
T = "tests/test_oracle_pins.py::"

# (name, text of the oracle, planted text, the pin that must fail)
MUTANTS = [
    ("alpha != 1 below the onset",
     "if (!(eps > e[0])) return 1.0;", "if (!(eps > e[0])) return a[0];",
     T + "test_sensor_is_off_below_the_onset"),
    ("sensor mean over V - 1 velocities",
     "eps /= (double)Q;", "eps /= (double)(Q - 1);",
     T + "test_sensor_is_off_below_the_onset"),
    ("sensor reads g as well",
     "eps += fabs(f[i] - feq[i]) / feq[i];",
     "eps += 0.5 * (fabs(f[i] - feq[i]) / feq[i] + fabs(g[i] - (2.0 * Cv - D_SPACE) * T * "
     "feq[i]) / ((2.0 * Cv - D_SPACE) * T * feq[i]));",
     T + "test_sensor_measure_is_the_mean_relative_departure_of_f"),
    ("staircase instead of the interpolated alpha",
     "if (l <= kx[k + 1]) return ky[k] + (ky[k + 1] - ky[k]) * (l - kx[k]) / (kx[k + 1] - kx[k]);",
     "if (l <= kx[k + 1]) return ky[k + 1];",
     T + "test_sensor_reading_knots_continuity_and_plateau"),
    ("dropped 1/2 in the x difference",
     "d[0] = 0.5 * (F[ry * nx + xp] - F[ry * nx + xm]);",
     "d[0] = (F[ry * nx + xp] - F[ry * nx + xm]);",
     T + "test_initial_shear_stress_uses_second_order_central_differences"),
    ("dropped 1/2 in the y difference",
     "d[1] = 0.5 * (F[yp * nx + rx] - F[ym * nx + rx]);",
     "d[1] = (F[yp * nx + rx] - F[ym * nx + rx]);",
     T + "test_initial_shear_stress_uses_second_order_central_differences"),
    ("one-sided y difference",
     "d[1] = 0.5 * (F[yp * nx + rx] - F[ym * nx + rx]);",
     "d[1] = 0.5 * (F[yp * nx + rx] - F[ry * nx + rx]);",
     T + "test_initial_heat_flux_uses_second_order_central_differences"),
    ("x difference across the wrong axis",
     "d[0] = 0.5 * (F[ry * nx + xp] - F[ry * nx + xm]);",
     "d[0] = 0.5 * (F[yp * nx + rx] - F[ym * nx + rx]);",
     T + "test_initial_heat_flux_uses_second_order_central_differences"),
    ("receiver's tau in a rebuild",
     "const double tau = 0.5 + c->nu / s->T[k];",
     "const double tau = 0.5 + c->nu / s->T[y * c->nx + x];",
     T + "test_rebuilt_pull_relaxes_with_the_sender_tau"),
    ("receiver's tau_Pr in a rebuild",
     "const double tau_pr = 0.5 + (c->nu / c->prandtl) / s->T[k];",
     "const double tau_pr = 0.5 + (c->nu / c->prandtl) / s->T[y * c->nx + x];",
     T + "test_rebuilt_pull_relaxes_with_the_sender_tau"),
    ("a failed node relaxed towards the failed equilibrium",
     "for (int i = 0; i < Q; ++i) { fs[i] = f[i]; gs[i] = g[i]; }",
     "for (int i = 0; i < Q; ++i) { fs[i] = 0.5 * (f[i] + feq[i]); gs[i] = g[i]; }",
     T + "test_failed_collision_leaves_the_node_uncollided"),
    ("fallback in the sender's lattice instead of the receiver's",
     "const double ubx = s->ux[k] - Upx, uby = s->uy[k] - Upy, T = s->T[k];",
     "const double ubx = s->ux[k], uby = s->uy[k] - Upy, T = s->T[k];",
     T + "test_failed_rebuild_falls_back_to_the_normalised_maxwellian_exponential"),
]


def _run_pin(lib, *args):
    env = dict(os.environ)
    env[O.OVERRIDE_ENV] = lib
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *args], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.mark.slow
def test_planted_mistakes_fail_their_pins(tmp_path):
    """Each planted mistake, built into a copy of the oracle, makes its pin fail
    (pytest exit code 1); the unchanged source built the same way passes all
    the pins of this file."""
    text = open(SRC).read()
    ctrl = obuild.compile_source(SRC, str(tmp_path / "control.so"))
    rc, out = _run_pin(ctrl, "tests/test_oracle_pins.py", "-k", "not planted_mistakes")
    assert rc == 0, out
    for j, (name, old, new, nodeid) in enumerate(MUTANTS):
        assert text.count(old) == 1, name
        src = tmp_path / ("m%d.c" % j)
        src.write_text(text.replace(old, new))
        lib = obuild.compile_source(str(src), str(tmp_path / ("m%d.so" % j)))
        rc, out = _run_pin(lib, nodeid)
        assert rc == 1, (name, rc, out)


# ---------------------------------------------------------------- failure policy

def test_failed_collision_leaves_the_node_uncollided():
    """Reading 11 (the paper is silent): a node whose root finder fails is not
    collided, f* = f and g* = g exactly, and the failure is reported."""
    cfg = O.make_config(4, 4, nu=1e-2, newton_maxit=0)
    st, lam, feq, _ = O.equilibrium(1.1, 0.3, -0.2, 0.7)
    rng = np.random.default_rng(3)
    f = feq * (1 + 0.01 * rng.standard_normal(21))
    g = (2 * CV - 2) * 0.7 * feq * (1 + 0.01 * rng.standard_normal(21))
    st, fs, gs = O.collide_node(cfg, f, g, 1, 0)
    assert st != O.OK
    assert np.array_equal(fs, f) and np.array_equal(gs, g)


def test_failed_rebuild_falls_back_to_the_normalised_maxwellian_exponential():
    """Reading 11: a rebuilt pull whose root finder fails takes the Maxwellian
    guess's exponential of the sender's state in the receiver's lattice,
    f_i = rho exp(-|xi_i - ubar|^2 / (2T)) / sum_j exp(-|xi_j - ubar|^2 / (2T)),
    ubar = u_sender - U', and g_i = (2 Cv - D) T f_i. Every node is forced
    from lattice (0, 0) into (1, 0) with the root finder allowed no step, so
    every pull is such a fallback."""
    nx, ny = 6, 5
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    rho = 1.0 + 0.1 * np.sin(2 * math.pi * xx / nx)
    T = 0.7 + 0.1 * np.cos(2 * math.pi * yy / ny)
    ux = 0.2 * np.sin(2 * math.pi * yy / ny)
    uy = 0.1 * np.cos(2 * math.pi * xx / nx)
    init = O.Simulation(O.make_config(nx, ny, nu=1e-2))
    assert init.init(*flows.conserved(rho, ux, uy, T)) == O.OK
    f0, g0 = init.populations()
    sx, sy = init.shifts()
    sim = O.Simulation(O.make_config(nx, ny, nu=1e-2, newton_maxit=0))
    sim.set_state(f0, g0, sx, sy)
    r0, u0, v0, T0 = sim.primitives()
    assert sim.step_forced(np.ones((ny, nx)), np.zeros((ny, nx))) == O.ENEWTON
    st = sim.stats()
    assert st["reconstructions"] == st["reconstruction_failures"] == 21 * nx * ny
    f, g = sim.populations()
    xi_x, xi_y = _xi()
    err = 0.0
    for j in range(ny):
        for i in range(nx):
            for q in range(21):
                a = (i - (int(xi_x[q]) + 1)) % nx
                b = (j - int(xi_y[q])) % ny
                ubx, uby = u0[b, a] - 1.0, v0[b, a]
                w = np.exp(-((xi_x - ubx) ** 2 + (xi_y - uby) ** 2) / (2 * T0[b, a]))
                fe = r0[b, a] * w[q] / w.sum()
                ge = (2 * CV - 2) * T0[b, a] * fe
                err = max(err, abs(f[j, i, q] - fe) / fe, abs(g[j, i, q] - ge) / ge)
    assert err <= 1e-13

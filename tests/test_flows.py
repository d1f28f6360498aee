"""The seeded input recipes of the batched and served workloads (CPU only):
the isentropic vortex at any background temperature, and the clamps that
keep every flow of the two mixes inside the lattice's operating range."""
import math

import numpy as np

from paper_2009_13426_gb300 import flows

G = flows.GAMMA


def _prims(fields):
    r, a, b, e = fields
    ux, uy = a / r, b / r
    T = (e / r - 0.5 * (ux * ux + uy * uy)) * (G - 1.0)
    return r, ux, uy, T


def test_vortex_scales_with_the_background_sound_speed():
    """The Shu vortex at background T_inf is the T_inf = 1 vortex in units of
    the background's sound speed: swirl velocities scale with sqrt(T_inf),
    temperatures with T_inf, and the density stays isentropic (p / rho^gamma
    uniform)."""
    n, radius = 64, 6.0
    ref = _prims(flows.isentropic_vortex(n, n, radius=radius, mach=0.0, noise=0.0, T_inf=1.0))
    for T_inf in (0.464, 0.8, 1.2):
        r, ux, uy, T = _prims(flows.isentropic_vortex(n, n, radius=radius, mach=0.0, noise=0.0,
                                                      T_inf=T_inf))
        np.testing.assert_allclose(ux, ref[1] * math.sqrt(T_inf), atol=1e-12)
        np.testing.assert_allclose(uy, ref[2] * math.sqrt(T_inf), atol=1e-12)
        np.testing.assert_allclose(T, ref[3] * T_inf, rtol=1e-12)
        s = r * T / r ** G
        np.testing.assert_allclose(s, s.flat[0], rtol=1e-12)


def _fastest(sp):
    r, ux, uy, T = _prims(sp.fields())
    return float(np.sqrt(ux * ux + uy * uy).max()), float(T.min()), float(T.max())


def test_mix_vortices_stay_in_the_operating_range():
    """Every vortex of the batched and served mixes: background temperature
    within [0.35 / 0.754, 1.2] (core no colder than 0.35), fastest node below
    |u| = 2.5, and `clamped` set exactly when the recipe's Mach number or
    temperature had to be changed."""
    specs = [sp for sp in flows.batched_flows() + flows.serving_requests()[:300]
             if sp.kind == "vortex"]
    assert specs
    core = 1.0 - (G - 1.0) * 25.0 / (8.0 * G * math.pi ** 2) * math.e
    for sp in specs[:60]:
        T_inf = sp.vortex_T_inf()
        assert 0.35 / core - 1e-12 <= T_inf <= flows.VORTEX_T_MAX + 1e-12
        small = flows.FlowSpec(sp.kind, 64, 64, sp.mach, sp.T_ratio, sp.nu, 1, seed=sp.seed)
        umax, Tmin, Tmax = _fastest(small)
        assert umax <= 2.5 + 1e-9
        assert Tmin >= 0.35 * (1 - 1e-3) - 1e-12 and Tmax <= flows.VORTEX_T_MAX + 1e-9
    for sp in specs:
        T_inf = sp.vortex_T_inf()
        u_cap = 2.5 - 5.0 / (2.0 * math.pi) * math.sqrt(T_inf)
        assert sp.mach * math.sqrt(G * T_inf) <= u_cap + 1e-12
        if T_inf != 0.35 * sp.T_ratio:
            assert sp.clamped


def test_vortex_clamps_are_recorded():
    # temperature ratio 1: the core would be at 0.264; the background is raised
    sp = flows.FlowSpec("vortex", 64, 64, 0.5, 1.0, 1e-4, 1)
    assert sp.clamped and abs(sp.vortex_T_inf() - 0.35 / 0.7543) < 1e-3
    # ratio 4 would put the background at 1.4; it is held at 1.2
    sp = flows.FlowSpec("vortex", 64, 64, 0.5, 4.0, 1e-4, 1)
    assert sp.clamped and sp.vortex_T_inf() == flows.VORTEX_T_MAX
    # Mach 3 at T_inf = 0.7: the fastest node would pass 2.5
    sp = flows.FlowSpec("vortex", 64, 64, 3.0, 2.0, 1e-4, 1)
    assert sp.clamped and sp.mach < 3.0
    # inside the range: untouched
    sp = flows.FlowSpec("vortex", 64, 64, 1.0, 2.0, 1e-4, 1)
    assert not sp.clamped and sp.mach == 1.0


def test_shear_layers_clamp_the_cold_stream():
    for sp in flows.batched_flows():
        if sp.kind != "shear":
            continue
        u0 = sp.mach * math.sqrt(G * 0.35)
        assert u0 <= 2.5 + 1e-12
    # Mach 3 of the cold stream is u0 = 2.1, inside; Mach 4 would be 2.8
    sp = flows.FlowSpec("shear", 64, 64, 4.0, 2.0, 1e-4, 1)
    assert sp.clamped and abs(sp.mach * math.sqrt(G * 0.35) - 2.5) < 1e-12
    sp = flows.FlowSpec("shear", 64, 64, 2.0, 2.0, 1e-4, 1)
    assert not sp.clamped and sp.mach == 2.0

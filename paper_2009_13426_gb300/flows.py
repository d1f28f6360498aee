"""Seeded synthetic initial fields for the validation and benchmark workloads.

This module holds no part of the lattice Boltzmann method: it only evaluates
analytic initial conditions (density, velocity, temperature) and converts them
to the conserved fields (rho, rho*ux, rho*uy, rho*E) with
rho*E = rho |u|^2 / 2 + rho * Cv * T, Cv = 1 / (gamma - 1), p = rho * T.
Both the CUDA path and the CPU oracle are fed from here. All arrays are
float64 of shape (ny, nx), x fastest. Randomness comes from numpy's seeded
PCG64 generator, so every field is reproducible from its seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 1.4
# strength of the batched and served vortices (the Shu vortex's beta) and
# their hottest background temperature
VORTEX_STRENGTH = 5.0
VORTEX_T_MAX = 1.2


def conserved(rho, ux, uy, T, gamma=GAMMA):
    """(rho, ux, uy, T) -> (rho, rho*ux, rho*uy, rho*E)."""
    cv = 1.0 / (gamma - 1.0)
    rho = np.asarray(rho, np.float64)
    return (rho.copy(), rho * ux, rho * uy, 0.5 * rho * (ux * ux + uy * uy) + rho * cv * T)


def uniform(nx, ny, rho=1.0, ux=0.0, uy=0.0, T=0.7, gamma=GAMMA):
    shape = (ny, nx)
    return conserved(np.full(shape, rho), np.full(shape, ux), np.full(shape, uy),
                     np.full(shape, T), gamma)


def isentropic_vortex(nx=64, ny=64, strength=5.0, radius=5.0, mach=1.2, rho_inf=1.0,
                      T_inf=1.0, noise=1e-3, seed=1, gamma=GAMMA):
    """Shu-type isentropic vortex centred in the box, carried by a uniform
    x-flow at the given Mach number, plus seeded uniform density noise
    (u and T kept, so the noise is an entropy perturbation). At a background
    temperature T_inf the vortex's velocities scale with sqrt(T_inf) and its
    temperatures with T_inf (the same vortex in units of the background's
    sound speed), so that it stays isentropic and in balance."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    xc, yc = nx / 2.0, ny / 2.0
    xb, yb = (x - xc) / radius, (y - yc) / radius
    r2 = xb * xb + yb * yb
    amp = strength / (2.0 * math.pi) * math.sqrt(T_inf) * np.exp(0.5 * (1.0 - r2))
    u_inf = mach * math.sqrt(gamma * T_inf)
    ux = u_inf - amp * yb
    uy = amp * xb
    T = T_inf * (1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * math.pi ** 2) * np.exp(1.0 - r2))
    rho = rho_inf * (T / T_inf) ** (1.0 / (gamma - 1.0))
    rng = np.random.default_rng(seed)
    rho = rho + noise * rng.uniform(-1.0, 1.0, size=rho.shape)
    return conserved(rho, ux, uy, T, gamma)


def riemann_1d(nx=2048, ny=4, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x0=None,
               gamma=GAMMA):
    """Two states (rho, ux, p) split at x0 (default nx/2): Sod's tube by default."""
    x0 = nx // 2 if x0 is None else x0
    x = np.broadcast_to(np.arange(nx, dtype=np.float64), (ny, nx))
    L = x < x0
    rho = np.where(L, left[0], right[0])
    ux = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    return conserved(rho, ux, np.zeros_like(rho), p / rho, gamma)


def riemann_2d(n=200, gamma=GAMMA):
    """Four-quadrant 2D Riemann problem with the quadrant states of the paper's
    Tab. 1 (configuration F of Schulz-Rinne et al., 12 of Lax & Liu).
    Quadrant 1 is x >= n/2, y >= n/2, then counter-clockwise."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    right, top = x >= n / 2, y >= n / 2
    q = np.where(right & top, 1, np.where(~right & top, 2, np.where(~right & ~top, 3, 4)))
    tab = {1: (0.513, 0.0, 0.0, 0.4), 2: (1.0, 0.7276, 0.0, 1.0),
           3: (0.8, 0.0, 0.0, 1.0), 4: (1.0, 0.0, 0.7276, 1.0)}
    rho = np.zeros_like(x); ux = np.zeros_like(x); uy = np.zeros_like(x); p = np.zeros_like(x)
    for k, (r, a, b, pp) in tab.items():
        m = q == k
        rho[m], ux[m], uy[m], p[m] = r, a, b, pp
    return conserved(rho, ux, uy, p / rho, gamma)


def shear_layer(n=4096, mach=2.5, T_cold=0.35, T_ratio=3.0, delta=8.0, amp=1e-2, modes=8,
                seed=3, gamma=GAMMA, ny=None):
    """Periodic double shear layer at y = n/4 and 3n/4: the middle (cold) stream
    moves at +u0, the outer (hot) one at -u0, u0 = mach * sqrt(gamma T_cold),
    with tanh profiles of width delta in velocity and temperature, uniform
    pressure p = T_cold (cold density 1), and seeded sinusoidal transverse
    perturbations in modes 1..modes localised on the layers."""
    ny = n if ny is None else ny
    nx = n
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    u0 = mach * math.sqrt(gamma * T_cold)
    T_hot = T_cold * T_ratio
    y1, y2 = ny / 4.0, 3.0 * ny / 4.0
    s = np.where(y < ny / 2.0, np.tanh((y - y1) / delta), -np.tanh((y - y2) / delta))
    ux = u0 * s
    T = T_cold + (T_hot - T_cold) * 0.5 * (1.0 - s)
    p0 = T_cold
    rho = p0 / T
    rng = np.random.default_rng(seed)
    phases = rng.uniform(0.0, 2.0 * math.pi, size=modes)
    env = np.exp(-((y - y1) / (2.0 * delta)) ** 2) + np.exp(-((y - y2) / (2.0 * delta)) ** 2)
    uy = np.zeros_like(x)
    for k in range(1, modes + 1):
        uy += amp * np.sin(2.0 * math.pi * k * x / nx + phases[k - 1])
    uy *= env
    return conserved(rho, ux, uy, T, gamma)


def shear_wave(nx=100, ny=1, u0=2.0, amp=1e-3, rho0=1.0, T0=0.7, gamma=GAMMA):
    """Sec. IV.B.1: uniform x-flow with a small sinusoidal transverse velocity."""
    x = np.broadcast_to(np.arange(nx, dtype=np.float64), (ny, nx))
    return conserved(np.full((ny, nx), rho0), np.full((ny, nx), u0),
                     amp * np.sin(2.0 * math.pi * x / nx), np.full((ny, nx), T0), gamma)


def entropy_spot(n=100, u0=2.0, amp=1e-3, rho0=1.0, T0=0.7, gamma=GAMMA):
    """Sec. IV.B.2: Gaussian hot spot at constant pressure in a uniform x-flow."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    R = n / 10.0
    r2 = ((x - n / 2.0) ** 2 + (y - n / 2.0) ** 2) / R ** 2
    g = np.exp(-r2)
    return conserved(rho0 * (1.0 - amp * g), np.full_like(x, u0), np.zeros_like(x),
                     T0 * (1.0 + amp * g), gamma)


def acoustic_pulse(n=100, u0=0.3, amp=1e-3, rho0=1.0, T0=0.7, gamma=GAMMA):
    """Sec. IV.B.3: Gaussian pressure pulse P = P0 (1 + A e^{-r^2}),
    r^2 = |x - x_c|^2 / R^2 with R = n / 10, in a uniform x-flow; density and
    temperature from the isentropic relations rho = rho0 (P/P0)^(1/gamma),
    T = T0 (rho/rho0)^(gamma - 1), P0 = rho0 T0."""
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    R = n / 10.0
    r2 = ((x - n / 2.0) ** 2 + (y - n / 2.0) ** 2) / R ** 2
    P0 = rho0 * T0
    P = P0 * (1.0 + amp * np.exp(-r2))
    rho = rho0 * (P / P0) ** (1.0 / gamma)
    T = T0 * (rho / rho0) ** (gamma - 1.0)
    return conserved(rho, np.full_like(x, u0), np.zeros_like(x), T, gamma)


# --------------------------------------------------------------------------
# Batched and serving workloads

@dataclass
class FlowSpec:
    """One independent periodic flow of a batched or served workload."""
    kind: str            # "vortex" | "shear" | "riemann2d" | "sod"
    nx: int
    ny: int
    mach: float
    T_ratio: float
    nu: float
    steps: int
    precision: str = "fp32"   # "fp32" | "fp64"
    seed: int = 0
    arrival: float = 0.0      # seconds from the start of a serving run
    clamped: bool = False     # velocity or temperature clamped to keep the lattice realizable

    def __post_init__(self):
        # The fastest velocity of the flow stays below |u| = 2.5: the carrier
        # velocity (Mach times the background's sound speed) is clamped; this
        # clamp and a vortex's temperature clamp are recorded.
        if self.kind == "vortex":
            T_inf = self.vortex_T_inf()
            self.clamped = T_inf != 0.35 * self.T_ratio
            c = math.sqrt(GAMMA * T_inf)
            u_max = 2.5 - VORTEX_STRENGTH / (2.0 * math.pi) * math.sqrt(T_inf)
        elif self.kind == "shear":
            c = math.sqrt(GAMMA * 0.35)
            u_max = 2.5
        else:
            return
        if self.mach * c > u_max:
            self.mach = u_max / c
            self.clamped = True

    def vortex_T_inf(self, gamma=GAMMA):
        """Background temperature of a vortex: 0.35 times the temperature
        ratio (the shear layer's hot stream), kept within [0.35 / 0.754, 1.2]:
        the core (0.754 T_inf for strength 5) no colder than the shear
        layer's cold stream, 0.35, and the background no hotter than the
        hottest vortex the lattice carries at Mach 1.2-3 with no failed
        rebuild in the oracle (1.3 gives one)."""
        core = 1.0 - (gamma - 1.0) * VORTEX_STRENGTH ** 2 / (8.0 * gamma * math.pi ** 2) * math.e
        return min(max(0.35 * self.T_ratio, 0.35 / core), VORTEX_T_MAX)

    def fields(self, gamma=GAMMA):
        if self.kind == "vortex":
            r = max(5.0, min(self.nx, self.ny) / 12.8)
            return isentropic_vortex(self.nx, self.ny, strength=VORTEX_STRENGTH, radius=r,
                                     mach=self.mach, T_inf=self.vortex_T_inf(gamma),
                                     seed=self.seed, gamma=gamma)
        if self.kind == "shear":
            return shear_layer(self.nx, mach=self.mach, T_cold=0.35, T_ratio=self.T_ratio,
                               delta=8.0, seed=self.seed, gamma=gamma,
                               ny=self.ny)
        if self.kind == "riemann2d":
            return riemann_2d(self.nx, gamma)
        if self.kind == "sod":
            return riemann_1d(self.nx, self.ny, gamma=gamma)
        raise ValueError(self.kind)


def batched_flows(count=256, seed=4, smin=64, smax=1024, steps=500):
    """256 periodic flows, side log-uniform in [smin, smax], vortex or shear
    layer, Mach U(0.5, 3), temperature ratio U(1, 4), nu log-uniform in
    [1e-5, 1e-3], FP32 form."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        side = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        kind = "vortex" if rng.uniform() < 0.5 else "shear"
        mach = rng.uniform(0.5, 3.0)
        ratio = rng.uniform(1.0, 4.0)
        nu = math.exp(rng.uniform(math.log(1e-5), math.log(1e-3)))
        out.append(FlowSpec(kind, side, side, mach, ratio, nu, steps, "fp32", seed=1000 + k))
    return out


def serving_requests(rate=50.0, duration=60.0, seed=5, smin=64, smax=2048, steps_min=100,
                     steps_max=5000):
    """Poisson arrivals at `rate` per second for `duration` seconds; each
    request has a log-uniform side and step count, FP32 or FP64 form, and a
    vortex, shear-layer or 2D Riemann initial state."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    k = 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        side = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        steps = int(round(math.exp(rng.uniform(math.log(steps_min), math.log(steps_max)))))
        prec = "fp32" if rng.uniform() < 0.5 else "fp64"
        kind = ("vortex", "shear", "riemann2d")[int(rng.integers(0, 3))]
        mach = rng.uniform(0.5, 3.0)
        ratio = rng.uniform(1.0, 4.0)
        nu = math.exp(rng.uniform(math.log(1e-5), math.log(1e-3)))
        out.append(FlowSpec(kind, side, side, mach, ratio, nu, steps, prec, seed=2000 + k,
                            arrival=t))
        k += 1
    return out

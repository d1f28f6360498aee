"""ctypes wrapper of the plain FP64 C oracle (oracle/alb_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only users. The product package never imports this
module, and this module imports nothing from the product package.
"""
import ctypes
import os

import numpy as np

from . import build as _build

Q = 21
M = 8
Q49 = 49
M13 = 13
D2Q21, D2Q49 = 21, 49
PERIODIC = 0
ZERO_GRADIENT = 1

OK = 0
ENEWTON = 1
ESINGULAR = 2
EUNREALIZABLE = 3


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("umax", ctypes.c_int),
        ("nu", ctypes.c_double), ("gamma", ctypes.c_double), ("n0", ctypes.c_double),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int), ("sensor", ctypes.c_int),
        ("sensor_eps", ctypes.c_double * 3), ("sensor_alpha", ctypes.c_double * 3),
        ("newton_tol", ctypes.c_double), ("newton_maxit", ctypes.c_int),
        ("overlap", ctypes.c_double), ("overlap_rule", ctypes.c_int),
        ("moments", ctypes.c_int), ("prandtl", ctypes.c_double), ("stencil", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("newton_calls", ctypes.c_longlong), ("newton_iters", ctypes.c_longlong),
        ("newton_failures", ctypes.c_longlong), ("reconstructions", ctypes.c_longlong),
        ("reconstruction_failures", ctypes.c_longlong),
    ]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_bp = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")
_lib = None


# A build of the oracle other than oracle/liboracle.so (used by the tests that
# plant a mistake in a copy of the source and check that a pin catches it).
OVERRIDE_ENV = "ALB_ORACLE_LIB_OVERRIDE"


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(os.environ.get(OVERRIDE_ENV) or _build.build())
        L.ora_velocities.argtypes = [ctypes.c_int, np.ctypeslib.ndpointer(np.int32),
                                     np.ctypeslib.ndpointer(np.int32)]
        L.ora_equilibrium13.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, _dp, _dp,
                                                                ctypes.POINTER(ctypes.c_int)]
        L.ora_equilibrium13.restype = ctypes.c_int
        L.ora_targets13.argtypes = [ctypes.c_double] * 4 + [_dp]
        L.ora_equilibrium.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, _dp, _dp,
                                                              ctypes.POINTER(ctypes.c_int)]
        L.ora_equilibrium.restype = ctypes.c_int
        L.ora_equilibrium4.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int, _dp, _dp,
                                                               ctypes.POINTER(ctypes.c_int)]
        L.ora_equilibrium4.restype = ctypes.c_int
        L.ora_targets.argtypes = [ctypes.c_double] * 4 + [_dp]
        L.ora_select_shift.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.ora_select_shift.restype = ctypes.c_int
        L.ora_select_shift_kept.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double]
        L.ora_select_shift_kept.restype = ctypes.c_int
        L.ora_select_shift_neighbours.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                  ctypes.c_double, ctypes.c_void_p, ctypes.c_int]
        L.ora_select_shift_neighbours.restype = ctypes.c_int
        L.ora_node_moments.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, _dp]
        L.ora_collide_node.argtypes = [ctypes.POINTER(Config), _dp, _dp, ctypes.c_int, ctypes.c_int,
                                       _dp, _dp]
        L.ora_collide_node.restype = ctypes.c_int
        L.ora_grad_populations.argtypes = [ctypes.POINTER(Config), ctypes.c_int, ctypes.c_int] + \
            [ctypes.c_double] * 4 + [_dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.ora_grad_populations.restype = ctypes.c_int
        L.ora_heat_flux.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, _dp]
        L.ora_create.argtypes = [ctypes.POINTER(Config)]
        L.ora_create.restype = ctypes.c_void_p
        L.ora_destroy.argtypes = [ctypes.c_void_p]
        L.ora_init.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.ora_init.restype = ctypes.c_int
        L.ora_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.ora_step.restype = ctypes.c_int
        L.ora_step_forced.argtypes = [ctypes.c_void_p, _bp, _bp]
        L.ora_step_forced.restype = ctypes.c_int
        L.ora_get_moments.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.ora_get_primitives.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.ora_get_shifts.argtypes = [ctypes.c_void_p, _bp, _bp]
        L.ora_get_populations.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.ora_set_state.argtypes = [ctypes.c_void_p, _dp, _dp, _bp, _bp]
        L.ora_get_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(Stats)]
        _lib = L
    return _lib


def make_config(nx, ny, umax=2, nu=1e-3, gamma=1.4, n0=0.5, bc_x=PERIODIC, bc_y=PERIODIC,
                sensor=False, sensor_eps=(0.01, 0.1, 1.0), sensor_alpha=(1.05, 1.35, 1.6),
                newton_tol=1e-12, newton_maxit=50, overlap=0.0, overlap_rule=0, moments=None,
                prandtl=1.0, stencil=D2Q21):
    c = Config()
    c.nx, c.ny, c.umax = nx, ny, umax
    c.nu, c.gamma, c.n0 = nu, gamma, n0
    c.bc_x, c.bc_y, c.sensor = bc_x, bc_y, int(bool(sensor))
    for k in range(3):
        c.sensor_eps[k] = sensor_eps[k]
        c.sensor_alpha[k] = sensor_alpha[k]
    c.newton_tol, c.newton_maxit = newton_tol, newton_maxit
    c.overlap = overlap
    c.overlap_rule = overlap_rule
    c.moments = (13 if stencil == D2Q49 else 8) if moments is None else moments
    c.prandtl = prandtl
    c.stencil = stencil
    return c


def velocities(stencil=D2Q21):
    n = Q49 if stencil == D2Q49 else Q
    x = np.zeros(n, np.int32)
    y = np.zeros(n, np.int32)
    lib().ora_velocities(stencil, x, y)
    return x, y


def equilibrium13(rho, ubx, uby, T, tol=1e-12, maxit=50):
    """The reference solver's 13-moment equilibrium on D2Q49 (App. C.1);
    returns (status, lambda, feq, iters)."""
    lam = np.zeros(M13)
    feq = np.zeros(Q49)
    it = ctypes.c_int(0)
    st = lib().ora_equilibrium13(rho, ubx, uby, T, tol, maxit, lam, feq, ctypes.byref(it))
    return st, lam, feq, it.value


def targets13(rho, ubx, uby, T):
    m = np.zeros(M13)
    lib().ora_targets13(rho, ubx, uby, T, m)
    return m


def equilibrium(rho, ubx, uby, T, tol=1e-12, maxit=50):
    """Numerical equilibrium in the lattice frame; returns (status, lambda, feq, iters)."""
    lam = np.zeros(M)
    feq = np.zeros(Q)
    it = ctypes.c_int(0)
    st = lib().ora_equilibrium(rho, ubx, uby, T, tol, maxit, lam, feq, ctypes.byref(it))
    return st, lam, feq, it.value


def equilibrium4(rho, ubx, uby, T, tol=1e-12, maxit=50):
    """Reduced (4-moment) numerical equilibrium; returns (status, lambda, feq, iters)."""
    lam = np.zeros(4)
    feq = np.zeros(Q)
    it = ctypes.c_int(0)
    st = lib().ora_equilibrium4(rho, ubx, uby, T, tol, maxit, lam, feq, ctypes.byref(it))
    return st, lam, feq, it.value


def targets(rho, ubx, uby, T):
    m = np.zeros(M)
    lib().ora_targets(rho, ubx, uby, T, m)
    return m


def select_shift(u, n0=0.5, umax=2):
    return lib().ora_select_shift(float(u), float(n0), int(umax))


RULE_HISTORY, RULE_NEIGHBOURS = 0, 1


def select_shift_neighbours(u, w, nb, n0=0.5, umax=2):
    arr = (ctypes.c_int * len(nb))(*[int(v) for v in nb])
    return lib().ora_select_shift_neighbours(float(u), float(n0), int(umax), float(w), arr,
                                             len(nb))


def select_shift_kept(u, current, w, n0=0.5, umax=2):
    return lib().ora_select_shift_kept(float(u), float(n0), int(umax), int(current), float(w))


def node_moments(f, g, Ux, Uy, gamma=1.4):
    out = np.zeros(4)
    lib().ora_node_moments(len(f), np.ascontiguousarray(f, np.float64),
                           np.ascontiguousarray(g, np.float64), int(Ux), int(Uy), gamma, out)
    return out


def _q(cfg):
    return Q49 if cfg.stencil == D2Q49 else Q


def collide_node(cfg, f, g, Ux, Uy):
    fs = np.zeros(_q(cfg))
    gs = np.zeros(_q(cfg))
    st = lib().ora_collide_node(ctypes.byref(cfg), np.ascontiguousarray(f, np.float64),
                                np.ascontiguousarray(g, np.float64), int(Ux), int(Uy), fs, gs)
    return st, fs, gs


def grad_populations(cfg, Ux, Uy, rho, ux, uy, T, du, dT, omega, w_pr=0.0):
    f = np.zeros(_q(cfg))
    g = np.zeros(_q(cfg))
    st = lib().ora_grad_populations(ctypes.byref(cfg), int(Ux), int(Uy), rho, ux, uy, T,
                                    np.ascontiguousarray(du, np.float64).reshape(4),
                                    np.ascontiguousarray(dT, np.float64), omega, w_pr, f, g)
    return st, f, g


def heat_flux(f, g, Ux, Uy, ux, uy):
    q = np.zeros(2)
    lib().ora_heat_flux(len(f), np.ascontiguousarray(f, np.float64),
                        np.ascontiguousarray(g, np.float64), int(Ux), int(Uy), float(ux), float(uy),
                        q)
    return q


class Simulation:
    """One oracle flow. Fields are (ny, nx) arrays, x fastest."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.nx, self.ny = cfg.nx, cfg.ny
        self._h = lib().ora_create(ctypes.byref(cfg))
        if not self._h:
            raise ValueError("oracle: invalid configuration")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ora_destroy(h)
            self._h = None

    def init(self, rho, rhoux, rhouy, rhoE):
        arrs = [np.ascontiguousarray(a, np.float64).reshape(-1) for a in (rho, rhoux, rhouy, rhoE)]
        return lib().ora_init(self._h, *arrs)

    def step(self, n):
        return lib().ora_step(self._h, int(n))

    def step_forced(self, ux, uy):
        """One step pulling into the given lattices (arrays (ny, nx) of shifts)."""
        return lib().ora_step_forced(self._h, np.ascontiguousarray(ux, np.int8).reshape(-1),
                                     np.ascontiguousarray(uy, np.int8).reshape(-1))

    def moments(self):
        n = self.nx * self.ny
        out = [np.zeros(n) for _ in range(4)]
        lib().ora_get_moments(self._h, *out)
        return [a.reshape(self.ny, self.nx) for a in out]

    def primitives(self):
        n = self.nx * self.ny
        out = [np.zeros(n) for _ in range(4)]
        lib().ora_get_primitives(self._h, *out)
        return [a.reshape(self.ny, self.nx) for a in out]

    def shifts(self):
        n = self.nx * self.ny
        ux = np.zeros(n, np.int8)
        uy = np.zeros(n, np.int8)
        lib().ora_get_shifts(self._h, ux, uy)
        return ux.reshape(self.ny, self.nx), uy.reshape(self.ny, self.nx)

    def populations(self):
        n, q = self.nx * self.ny, _q(self.cfg)
        f = np.zeros(n * q)
        g = np.zeros(n * q)
        lib().ora_get_populations(self._h, f, g)
        return f.reshape(self.ny, self.nx, q), g.reshape(self.ny, self.nx, q)

    def set_state(self, f, g, ux, uy):
        lib().ora_set_state(self._h, np.ascontiguousarray(f, np.float64).reshape(-1),
                            np.ascontiguousarray(g, np.float64).reshape(-1),
                            np.ascontiguousarray(ux, np.int8).reshape(-1),
                            np.ascontiguousarray(uy, np.int8).reshape(-1))

    def stats(self):
        s = Stats()
        lib().ora_get_stats(self._h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

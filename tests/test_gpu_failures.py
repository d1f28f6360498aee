"""Failure detection made on the host, none of it faulting the GPU.

* Root-finder failure (Sec. II.C.2: the numerical equilibrium exists only
  where the root finder converges): a flow whose Newton iterations are capped
  below what some of its states need. alb_sync must report ALB_ENEWTON, the
  counts of failed collisions and failed rebuilds must equal the oracle's
  under the same cap, and a failed node must be left uncollided, population
  for population (the failure policy: uncollided node, Maxwellian-guess
  exponential for a failed rebuild), as the oracle does.
* A bounded wait that runs out: alb_sync with a 1 ms limit on a queued
  multi-step run returns ALB_ETIMEDOUT, and a later unbounded alb_sync
  completes the same run.
* The same for the serving loop's drain.
"""
import math
import time

import numpy as np
import pytest

import oracle as O
from paper_2009_13426_gb300 import flows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, NU, CAP, STEPS = 32, 1e-3, 5, 8


@pytest.fixture(scope="module")
def alb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13426_gb300 import alb as A
    A.lib()
    return A


def two_region_pulse(n=N, amp=0.6):
    """A band moving at u_x = 0.45 between two bands at rest, all in lattice
    (0, 0), and a pressure pulse in the middle whose expansion carries nodes
    past u_x = 1/2 into lattice (1, 0). From the Maxwellian start the resting
    states need five Newton steps, the moving ones six, so a cap of five
    makes some collisions fail and not others; the rebuilds at the lattice
    interfaces fail under it too."""
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    ux = 0.45 * 0.5 * (np.tanh((yy - n / 4) / 1.5) - np.tanh((yy - 3 * n / 4) / 1.5))
    p = 0.7 * (1 + amp * np.exp(-((xx - n / 2) ** 2 + (yy - n / 2) ** 2) / 16))
    T = 0.7 * (p / 0.7) ** (0.4 / 1.4)
    return flows.conserved(p / T, ux, 0 * ux, T)


def test_capped_root_finder_fails_like_the_oracle(alb):
    fields = two_region_pulse()
    # The initial state and its first collision under the default root finder,
    # on both sides; the first pull changes no lattice (checked), so from
    # there on every solve runs under the cap.
    ga = alb.Flow(N, N, nu=NU, precision=alb.ALB_FP64_PLAIN)
    ga.init(*fields)
    ckpt = ga.checkpoint()
    ga.close()
    oa = O.Simulation(O.make_config(N, N, nu=NU))
    assert oa.init(*fields) == O.OK
    assert oa.step(1) == O.OK
    assert oa.stats()["reconstructions"] == 0
    f1, g1 = oa.populations()
    sx1, sy1 = oa.shifts()

    gb = alb.Flow(N, N, nu=NU, precision=alb.ALB_FP64_PLAIN, newton_maxit=CAP)
    gb.restore(ckpt)
    s0 = gb.stats()
    gb.step(STEPS)
    with pytest.raises(alb.AlbError) as ei:
        gb.sync()
    assert ei.value.code == alb.ALB_ENEWTON
    s1 = gb.stats()
    d = {k: s1[k] - s0[k] for k in s1}

    cfg = O.make_config(N, N, nu=NU, newton_maxit=CAP)
    ob = O.Simulation(cfg)
    ob.set_state(f1, g1, sx1, sy1)
    assert ob.step(STEPS - 1) == O.ENEWTON
    ost = ob.stats()
    # the GPU's last collision is the oracle's next one, node by node
    f, g = ob.populations()
    sx, sy = ob.shifts()
    fs = np.empty_like(f)
    gs = np.empty_like(g)
    last_fail = 0
    for j in range(N):
        for i in range(N):
            st, a, b = O.collide_node(cfg, f[j, i], g[j, i], int(sx[j, i]), int(sy[j, i]))
            if st != O.OK:
                last_fail += 1
                assert np.array_equal(a, f[j, i]) and np.array_equal(b, g[j, i])
            fs[j, i], gs[j, i] = a, b
    assert d["newton_failures"] == ost["newton_failures"] + last_fail
    assert 0 < d["newton_failures"] < d["node_updates"]
    assert d["reconstructions"] == ost["reconstructions"] > 0
    assert d["reconstruction_failures"] == ost["reconstruction_failures"] > 0
    # moments and lattices of the pulled state
    r, a, b, e = gb.moments()
    R, A, B, E = ob.moments()
    for x, y in ((r, R), (a, A), (b, B), (e, E)):
        assert np.abs(x - y).max() <= 1e-11 * np.abs(y).max()
    gx, gy = gb.shifts()
    assert (gx == sx).all() and (gy == sy).all()
    assert (gx == 1).any()
    # post-collision populations: collided where the root finder converged,
    # the pulled populations unchanged where it failed
    pf, pg = gb.populations()
    pf = np.moveaxis(pf, 0, -1)
    pg = np.moveaxis(pg, 0, -1)
    scale = np.abs(fs).max(axis=-1, keepdims=True)
    assert (np.abs(pf - fs) <= 1e-11 * scale).all()
    assert (np.abs(pg - gs) <= 1e-11 * np.abs(gs).max(axis=-1, keepdims=True)).all()
    gb.close()


def test_bounded_sync_times_out_then_completes(alb):
    n, steps = 2048, 40
    fl = alb.Flow(n, n, nu=1e-5, precision=alb.ALB_FP32_FORM, sensor=1)
    fl.init(*flows.shear_layer(n))
    fl.sync()
    t0 = time.perf_counter()
    fl.step(steps)
    with pytest.raises(alb.AlbError) as ei:
        fl.sync(1)
    assert ei.value.code == alb.ALB_ETIMEDOUT
    assert time.perf_counter() - t0 < 5.0
    assert fl.sync(-1) == alb.ALB_OK
    assert fl.stats()["steps"] == steps
    r = fl.moments()[0]
    assert np.isfinite(r).all()
    fl.close()


def test_server_drain_times_out_then_completes(alb):
    srv = alb.Server()
    try:
        n = 1024
        rid = srv.submit(300, fields=flows.shear_layer(n), nx=n, ny=n, nu=1e-5, sensor=1,
                         precision=alb.ALB_FP32_FORM)
        with pytest.raises(alb.AlbError) as ei:
            srv.drain(1)
        assert ei.value.code == alb.ALB_ETIMEDOUT
        srv.drain(-1)
        st, res = srv.poll(rid)
        assert st == alb.ALB_DONE and res["status"] == alb.ALB_OK and res["steps"] == 300
        assert math.isfinite(float(res["moments"][0].sum()))
    finally:
        srv.close()

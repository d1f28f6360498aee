"""The FP32 form on a 256^2 shear layer over 200 steps (the recipe of the
4096^2 benchmark flow: Mach 2.5 cold stream, temperature ratio 3, tanh width
8, nu = 1e-5, kinetic sensor on), against the FP64 oracle.

Two comparisons:
* replayed: the oracle steps with the GPU's lattice decisions, which isolates
  the arithmetic of the step: <= 1e-5 relative (max norm);
* free-running: the oracle takes its own decisions. Eq. criterion compares u
  with half-integers; where the FP32 sums put u on the other side of a
  threshold than the FP64 oracle does, that node changes lattice (every pull
  rebuilt, an O(1e-2) change at that node) and the two runs part there. The
  test counts those flipped decisions and bounds the free-running error.
The figures are written to the test's output (pytest -s)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2009_13426_gb300 import flows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, STEPS, NU = 256, 200, 1e-5
FP32_TOL = 1e-5
# stated bounds of the free-running comparison (measured on one GB300: max_rel
# 2.3e-2, l2_rel 2.5e-3 from two flipped decisions in 13 M node-steps)
FREE_MAX_REL = 5e-2
FREE_L2_REL = 1e-2


@pytest.fixture(scope="module")
def alb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13426_gb300 import alb as A
    A.lib()
    return A


def errors(got, ref):
    r, a, b, e = got
    R, A, B, E = ref
    dm = np.sqrt((a - A) ** 2 + (b - B) ** 2)
    mm = np.sqrt(A ** 2 + B ** 2)
    mx = max(np.abs(r - R).max() / np.abs(R).max(), dm.max() / mm.max(),
             np.abs(e - E).max() / np.abs(E).max())
    l2 = max(np.linalg.norm(r - R) / np.linalg.norm(R), np.linalg.norm(dm) / np.linalg.norm(mm),
             np.linalg.norm(e - E) / np.linalg.norm(E))
    return mx, l2


def criterion(u, n0=0.5, umax=2):
    """Eq. criterion on an array: U = n iff n - n0 < u <= n + 1 - n0, clamped
    (for counting decisions only; the oracle's own function is pinned
    elsewhere)."""
    return np.clip(np.ceil(u + n0) - 1, -umax, umax).astype(np.int8)


def test_shear_layer_256_fp32_form_against_the_oracle(alb):
    fields = flows.shear_layer(N)
    okw = dict(umax=2, nu=NU, sensor=True)
    fl = alb.Flow(N, N, u_max=2, nu=NU, precision=alb.ALB_FP32_FORM, sensor=1)
    fl.init(*fields)
    rep = O.Simulation(O.make_config(N, N, **okw))
    assert rep.init(*fields) == O.OK
    flips = 0
    for _ in range(STEPS):
        r, ux, uy, T = rep.primitives()  # the moments of this step's collision
        fx, fy = criterion(ux), criterion(uy)
        fl.step(1)
        gx, gy = fl.shifts()
        flips += int((gx != fx).sum() + (gy != fy).sum())
        assert rep.step_forced(gx, gy) == O.OK
    fl.sync()
    got = fl.moments()
    gsx, gsy = fl.shifts()
    st = fl.stats()
    fl.close()
    free = O.Simulation(O.make_config(N, N, **okw))
    assert free.init(*fields) == O.OK
    assert free.step(STEPS) == O.OK
    fsx, fsy = free.shifts()
    rep_max, rep_l2 = errors(got, rep.moments())
    free_max, free_l2 = errors(got, free.moments())
    final_differ = int((gsx != fsx).sum() + (gsy != fsy).sum())
    print("\nshear layer %d^2, %d steps, FP32 form vs FP64 oracle: replayed max_rel %.3e "
          "l2_rel %.3e; free-running max_rel %.3e l2_rel %.3e; flipped decisions %d "
          "(%.2e per node-step); lattices differing at the end %d; rebuilt pulls per node-step "
          "%.4f" % (N, STEPS, rep_max, rep_l2, free_max, free_l2, flips,
                    flips / (N * N * STEPS), final_differ,
                    st["reconstructions"] / (N * N * STEPS)))
    assert st["newton_failures"] == 0 and st["reconstruction_failures"] == 0
    assert rep_max <= FP32_TOL
    assert free_max <= FREE_MAX_REL and free_l2 <= FREE_L2_REL
    assert flips <= 1e-4 * N * N * STEPS
    assert math.isfinite(free_max)

"""The benchmark's shear layer through the C ABI, as a small case for profilers.

The n^2 periodic double shear layer of the benchmark's recipe (Mach 2.5 cold
stream, temperature ratio 3, nu 1e-5, kinetic sensor on), FP32 form unless
--fp64. Three uses:

  python -m paper_2009_13426_gb300.shear_case --n 1024 --steps 3
      alb_init, then `steps` launches of the step kernel;
  python -m paper_2009_13426_gb300.shear_case --n 1024 --advance 1900 --steps 0 --save F
      advance 1900 steps and write an alb_checkpoint to the file F;
  python -m paper_2009_13426_gb300.shear_case --n 1024 --load F --steps 3
      restore the checkpoint F into a new flow, then `steps` launches, so a
      profiler sees the developed flow after a handful of launches.

Prints the flow's counters per node update of the stepped launches.
"""
import argparse
import os
import sys

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2009_13426_gb300 import alb, flows  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--advance", type=int, default=0)
    ap.add_argument("--save", default=None)
    ap.add_argument("--load", default=None)
    ap.add_argument("--fp64", action="store_true")
    a = ap.parse_args(argv)
    n = a.n
    prec = alb.ALB_FP64_PLAIN if a.fp64 else alb.ALB_FP32_FORM
    fl = alb.Flow(n, n, u_max=2, nu=1e-5, precision=prec, sensor=1)
    fl.init(*flows.shear_layer(n))
    if a.load:
        fl.restore(np.load(a.load))
    left = a.advance
    while left > 0:
        fl.step(min(100, left))
        left -= min(100, left)
    fl.sync()
    s0 = fl.stats()
    fl.step(a.steps)
    fl.sync()
    s1 = fl.stats()
    k = max(1, a.steps) * n * n
    print({key: round((s1[key] - s0[key]) / k, 4) for key in s1 if key != "steps"})
    if a.save:
        np.save(a.save, fl.checkpoint())
    fl.close()


if __name__ == "__main__":
    main()

"""Work model of the step kernel, used for the roofline of the benchmark.

The step is bound by the FP64 pipe, not by HBM: on GB300 the FP64 rate is
1/62 of the FP32 rate. Its arithmetic is counted in FP64 issue slots: one slot per
DFMA/DADD/DMUL/DMNMX/DSETP lane-operation, and for the FP64 routines the
measured cost relative to a DFMA of a throughput microbenchmark on GB300:
exp 20.2 slots, divide/reciprocal 10.2 slots, square root 10, log 20. The
counts below come from the structure of the kernel's unrolled loops over the
D2Q21 velocity table (only non-zero monomials are touched).

A slot is one FMA: the FP64 roofline peak is 152 SMs x 2 FP64 FMA/clk/SM x
2 flop x 2.07 GHz = 1.259 TFLOP/s (the GB300's quoted dense FP64 rate), and
achieved FLOP/s = 2 x slots / time.

Bytes per node update (algorithmic, one read and one write of every plane):
FP32 form 42*4*2 + 4*4 (moments written) + 2 + 2 (lattice codes) = 356 B;
FP64 plain 42*8*2 + 4*8 + 4 = 708 B.
"""
from __future__ import annotations

W_EXP = 20.2
W_DIV = 10.2
W_SQRT = 10.0
W_LOG = 20.0

FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 1.2586

# Ratio of the FP64-pipe thread instructions that ncu counted for one launch
# of the step kernel (1024^2 shear layer, FP32 form: 9235 per node) to the
# slots this model gives for the same launch (11536 per node). It absorbs the
# difference between the microbenchmark's routine costs and their cost inside
# the kernel. It must be measured again whenever the kernel changes.
CALIBRATION = 9235.0 / 11536.0

BYTES_PER_NODE = {"fp32": 42 * 4 * 2 + 4 * 4 + 4, "fp64": 42 * 8 * 2 + 4 * 8 + 4}

_XI = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1),
       (2, 0), (0, 2), (-2, 0), (0, -2), (2, 2), (-2, 2), (-2, -2), (2, -2),
       (3, 0), (0, 3), (-3, 0), (0, -3)]


def _mono(k, x, y):
    r2 = x * x + y * y
    return (1, x, y, x * x, x * y, y * y, x * r2, y * r2)[k]


def _nnz(k):
    return sum(1 for x, y in _XI if _mono(k, x, y) != 0)


def _nnz2(a, b):
    return sum(1 for x, y in _XI if _mono(a, x, y) * _mono(b, x, y) != 0)


def slots_exp_family():
    """21 exponents (1 + lambda_0 plus the non-zero monomials) and 21 exp."""
    ops = sum(1 + sum(1 for k in range(1, 8) if _mono(k, x, y) != 0) for x, y in _XI)
    return ops + 21 * W_EXP


def slots_eval():
    """One evaluation: exponentials plus the dual value (21 adds + 8 FMA)."""
    return slots_exp_family() + 21 + 8


def slots_newton_step():
    """Residual, Jacobian, Cholesky, two triangular solves, step, line-search
    bookkeeping (the line-search evaluation itself is counted as an eval)."""
    g = sum(_nnz(k) for k in range(8)) + 8
    h = sum(_nnz2(a, b) for a in range(8) for b in range(a + 1))
    chol = 0.0
    for j in range(8):
        chol += j + 1 + W_SQRT + W_DIV + sum(j + 1 for _ in range(j + 1, 8))
    solves = 2 * (28 + 8 * W_DIV)
    return g + h + chol + solves + 8 + 8 + 4


def slots_call():
    """Targets, Maxwellian guess (reciprocal, normalisation, log)."""
    return 8 + W_DIV + 4 + 21 + W_LOG


def slots_collision(precision):
    if precision == "fp64":
        return 90 + 3 * W_DIV + 5 + 2 + 8 + (W_DIV + 1) + W_DIV + 21 * 7 + 2
    return 5 + 3 * W_DIV + 2 + 8 + (W_DIV + 1) + W_DIV + 21 * 3 + 2


def slots_rebuild_extra():
    return 12 + 2 + 2 + 2 * (W_DIV + 1) + (8 + W_EXP) + (40 + 3 * W_DIV) + 8


def fp64_slots(stats: dict, precision: str) -> float:
    """FP64 slots of the work recorded by the kernel counters (a stats delta),
    scaled by the ncu calibration of the kernel."""
    return CALIBRATION * (stats["fp64_evaluations"] * slots_eval()
            + stats["newton_iterations"] * slots_newton_step()
            + stats["newton_calls"] * slots_call()
            + stats["node_updates"] * slots_collision(precision)
            + stats["reconstructions"] * slots_rebuild_extra())


def describe():
    return {
        "slots_per_eval": round(slots_eval(), 1),
        "slots_per_newton_step": round(slots_newton_step(), 1),
        "slots_per_call": round(slots_call(), 1),
        "slots_per_collision_fp32": round(slots_collision("fp32"), 1),
        "slots_per_collision_fp64": round(slots_collision("fp64"), 1),
        "slots_per_rebuild_extra": round(slots_rebuild_extra(), 1),
        "fp64_peak_tflops": round(FP64_PEAK_TFLOPS, 4),
        "calibration": round(CALIBRATION, 4),
    }


if __name__ == "__main__":
    print(describe())

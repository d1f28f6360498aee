"""Work model of the step kernel, used for the roofline of the benchmark.

The step is bound by the FP64 pipe, not by HBM: on GB300 the FP64 rate is
1/62 of the FP32 rate. Its FP64 arithmetic is counted in issue slots: one
slot per FP64 lane operation (DFMA, DADD, DMUL, DMNMX, DSETP, hardware
conversions to or from FP64; the FP32 form's hot conversions are assembled
on the integer pipe instead and cost no slot), and for CUDA's FP64 routines
their measured cost in slots
(throughput microbenchmark on GB300, independent chains, loop overhead
removed): exp 18.2, divide/reciprocal 9.2, square root 10, log 20. The counts
come from the structure of the kernel's unrolled code over the D2Q21 velocity
table. The kernel's device counters give the number of each unit of work in
a launch (equilibrium solves, FP64 residual evaluations, full FP64 Newton
steps, rebuilt pulls, node updates).

A slot is one FMA: the FP64 roofline peak is 152 SMs x 2 FP64 FMA/clk/SM x
2 flop x 2.07 GHz = 1.259 TFLOP/s (the GB300's quoted dense FP64 rate), and
achieved FLOP/s = 2 x slots / time.

Bytes per node update (algorithmic, one read and one write of every plane):
FP32 form 42*4*2 + 4*4 (moments written) + 2 + 2 (lattice codes) + 8*4*2
(multipliers of the warm start) = 420 B; FP64 plain 42*8*2 + 4*8 + 4 + 8*8*2
= 836 B.
"""
from __future__ import annotations

W_EXP = 18.2
W_DIV = 9.2
W_SQRT = 10.0
W_LOG = 20.0

FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 1.2586

# Ratio of the FP64-pipe instructions ncu counted for one launch of each
# step kernel to the slots this model gives for the same launch; it absorbs
# what the hand count misses (compiler scheduling, predication) and is
# measured again whenever a kernel changes.
CALIBRATION = {"fp32": 405.4 / 385.2, "fp64": 5573.7 / 6073.3}

BYTES_PER_NODE = {"fp32": 42 * 4 * 2 + 4 * 4 + 4 + 8 * 4 * 2,
                  "fp64": 42 * 8 * 2 + 4 * 8 + 4 + 8 * 8 * 2}

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


# ---------------------------------------------------------------- FP64 plain

# The groups of the D2Q21 set: the rest velocity, six symmetric axis pairs
# (point indices), two diagonal quadruples.
_PAIRS = [(1, 3), (2, 4), (9, 11), (10, 12), (17, 19), (18, 20)]
_QUADS = [(5, 6, 7, 8), (13, 14, 15, 16)]


def _pm(k, i):
    return _mono(k, *_XI[i])


def plain_eval():
    """Grouped exponents (55), 21 table-driven exponentials (9 each), grouped
    constraint sums incl. sum p (68), dual value lambda . m (8)."""
    return 55 + 21 * 9 + 68 + 8


def plain_jacobian():
    """Jacobian from the groups: one FMA per non-zero coefficient and group,
    plus the pair sums/differences and the quadruple butterflies."""
    n = 0
    for ip, _ in _PAIRS:
        n += 2 + sum(1 for a in range(8) for b in range(a + 1) if _pm(a, ip) * _pm(b, ip) != 0)
    for q in _QUADS:
        n += 8 + sum(1 for a in range(8) for b in range(a + 1) if _pm(a, q[0]) * _pm(b, q[0]) != 0)
    return n


def plain_newton_step():
    """Residual and its maximum, grouped Jacobian, Cholesky with reciprocal
    pivots, two triangular solves by multiplication, step and line-search
    bookkeeping (the line-search evaluation itself is an eval)."""
    g = 8 + 8
    chol = sum(j + W_SQRT + W_DIV + (7 - j) * (j + 1) for j in range(8))
    solves = 2 * (28 + 8)
    return g + plain_jacobian() + chol + solves + 8 + 8 + 4


def plain_call():
    """Targets, Maxwellian start (reciprocal of T, log and reciprocal of the
    normalisation, scaling of the 21 populations and 8 sums)."""
    return 8 + W_DIV + 4 + W_LOG + W_DIV + 21 + 8


# ---------------------------------------------------------------- FP32 form

def mixed_eval():
    """FP64 residual evaluation of the refinement: grouped exponents (55),
    21 table-driven exponentials (4 each: the one-step reduction, the
    degree-2 polynomial 2, the scaling; the table index comes from an FP32
    copy of the exponent and reaches FP64 through the integer pipe), grouped
    constraint sums started at -m so that they end as the residual (68). Its
    FP32 copy is rounded on the integer pipe (its maximum is taken in FP32,
    and the FP32 corrections join the FP64 multipliers only before a further
    full evaluation)."""
    return 55 + 21 * 4 + 68


def mixed_update():
    """Multiplicative FP64 update of the refinement after a small step: per
    velocity one FMA with the FP32 factor exp(-d) - 1 (21; the exponent
    changes d are FP32, the factor reaches FP64 through the integer pipe),
    grouped constraint sums started at -m (68); the residual's FP32 copy is
    rounded on the integer pipe."""
    return 21 + 68


def mixed_call():
    """Targets (the inputs and the FP32 multipliers change precision on the
    integer pipe)."""
    return 8


COLLISION = {
    # FP64 part only: one reciprocal of rho and 8 operations for u and T,
    # the velocities in the absolute frame (2); the FP32 sums, the FP32 view
    # of the equilibrium column, T, rho and the stored moments change
    # precision on the integer pipe, the criterion compares there too, tau,
    # the sensor and BGK run in FP32, and the stored multipliers come out of
    # the solver in FP32
    "fp32": W_DIV + 8 + 2,
    "fp64": 90 + 3 * W_DIV + 5 + 2 + 24 + (W_DIV + 1) + W_DIV + 21 * 7 + 2,
}

REBUILD_EXTRA = {
    # conversions of the sender's moments, central differences, relaxation
    # factors, the one population (exponent + exp), Grad factors
    "fp32": 12 + 12 + 2 + 2 * W_DIV + 2 + (8 + 11) + 1 + 4 + (40 + 3 * W_DIV) + 6,
    "fp64": 12 + 2 + 2 + 2 * (W_DIV + 1) + (8 + W_EXP) + (40 + 3 * W_DIV) + 8,
}


def fp64_slots(stats: dict, precision: str) -> float:
    """FP64 slots of the work recorded by the kernel counters (a stats delta)."""
    if precision == "fp32":
        raw = (stats["fp64_evaluations"] * mixed_eval()
               + stats.get("fp64_updates", 0) * mixed_update()
               + stats["newton_calls"] * mixed_call())
        # full FP64 Newton fallback, if any: its steps and evaluations
        raw += stats["newton_iterations"] * (plain_newton_step() + plain_eval() - mixed_eval())
    else:
        raw = (stats["fp64_evaluations"] * plain_eval()
               + stats["newton_iterations"] * plain_newton_step()
               + stats["newton_calls"] * plain_call())
    raw += stats["node_updates"] * COLLISION[precision]
    raw += stats["reconstructions"] * REBUILD_EXTRA[precision]
    return CALIBRATION[precision] * raw


def method_floor(mlups: float) -> dict:
    """The method's own minimum FP64 work per node update, beside the count of
    what the kernel executes: one FP64 evaluation of the equilibrium (the
    grouped exponents of the 21 velocities, their table exponentials, the 8
    constraint sums), the least a solve needs to confirm max|G|/rho <= 1e-12
    in FP64 (App. C.1). Returns that count, the MLUPS the FP64 pipe would
    allow if it were all the work, and the fraction of it `mlups` reaches."""
    slots = 55 + 21 * 4 + 68
    cap = FP64_PEAK_TFLOPS * 1e12 / 2.0 / slots / 1e6
    return {"fp64_slots_per_node": slots, "mlups_at_fp64_peak": round(cap, 1),
            "frac": round(mlups / cap, 4)}


def describe():
    return {
        "plain_eval": round(plain_eval(), 1),
        "plain_newton_step": round(plain_newton_step(), 1),
        "plain_call": round(plain_call(), 1),
        "mixed_eval": round(mixed_eval(), 1),
        "mixed_update": round(mixed_update(), 1),
        "mixed_call": round(mixed_call(), 1),
        "collision": {k: round(v, 1) for k, v in COLLISION.items()},
        "rebuild_extra": {k: round(v, 1) for k, v in REBUILD_EXTRA.items()},
        "fp64_peak_tflops": round(FP64_PEAK_TFLOPS, 4),
        "calibration": CALIBRATION,
    }


if __name__ == "__main__":
    print(describe())


# ---------------------------------------------------------------- D2Q49

# Slots of the D2Q49 step (alb_q49.cu), counted like the rest of this file:
# per Newton step, moments from the row sums (664), residual and its maximum
# (45), Jacobian entries from the moments (140), Cholesky with reciprocal
# pivots (690), two triangular solves (182), one line-search evaluation of
# the 49 exponentials with the dual value (1060); per solve, targets, the
# Maxwellian start's evaluation, log and normalisation (1220); per node,
# moments, shift choice and BGK store (550); per rebuilt pull, the sender's
# central differences, its exponential from the shared solve's multipliers
# and the Grad factors (107).
Q49_PER_ITER = 664 + 45 + 140 + 690 + 182 + 13 + 1060
Q49_PER_CALL = 1220
Q49_PER_NODE = 550
Q49_PER_REBUILD = 12 + 9 + 9 + 1 + 40 + 3 * W_DIV + 8
# ncu counted 30,696 FP64-pipe thread instructions per node on the 512^2
# shear layer (7.10 Newton steps, 1.26 solves, 1.32 rebuilt pulls per node),
# where the count above gives 22,067.
CALIBRATION["q49"] = 30696.0 / 22067.0


def q49_slots(delta, node_updates):
    """FP64 slots of D2Q49 launches from their counters."""
    rebuilds = delta["reconstructions"]
    raw = (Q49_PER_ITER * delta["newton_iterations"] + Q49_PER_CALL * delta["newton_calls"]
           + Q49_PER_NODE * node_updates + Q49_PER_REBUILD * rebuilds)
    return CALIBRATION["q49"] * raw

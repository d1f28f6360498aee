"""The work model behind the benchmark's roofline (CPU only): the unit costs
are consistent with the kernel's structure, and the slots follow the device
counters, including the FP32 form's multiplicative updates."""
import pytest

from paper_2009_13426_gb300 import costmodel as C


def base_stats(**kw):
    st = {"newton_iterations": 0, "newton_calls": 100, "fp64_evaluations": 100,
          "fp64_updates": 0, "fp32_iterations": 80, "reconstructions": 5, "node_updates": 100}
    st.update(kw)
    return st


def test_update_is_cheaper_than_an_evaluation():
    # an update replaces the 21 exponents and exponentials by one FMA per
    # velocity; the constraint sums are shared, and every change of precision
    # runs on the integer pipe (no FP64 slot)
    shared = 68
    assert C.mixed_eval() - shared == 55 + 21 * 4
    assert C.mixed_update() - shared == 21
    assert C.mixed_update() < C.mixed_eval()


def test_slots_follow_the_counters():
    s0 = C.fp64_slots(base_stats(), "fp32")
    s1 = C.fp64_slots(base_stats(fp64_updates=50), "fp32")
    assert s1 - s0 == pytest.approx(50 * C.mixed_update() * C.CALIBRATION["fp32"])
    s2 = C.fp64_slots(base_stats(fp64_evaluations=150), "fp32")
    assert s2 - s0 == pytest.approx(50 * C.mixed_eval() * C.CALIBRATION["fp32"])


def test_counters_without_updates_are_accepted():
    st = base_stats()
    del st["fp64_updates"]
    assert C.fp64_slots(st, "fp32") == C.fp64_slots(base_stats(), "fp32")


def test_calibrations_are_near_the_hand_count():
    # ncu's FP64-pipe instruction count against the model's slots for the
    # same launches: the hand count may miss a little, not a factor
    for k in ("fp32", "fp64"):
        assert 0.8 < C.CALIBRATION[k] < 1.1, k
    assert 1.0 < C.CALIBRATION["q49"] < 1.6


def test_peak_is_the_fp64_unit_count():
    assert C.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)


def test_method_floor_is_one_fp64_evaluation():
    # one FP64 evaluation of the equilibrium: the least FP64 work a solve
    # needs; at the FP64 peak it allows this rate
    f = C.method_floor(500.0)
    assert f["fp64_slots_per_node"] == C.mixed_eval()
    cap = 152 * 2 * 2.07e9 / f["fp64_slots_per_node"] / 1e6
    assert f["mlups_at_fp64_peak"] == pytest.approx(cap, rel=1e-3)
    assert f["frac"] == pytest.approx(500.0 / cap, rel=1e-3)


def test_fp32_calibration_is_the_profiled_capture():
    # the FP32 form's factor is ncu's FP64-pipe thread instructions per node
    # (405.4, 1024^2 shear layer, first three launches) over this model's
    # slots for the counters of the same launches: 1.0973 solves and full
    # evaluations, 1.1581 multiplicative updates, 0.1875 rebuilt pulls
    st = {"newton_iterations": 0, "newton_calls": 1.0973, "fp64_evaluations": 1.0973,
          "fp64_updates": 1.1581, "reconstructions": 0.1875, "node_updates": 1.0}
    raw = C.fp64_slots(st, "fp32") / C.CALIBRATION["fp32"]
    assert raw == pytest.approx(385.2, abs=0.05)
    assert C.fp64_slots(st, "fp32") == pytest.approx(405.4, abs=0.05)

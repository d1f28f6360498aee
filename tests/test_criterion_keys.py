"""The step kernel compares velocities with the criterion's thresholds on the
integer pipe: a double's bits mapped to a signed key in IEEE order (negative
values with their magnitude bits flipped). This CPU test restates that map
and checks the order it gives against IEEE comparisons, and that the host's
thresholds are never -0, the one value pair (+0 against -0) where the two
orders differ."""
import numpy as np

MAG = np.int64(0x7FFFFFFFFFFFFFFF)


def order_key(v):
    b = np.asarray(v, dtype=np.float64).view(np.int64)
    return b ^ ((b >> np.int64(63)) & MAG)


def test_key_order_is_ieee_order():
    rng = np.random.default_rng(11)
    vals = np.concatenate([
        rng.normal(0.0, 3.0, 4000),
        rng.normal(0.0, 1e-300, 200),
        np.array([0.0, 1.0, -1.0, 0.5, -0.5, 1.5, -1.5, 2.5, -2.5, np.inf, -np.inf,
                  5e-324, -5e-324, 1.7976931348623157e308, -1.7976931348623157e308]),
        np.nextafter(np.array([0.5, -0.5, 1.49, -1.51]), np.inf),
        np.nextafter(np.array([0.5, -0.5, 1.49, -1.51]), -np.inf),
    ])
    k = order_key(vals)
    a, b = np.meshgrid(vals, vals[:400], indexing="ij")
    ka, kb = np.meshgrid(k, k[:400], indexing="ij")
    assert np.array_equal(ka > kb, a > b)
    assert np.array_equal(ka <= kb, a <= b)


def test_zero_signs_are_the_only_mismatch():
    assert order_key(0.0) > order_key(-0.0)  # IEEE: equal
    assert not (order_key(-0.0) > order_key(0.0))


def test_host_thresholds_are_never_minus_zero():
    # (t + 1) - n0 and the widened bounds (n - n0) - w, ((n + 1) - n0) + w,
    # as the host forms them, for shift sets up to 3 and offsets and widths
    # on a fine grid including exact integers
    for umax in (1, 2, 3):
        for n0 in np.concatenate([np.linspace(0.0, 1.0, 101), [0.51]]):
            thr = np.array([float(t - umax + 1) - n0 for t in range(2 * umax)])
            assert not np.any(np.signbit(thr) & (thr == 0.0))
            for w in np.linspace(0.0, 1.0, 21):
                for n in range(-umax, umax + 1):
                    lo = (float(n) - n0) - w
                    hi = (float(n + 1) - n0) + w
                    assert not (lo == 0.0 and np.signbit(lo))
                    assert not (hi == 0.0 and np.signbit(hi))


def test_velocity_in_the_absolute_frame_is_never_minus_zero():
    # u = ubar + U with an integer U: -0 + 0 is +0 in round-to-nearest
    for ubar in (-0.0, 0.0):
        for U in range(-3, 4):
            u = ubar + float(U)
            assert not (u == 0.0 and np.signbit(u))

"""Argument and configuration checks of the C ABI that run before any device
work (no GPU needed): every out-of-range field is refused with ALB_EINVAL
(or ALB_EUNSUPPORTED) and a message; empty inputs are accepted."""
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2009_13426_gb300 import build as B
    try:
        B.build()
    except RuntimeError as e:  # no nvcc in this environment
        pytest.skip(str(e))
    from paper_2009_13426_gb300 import alb
    return alb


@pytest.mark.parametrize("field,value", [
    ("nx", 0), ("ny", -3), ("ny", 65536),            # ny is a grid dimension of the launch
    ("u_max", -1), ("u_max", 4),
    ("nu", -1e-3), ("gamma", 1.0), ("n0", 0.0), ("n0", 1.0),
    ("precision", 5), ("bc_x", 3), ("bc_y", -1),
    ("newton_tol", 0.0), ("newton_maxit", 0), ("newton_start", 7),
    ("shift_overlap", -0.1), ("shift_overlap", 1.5), ("shift_rule", 2), ("moments", 6),
    ("prandtl", 0.0), ("prandtl", -0.7), ("prandtl", float("nan")), ("prandtl", float("inf")),
    ("moments", 13),                                  # 13 moments belong to D2Q49
])
def test_configuration_out_of_range_is_refused(lib, field, value):
    cfg = lib.alb_config_default(**{field: value})
    with pytest.raises(lib.AlbError) as ei:
        lib.alb_create(cfg)
    assert ei.value.code == lib.ALB_EINVAL
    assert lib.alb_last_error()


def test_grid_larger_than_the_index_range_is_refused(lib):
    cfg = lib.alb_config_default(nx=65536, ny=32769)  # 2^31 + 2^16 nodes
    with pytest.raises(lib.AlbError) as ei:
        lib.alb_create(cfg)
    assert ei.value.code == lib.ALB_EINVAL


def test_sensor_knots_must_increase(lib):
    cfg = lib.alb_config_default(sensor=1, sensor_eps=(0.1, 0.01, 1.0))
    with pytest.raises(lib.AlbError) as ei:
        lib.alb_create(cfg)
    assert ei.value.code == lib.ALB_EINVAL


def test_stateless_entry_points_accept_empty_and_refuse_negative(lib):
    assert lib.alb_equilibrium(None, None, None, None, 0, 1e-12, 50, None) == lib.ALB_OK
    assert lib.alb_exp_neg(None, 0, None) == lib.ALB_OK
    assert lib.alb_select_shift(None, None, 0, 0.5, 2, None) == lib.ALB_OK
    for call in (lambda: lib.alb_equilibrium(None, None, None, None, -1, 1e-12, 50, None),
                 lambda: lib.alb_exp_neg(None, -1, None),
                 lambda: lib.alb_select_shift(None, None, -1, 0.5, 2, None),
                 lambda: lib.alb_select_shift(None, None, 0, 0.5, 4, None),
                 lambda: lib.alb_equilibrium(None, None, None, None, 0, 0.0, 50, None)):
        with pytest.raises(lib.AlbError) as ei:
            call()
        assert ei.value.code == lib.ALB_EINVAL


def test_batch_and_server_arguments_are_checked(lib):
    with pytest.raises(lib.AlbError) as ei:
        lib.alb_batch_create([], None)
    assert ei.value.code == lib.ALB_EINVAL
    with pytest.raises(lib.AlbError) as ei:
        lib.Server(hbm_fraction=0.0)
    assert ei.value.code == lib.ALB_EINVAL
    with pytest.raises(lib.AlbError) as ei:
        lib.Server(max_chunk=0)
    assert ei.value.code == lib.ALB_EINVAL
    with pytest.raises(lib.AlbError) as ei:
        lib.alb_batch_variants(9)
    assert ei.value.code == lib.ALB_EINVAL
    assert lib.alb_batch_variants(lib.ALB_FP32_FORM)[0] == (128, 4)


@pytest.mark.parametrize("fields,code", [
    (dict(stencil=49), "EINVAL"),                     # D2Q49 needs moments = 13
    (dict(stencil=49, moments=13, precision=1), "EUNSUPPORTED"),
    (dict(stencil=49, moments=13, newton_start=2), "EUNSUPPORTED"),
    (dict(stencil=37), "EUNSUPPORTED"),
])
def test_d2q49_configuration_limits(lib, fields, code):
    cfg = lib.alb_config_default(**fields)
    with pytest.raises(lib.AlbError) as ei:
        lib.alb_create(cfg)
    assert ei.value.code == getattr(lib, "ALB_" + code)

"""The C ABI library loads and exports every symbol include/alb.h declares
(no GPU needed: nothing is called that touches the device)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "alb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(alb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_13426_gb300 import build as B
    try:
        B.build()
    except RuntimeError as e:  # no nvcc in this environment
        pytest.skip(str(e))
    from paper_2009_13426_gb300 import alb
    return alb


def test_header_declares_the_boundary():
    names = declared()
    for must in ("alb_create", "alb_init", "alb_step", "alb_moments", "alb_shifts", "alb_sync",
                 "alb_destroy", "alb_last_error", "alb_equilibrium", "alb_select_shift"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(alb_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    L = lib.lib()
    for n in declared():
        assert hasattr(L, n)


def test_binding_covers_the_header(lib):
    assert set(declared()) <= set(lib.declared_symbols())


def test_host_side_calls_without_gpu(lib):
    cfg = lib.alb_config_default()
    assert cfg.nx == 64 and cfg.stencil == 21 and cfg.newton_tol == 1e-12
    assert cfg.moments == 8 and cfg.prandtl == 1.0 and cfg.stream is None
    x, y = lib.alb_velocities()
    import oracle as O
    ox, oy = O.velocities()
    assert (x == ox).all() and (y == oy).all()
    bad = lib.alb_config_default(stencil=9)
    with pytest.raises(lib.AlbError) as ei:
        lib.alb_create(bad)
    assert ei.value.code == lib.ALB_EUNSUPPORTED
    bad = lib.alb_config_default(nx=0)
    with pytest.raises(lib.AlbError) as ei:
        lib.alb_create(bad)
    assert ei.value.code == lib.ALB_EINVAL
    assert "empty" in lib.alb_last_error()

"""Checkpoint / restart (alb_checkpoint_*) and the state exports
(alb_populations, alb_primitives, alb_next_shifts): continuing from a
restored image must give what continuing the saved flow gives, bit for bit."""
import numpy as np
import pytest

from paper_2009_13426_gb300 import flows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def alb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_13426_gb300 import alb as A
    A.lib()
    return A


def full_state(fl):
    f, g = fl.populations()
    return [f, g] + list(fl.primitives()) + list(fl.shifts()) + list(fl.next_shifts())


@pytest.mark.parametrize("precision", [0, 1])
def test_restore_continues_bit_for_bit(alb, precision):
    nx, ny = 72, 40
    fields = flows.isentropic_vortex(nx, ny, radius=6.0, mach=1.2, seed=3)
    a = alb.Flow(nx, ny, precision=precision, nu=1e-3)
    a.init(*fields)
    a.step(5)
    img = a.checkpoint()
    st5 = a.stats()
    a.step(7)
    ref = full_state(a)
    ref_moments = a.moments()
    # the same handle, rewound
    a.restore(img)
    assert a.stats()["steps"] == st5["steps"]
    a.step(7)
    for x, y in zip(full_state(a), ref):
        assert np.array_equal(x, y)
    # a new flow of the same configuration
    b = alb.Flow(nx, ny, precision=precision, nu=1e-3)
    b.restore(img)
    b.step(7)
    for x, y in zip(b.moments(), ref_moments):
        assert np.array_equal(x, y)
    assert b.stats() == a.stats()
    # another configuration is refused
    c = alb.Flow(nx + 1, ny, precision=precision, nu=1e-3)
    with pytest.raises(alb.AlbError) as ei:
        c.restore(img)
    assert ei.value.code == alb.ALB_EINVAL
    bad = img.copy()
    bad[:8] = 0
    with pytest.raises(alb.AlbError):
        b.restore(bad)


def test_exports_are_consistent(alb):
    """Moments of the exported populations equal alb_moments (collisions
    conserve them); exported primitives give the same conserved fields."""
    nx, ny = 48, 32
    fields = flows.shear_layer(nx, ny=ny, mach=1.5, delta=4.0, seed=2)
    fl = alb.Flow(nx, ny, precision=0, nu=1e-3)
    fl.init(*fields)
    fl.step(3)
    f, g = fl.populations()
    r, ux, uy, T = fl.primitives()
    sx, sy = fl.shifts()
    xi_x, xi_y = alb.alb_velocities()
    cx = xi_x[:, None, None] + sx[None].astype(np.float64)
    cy = xi_y[:, None, None] + sy[None].astype(np.float64)
    rho = f.sum(0)
    jx = (f * cx).sum(0)
    jy = (f * cy).sum(0)
    E2 = (f * (cx ** 2 + cy ** 2) + g).sum(0)
    R, A, B, E = fl.moments()
    # the collision conserves them up to the Newton tolerance (1e-12 relative)
    np.testing.assert_allclose(rho, R, rtol=5e-12)
    np.testing.assert_allclose(jx, A, rtol=5e-12, atol=5e-12)
    np.testing.assert_allclose(jy, B, rtol=5e-12, atol=5e-12)
    np.testing.assert_allclose(0.5 * E2, E, rtol=5e-12)
    np.testing.assert_allclose(r, R, rtol=1e-15)
    np.testing.assert_allclose(r * ux, A, rtol=1e-14, atol=1e-15)
    nsx, nsy = fl.next_shifts()
    assert nsx.min() >= -2 and nsx.max() <= 2 and nsy.min() >= -2 and nsy.max() <= 2


def test_shear_case_saves_and_restores_the_developed_flow(alb, tmp_path, capsys):
    """The profiling case (paper_2009_13426_gb300.shear_case): a checkpoint
    saved after some steps and restored into a new flow continues exactly as
    the flow that kept running (same counters per node over the next steps)."""
    from paper_2009_13426_gb300 import shear_case
    f = str(tmp_path / "case.npy")
    shear_case.main(["--n", "64", "--advance", "30", "--steps", "0", "--save", f])
    capsys.readouterr()
    shear_case.main(["--n", "64", "--load", f, "--steps", "4"])
    restored = capsys.readouterr().out.strip().splitlines()[-1]
    shear_case.main(["--n", "64", "--advance", "30", "--steps", "4"])
    straight = capsys.readouterr().out.strip().splitlines()[-1]
    assert restored == straight

"""Edge cases of fse_step through the C ABI: zero steps, rejected arguments, the
largest and smallest axis lengths, and mixed radix-3/radix-2 shapes."""
import ctypes as ct
import math

import numpy as np
import pytest

import oracle as O
from tolerances import assert_parity, bounds

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _gauss(p):
    X = O.coords(p)
    e = sum(-0.5 * (1.0 + 0.2 * j) * (X[j] - 0.3) ** 2 + 0.3j * X[j] for j in range(p.dim))
    psi = np.exp(e)
    return psi / math.sqrt(O.mass(psi, p))


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_zero_steps_leave_psi_and_launch_nothing(lib):
    d = dict(dim=2, n=(64, 48), lo=(-6.0, -5.0), hi=(6.0, 5.0), s=0.7, omega=0.5, beta=20.0, lam=5.0,
             kernel="coulomb", gamma=(1.0, 1.2), dt=1e-2, prec="f32")
    plan = lib.Plan(d)
    x = plan.to_device(_gauss(O.params(d)))
    before = x.clone()
    n0 = plan.launches
    plan.step(x, 0.0, 0)
    torch.cuda.synchronize()
    assert torch.equal(x, before)
    assert plan.launches == n0


def test_bad_arguments_are_rejected_before_any_launch(lib):
    d = dict(dim=2, n=(32, 32), lo=(-4.0, -4.0), hi=(4.0, 4.0), kernel="none", dt=1e-2, prec="f32")
    plan = lib.Plan(d)
    x = plan.to_device(_gauss(O.params(d)))
    L = lib.load()
    n0 = plan.launches
    assert L.fse_step(plan.handle, ct.c_void_p(x.data_ptr() + 4), ct.c_double(0.0), 1, None) == 1   # misaligned
    assert L.fse_step(plan.handle, ct.c_void_p(x.data_ptr()), ct.c_double(0.0), -1, None) == 1      # nsteps < 0
    assert L.fse_step(plan.handle, None, ct.c_double(0.0), 1, None) == 1                              # null psi
    assert plan.launches == n0


@pytest.mark.parametrize("dim", [2, 3])
def test_element_aligned_psi_matches_aligned_psi(lib, dim):
    """A float32 field 8- but not 16-byte aligned (one element into its buffer)
    takes the element-wise global accesses of the column passes instead of the
    16-byte ones, and pass A leaves out its bulk L2 prefetch (which needs a
    16-byte aligned start); its steps are bit-identical to those of the same
    field 16-byte aligned."""
    if dim == 2:
        d = dict(dim=2, n=(64, 48), lo=(-6.0, -5.0), hi=(6.0, 5.0), s=0.7, omega=0.5, beta=20.0, lam=5.0,
                 kernel="coulomb", gamma=(1.0, 1.2), dt=1e-2, prec="f32")
    else:
        d = dict(dim=3, n=(32, 24, 48), lo=(-5.0, -4.0, -6.0), hi=(5.0, 4.0, 6.0), s=0.7, omega=0.8, beta=50.0,
                 lam=20.0, kernel="ddi3d", dip_n=(1 / math.sqrt(2), 0.0, 1 / math.sqrt(2)),
                 gamma=(1.0, 1.2, 2.0), dt=5e-3, prec="f32")
    plan = lib.Plan(d)
    x = plan.to_device(_gauss(O.params(d)))
    buf = torch.empty(x.numel() + 1, dtype=x.dtype, device=x.device)
    y = buf[1:].view(x.shape)
    y.copy_(x)
    assert x.data_ptr() % 16 == 0 and y.data_ptr() % 16 == 8
    plan.step(x, 0.0, 3)
    plan.step(y, 0.0, 3)
    torch.cuda.synchronize()
    assert torch.equal(x, y)


@pytest.mark.parametrize("n", [(256, 8, 8), (8, 8, 8), (8, 256, 16), (24, 12, 96)])
def test_extreme_axis_lengths_3d_f64(lib, n):
    """Long x lines against the shortest y and z tiles, the smallest grid, and
    radix-3 lengths on every axis, against the oracle."""
    d = dict(dim=3, n=n, lo=(-5.0, -4.0, -6.0), hi=(5.0, 4.0, 6.0), s=0.8, omega=0.6, beta=30.0, lam=10.0,
             kernel="coulomb", gamma=(1.0, 1.3, 0.8), dt=5e-3, prec="f64")
    p = O.params(d)
    psi0 = _gauss(p)
    ref = O.evolve(psi0, p, 0.1, 2)
    plan = lib.Plan(d)
    x = plan.to_device(psi0)
    plan.step(x, 0.1, 2)
    torch.cuda.synchronize()
    assert _rel(x.cpu().numpy(), ref) < 2e-12


@pytest.mark.parametrize("n", [(384, 24), (12, 192)])
def test_mixed_radix_2d_f32(lib, n):
    d = dict(dim=2, n=n, lo=(-6.0, -5.0), hi=(6.0, 5.0), s=0.9, omega=0.4, beta=40.0, lam=8.0,
             kernel="coulomb", gamma=(1.0, 1.1), dt=5e-3, prec="f32")
    p = O.params(d)
    psi0 = _gauss(p)
    ref = O.evolve(psi0, p, 0.0, 3)
    plan = lib.Plan(d)
    x = plan.to_device(psi0)
    plan.step(x, 0.0, 3)
    torch.cuda.synchronize()
    assert_parity(x.cpu().numpy().astype(np.complex128), ref, *bounds("f32", 3), f"mixed radix {n}")

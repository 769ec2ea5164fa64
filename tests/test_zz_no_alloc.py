"""The allocation-free mass entry point (fse_mass_noalloc).

fse_mass_noalloc serves callers that cannot allocate device memory (a hook
between steps inside a framework whose caching allocator owns the device): it
keeps its partial sums in a static device array instead of a workspace. Its
result is checked against the plan-based mass (fse_observables) and against a
float64 sum on the host of the same stored values, on two calls in a row
(the second call reuses the array the first one filled). This file is
collected last so that a failure here leaves every other test run.
"""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CHUNK = 65536          # points summed by one block of the entry point
LIMIT = 4096 * CHUNK   # FSE_NOALLOC_MAX_POINTS


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * 0.1


def _host_mass(x, npoints, cell):
    """float64 sum of |psi|^2 on the host over the first npoints stored values."""
    v = x.reshape(-1)[:npoints].cpu().numpy().astype(np.complex128)
    return cell * float(np.sum(v.real * v.real + v.imag * v.imag))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_mass_matches_observables_on_two_calls(lib, prec):
    d = dict(dim=3, n=(48, 32, 24), lo=(-5.0, -4.0, -3.0), hi=(5.0, 4.0, 3.0), s=0.7, omega=0.5,
             beta=10.0, lam=5.0, dt=1e-3, kernel="ddi3d", dip_n=(0.0, 0.0, 1.0), gamma=(1.0, 1.0, 1.0),
             prec=prec)
    plan = lib.Plan(d)
    cell = float(np.prod([(d["hi"][j] - d["lo"][j]) / d["n"][j] for j in range(3)]))
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((1, 2)):
        x = plan.to_device(_field(tuple(reversed(d["n"])), seed) * (1.0 + call))
        ref = plan.observables(x, 0.0)["mass"]
        lib.fse_mass_noalloc(x, prec, x.numel(), cell, out, stream)
        torch.cuda.synchronize()
        got = float(out.item())
        # all three sum float64 squares of the same stored values; they differ only in summation order
        assert abs(got - ref) <= 1e-12 * abs(ref), (call, got, ref)
        host = _host_mass(x, x.numel(), cell)
        assert abs(got - host) <= 1e-12 * abs(host), (call, got, host)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_mass_several_chunks_ragged_and_empty(lib, prec):
    """3 full chunks of 65536 points plus one point (four partials, the last
    holding a single value), then a prefix of the same buffer, then npoints = 0
    (mass 0): three calls in a row on one array of partials."""
    dt = torch.complex64 if prec == "f32" else torch.complex128
    n = 3 * CHUNK + 1
    x = torch.as_tensor(_field((n,), 7)).to("cuda", dt)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    cell = 0.37
    for npts in (n, CHUNK + 5):
        lib.fse_mass_noalloc(x, prec, npts, cell, out)
        torch.cuda.synchronize()
        ref = _host_mass(x, npts, cell)
        assert abs(float(out.item()) - ref) <= 1e-12 * ref, (npts, float(out.item()), ref)
    lib.fse_mass_noalloc(x, prec, 0, cell, out)
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0


def test_noalloc_rejects_sizes_beyond_the_static_scratch(lib):
    """The C entry point itself (called through ctypes, below the binding's
    tensor checks) refuses counts the static array cannot hold."""
    L = lib.load()
    x = torch.zeros(4, dtype=torch.complex64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    px, po = ct.c_void_p(x.data_ptr()), ct.c_void_p(out.data_ptr())
    assert L.fse_mass_noalloc(px, 0, LIMIT + 1, 1.0, po, None) == 2   # FSE_ERR_UNSUPPORTED
    assert L.fse_mass_noalloc(px, 0, -1, 1.0, po, None) == 1          # FSE_ERR_INVALID
    assert L.fse_mass_noalloc(px, 7, 4, 1.0, po, None) == 1           # unknown precision
    assert L.fse_mass_noalloc(None, 0, 4, 1.0, po, None) == 1          # null field


def test_noalloc_binding_checks_the_tensors(lib):
    x = torch.zeros(4, dtype=torch.complex64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        lib.fse_mass_noalloc(x, "f32", 5, 1.0, out)          # more points than the tensor holds
    with pytest.raises(ValueError):
        lib.fse_mass_noalloc(x, "f64", 4, 1.0, out)          # complex64 data read as float64 pairs
    with pytest.raises(ValueError):
        lib.fse_mass_noalloc(x, "f32", 4, 1.0, out.float())  # float32 result buffer
    with pytest.raises(ValueError):
        lib.fse_mass_noalloc(x.cpu(), "f32", 4, 1.0, out)    # host tensor

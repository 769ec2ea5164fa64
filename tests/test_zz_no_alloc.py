"""The allocation-free mass entry point (fse_mass_noalloc) against the plan-based one.

fse_mass_noalloc serves callers that cannot allocate device memory (a hook
between steps inside a framework whose caching allocator owns the device): it
keeps its partial sums in a static device array instead of a workspace. This
file is collected last so that a failure here leaves every other test run.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * 0.1


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
        # both sum float64 squares of the same stored values; they differ only in summation order
        assert abs(got - ref) <= 1e-12 * abs(ref), (call, got, ref)


def test_noalloc_rejects_sizes_beyond_the_static_scratch(lib):
    x = torch.zeros(4, dtype=torch.complex64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    lim = 4096 * 65536
    with pytest.raises(lib.FseError) as e:
        lib.fse_mass_noalloc(x, "f32", lim + 1, 1.0, out)
    assert e.value.status == 2
    with pytest.raises(lib.FseError):
        lib.fse_mass_noalloc(x, "f32", -1, 1.0, out)

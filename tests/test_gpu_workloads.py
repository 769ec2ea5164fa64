"""Full-size workloads on the GPU: float32 against float64 accuracy over the
workloads' own step counts, mass drift, and reversibility."""
import math

import numpy as np
import pytest

import fse_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _mass(x, d):
    h = np.prod([(d["hi"][j] - d["lo"][j]) / d["n"][j] for j in range(d["dim"])])
    return float((x.abs().double() ** 2).sum()) * h


def test_3d_dipolar_128_float32_vs_float64_1000_steps(lib):
    """128^3 dipolar workload, 1000 steps: float32 within 5e-5 (relative L2) of float64;
    with renormalisation the float32 mass drift stays below 1e-6."""
    d = I.workload("3d_dipolar_128")
    psi0 = I.psi0("3d_dipolar_128")
    nst = d["steps"]
    p64 = lib.Plan(dict(d, prec="f64"))
    x64 = p64.to_device(psi0)
    p64.step(x64, 0.0, nst)
    # sensitivity floor: the same float64 run from the float32-rounded initial state
    x64r = p64.to_device(psi0.astype(np.complex64).astype(np.complex128))
    p64.step(x64r, 0.0, nst)
    p32 = lib.Plan(dict(d, prec="f32"))
    x32 = p32.to_device(psi0)
    m0 = _mass(x32, d)
    p32.step(x32, 0.0, nst)
    p32r = lib.Plan(dict(d, prec="f32", renormalize=1))
    x32r = p32r.to_device(psi0)
    p32r.step(x32r, 0.0, nst)
    torch.cuda.synchronize()
    err = _rel(x32.to(torch.complex128), x64)
    err_r = _rel(x32r.to(torch.complex128), x64)
    floor = _rel(x64r, x64)
    drift = abs(_mass(x32, d) - m0) / m0
    drift_r = abs(_mass(x32r, d) - m0) / m0
    print(f"f32 vs f64 rel L2 {err:.3e} (renorm {err_r:.3e}), floor {floor:.3e}, "
          f"mass drift {drift:.3e} (renorm {drift_r:.3e})")
    assert err < 5e-5 and err_r < 5e-5
    assert drift_r < 1e-6
    assert drift < 2e-5


def test_3d_dipolar_128_float64_matches_oracle_two_steps(lib):
    d = dict(I.workload("3d_dipolar_128"), prec="f64")
    psi0 = I.psi0("3d_dipolar_128")
    p = O.params(d)
    ref = O.evolve(psi0, p, 0.0, 2)
    plan = lib.Plan(d)
    x = plan.to_device(psi0)
    plan.step(x, 0.0, 2)
    got = x.cpu().numpy()
    assert float(np.linalg.norm(got - ref) / np.linalg.norm(ref)) < 2e-12


def test_3d_dipolar_256_float32_vs_float64_1000_steps(lib):
    """The benchmark workload (256^3 dipolar, float32) against the float64 GPU
    path after 1000 steps: relative L2 within 5e-5 (with and without
    renormalisation), every element within 5e-5 of max|psi|, and the
    renormalised float32 mass drift within 1e-6. The float64 path is itself
    held to the oracle per step (test_gpu_full_size.py). Also printed: the
    sensitivity floor, i.e. the float64 run from the float32-rounded initial
    state against the float64 run from the exact one."""
    name = "3d_dipolar_256"
    d = I.workload(name)
    psi0 = I.psi0(name)
    nst = 1000
    p64 = lib.Plan(dict(d, prec="f64"))
    x64 = p64.to_device(psi0)
    p64.step(x64, 0.0, nst)
    x64r = p64.to_device(psi0.astype(np.complex64).astype(np.complex128))
    p64.step(x64r, 0.0, nst)
    p32 = lib.Plan(dict(d, prec="f32"))
    x32 = p32.to_device(psi0)
    m0 = _mass(x32, d)
    p32.step(x32, 0.0, nst)
    p32r = lib.Plan(dict(d, prec="f32", renormalize=1))
    x32r = p32r.to_device(psi0)
    p32r.step(x32r, 0.0, nst)
    torch.cuda.synchronize()
    err = _rel(x32.to(torch.complex128), x64)
    err_r = _rel(x32r.to(torch.complex128), x64)
    floor = _rel(x64r, x64)
    amax = float(x64.abs().max())
    el = float((x32.to(torch.complex128) - x64).abs().max()) / amax
    el_r = float((x32r.to(torch.complex128) - x64).abs().max()) / amax
    drift = abs(_mass(x32, d) - m0) / m0
    drift_r = abs(_mass(x32r, d) - m0) / m0
    print(f"256^3, 1000 steps: f32 vs f64 rel L2 {err:.3e} (renorm {err_r:.3e}), max element {el:.3e} "
          f"(renorm {el_r:.3e}), floor {floor:.3e}, mass drift {drift:.3e} (renorm {drift_r:.3e})")
    assert err < 5e-5 and err_r < 5e-5
    assert el < 5e-5 and el_r < 5e-5
    assert drift_r < 1e-6
    assert drift < 2e-5


def test_3d_dipolar_256_reversible_and_mass_conserving(lib):
    """20 float64 steps forward and 20 back (dt -> -dt) return the initial state;
    float32 mass drift over 20 steps below 1e-6."""
    d = I.workload("3d_dipolar_256")
    psi0 = I.psi0("3d_dipolar_256")
    p32 = lib.Plan(d)
    x = p32.to_device(psi0)
    m0 = _mass(x, d)
    p32.step(x, 0.0, 20)
    p64 = lib.Plan(dict(d, prec="f64"))
    y = p64.to_device(psi0)
    p64.step(y, 0.0, 20)
    torch.cuda.synchronize()
    drift = abs(_mass(x, d) - m0) / m0
    assert drift < 1e-6
    back = lib.Plan(dict(d, prec="f64", dt=-d["dt"]))
    back.step(y, 20 * d["dt"], 20)
    z = p64.to_device(psi0)
    assert _rel(y, z) < 1e-11

"""Batched 2D runs (fse_batch_*): each run bit-identical to the same run advanced alone
with fse_step, and within the float32 tolerance of the FP64 oracle."""
import math

import numpy as np
import pytest

import fse_inputs as I
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _runs(kernel="coulomb"):
    sizes = [16, 24, 32, 16, 48, 24, 32]
    rng = np.random.default_rng(21)
    out = []
    for r, n in enumerate(sizes):
        out.append(dict(dim=2, n=(n, n), lo=(-6.0, -6.0), hi=(6.0, 6.0), s=0.3 + 0.7 * rng.random(),
                        m=0.0, omega=0.95 * rng.random(), beta=50.0 + 450.0 * rng.random(), lam=10.0,
                        dt=1e-3, kernel=kernel, gamma=(1.0, 1.0 + 0.3 * rng.random()), prec="f32"))
    return out


def _psi(d, seed):
    p = O.params(d)
    X = O.coords(p)
    rng = np.random.default_rng(seed)
    e = -0.5 * ((X[0] - rng.uniform(-1, 1)) ** 2 + X[1] ** 2) + 1j * rng.uniform(-0.5, 0.5) * X[0]
    psi = np.exp(e)
    return psi / math.sqrt(O.mass(psi, p))


@pytest.mark.parametrize("kernel", ["coulomb", "none"])
def test_batch_matches_single_runs_bitwise(lib, kernel):
    runs = _runs(kernel)
    psis = [_psi(d, k) for k, d in enumerate(runs)]
    b = lib.Batch(runs)
    xs = b.to_device(psis)
    b.step(xs, 0.2, 5)
    torch.cuda.synchronize()
    for d, p0, x in zip(runs, psis, xs):
        plan = lib.Plan(d)
        y = plan.to_device(p0)
        plan.step(y, 0.2, 5)
        torch.cuda.synchronize()
        assert torch.equal(x, y)


def test_batch_matches_oracle(lib):
    runs = _runs()
    psis = [_psi(d, 10 + k) for k, d in enumerate(runs)]
    b = lib.Batch(runs)
    xs = b.to_device(psis)
    b.step(xs, 0.0, 4)
    torch.cuda.synchronize()
    for d, p0, x in zip(runs, psis, xs):
        ref = O.evolve(p0, O.params(d), 0.0, 4)
        got = x.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 4 * 5e-6


def test_batched_workload_draws(lib):
    """The 256-run workload's parameter draws build a valid batch (sizes 128..512)."""
    runs = I.batched_runs(16)
    b = lib.Batch(runs)
    xs = b.to_device([I.psi0(r) for r in runs])
    b.step(xs, 0.0, 2)
    torch.cuda.synchronize()
    for d, x in zip(runs, xs):
        h = np.prod([(d["hi"][j] - d["lo"][j]) / d["n"][j] for j in range(2)])
        m = float((x.abs().double() ** 2).sum()) * h
        assert abs(m - 1.0) < 1e-5

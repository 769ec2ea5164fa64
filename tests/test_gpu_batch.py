"""Batched 2D runs (fse_batch_*): each run bit-identical to the same run advanced alone
with fse_step, and within the float32 tolerance of the FP64 oracle."""
import math

import numpy as np
import pytest

import fse_inputs as I
import oracle as O
from tolerances import assert_parity, bounds

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
        assert_parity(got, ref, *bounds("f32", 4), f"batch run n={d['n'][0]}")


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


def _one_run_per_size():
    """The first run of each grid size among the batched workload's draws."""
    seen, out = set(), []
    for r in I.batched_runs():
        if r["n"][0] not in seen:
            seen.add(r["n"][0])
            out.append(r)
    return sorted(out, key=lambda r: r["n"][0])


def test_batch_workload_sizes_match_oracle(lib):
    """One run of each workload size (128, 192, 256, 384, 512; radix-3 plans at
    192 and 384) advanced together in one batch for 3 steps: each run within the
    float32 bounds of the FP64 oracle, element by element, and bit-identical to
    the same run advanced alone."""
    runs = _one_run_per_size()
    assert [r["n"][0] for r in runs] == [128, 192, 256, 384, 512]
    psis = [I.psi0(r) for r in runs]
    b = lib.Batch(runs)
    xs = b.to_device(psis)
    b.step(xs, 0.0, 3)
    torch.cuda.synchronize()
    for d, p0, x in zip(runs, psis, xs):
        ref = O.evolve(p0, O.params(d), 0.0, 3)
        got = x.cpu().numpy().astype(np.complex128)
        assert_parity(got, ref, *bounds("f32", 3), f"batched workload run n={d['n'][0]}")
        plan = lib.Plan(d)
        y = plan.to_device(p0)
        plan.step(y, 0.0, 3)
        torch.cuda.synchronize()
        assert torch.equal(x, y)


def test_batch_graph_replay_matches_single_runs(lib):
    """Two calls with the same step count (the second one replays the graph the
    first one captured, with new wave-function pointers and a new start time)
    and a call with another count: each run bit-identical to the same calls of
    fse_step on a plan of its own."""
    runs = _runs()
    psis = [_psi(d, 30 + k) for k, d in enumerate(runs)]
    b = lib.Batch(runs)
    xs = b.to_device(psis)
    dt = runs[0]["dt"]
    b.step(xs, 0.1, 3)
    ys = [x.clone() for x in xs]   # fresh buffers for the replay
    b.step(ys, 0.1 + 3 * dt, 3)
    b.step(ys, 0.1 + 6 * dt, 2)
    torch.cuda.synchronize()
    for d, p0, y in zip(runs, psis, ys):
        plan = lib.Plan(d)
        z = plan.to_device(p0)
        plan.step(z, 0.1, 3)
        plan.step(z, 0.1 + 3 * dt, 3)
        plan.step(z, 0.1 + 6 * dt, 2)
        torch.cuda.synchronize()
        assert torch.equal(y, z)

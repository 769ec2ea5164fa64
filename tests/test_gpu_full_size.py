"""Oracle parity of the kernel instantiations that the 256^3 benchmark times.

The 256^3 dipolar step runs the column passes at length 512 along both
padded axes (F and H along y, G along z: k_colpass<Real, 512, 2/3/5>), the
kinetic passes at length 256 (B, C, D) and the x passes at n_x = 256 (E and
A, whose packed real transforms have length 512); the batched workload's
largest runs take the packed x passes at n_x = 512. Each test below drives one
of those axes at its benchmark length on a grid the oracle finishes in
seconds, in float32 and float64, element by element; then the benchmark
workload itself (256^3, two steps, so that the merged kinetic half step runs)
is compared with the oracle over the whole field.

Paper: Section 4.2, Eqs. tssp1-tssp3 (the step); Section 2, Eqs. FourSeriB3
and tensor (the zero-padded convolution).
"""
import math

import numpy as np
import pytest

import fse_inputs as I
import oracle as O
from tolerances import assert_parity, bounds

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SQ = 1.0 / math.sqrt(2.0)


def _case(n, prec):
    return dict(dim=3, n=n, lo=(-6.0, -5.0, -7.0), hi=(6.0, 5.0, 7.0), s=0.6, m=0.0, omega=0.9, beta=80.0,
                lam=30.0, dt=2e-3, kernel="ddi3d", dip_n=(SQ, 0.0, SQ), gamma=(1.0, 1.2, 2.0), prec=prec)


def _state(d, seed):
    """Displaced Gaussian with a momentum and 5 % seeded complex noise (every
    frequency bin of every pass carries data); unit mass."""
    p = O.params(d)
    X = O.coords(p)
    e = sum(-0.5 * (1.0 + 0.15 * j) * (X[j] - 0.4 + 0.2 * j) ** 2 + 1j * (0.5 - 0.3 * j) * X[j]
            for j in range(p.dim))
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(X[0].shape) + 1j * rng.standard_normal(X[0].shape)
    psi = np.exp(e) * (1.0 + 0.05 * noise)
    return psi / math.sqrt(O.mass(psi, p))


def _gpu(lib, d, psi0, t0, nsteps):
    plan = lib.Plan(d)
    x = plan.to_device(psi0)
    plan.step(x, t0, nsteps)
    torch.cuda.synchronize()
    return x.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("n", [(16, 16, 256), (16, 256, 16), (256, 16, 16), (48, 24, 256), (24, 256, 48),
                               (512, 8, 8)],
                         ids=["z512", "y512", "x256", "z512-ragged", "y512-ragged", "x512"])
def test_benchmark_lengths_match_oracle(lib, n, prec):
    """Length-512 padded transforms along z (pass G) and y (F, H), length-256
    kinetic transforms (B, C, D) and n_x = 256 x passes (E, A); the packed x
    passes at n_x = 512 (16-line tiles of 512 threads) in 3D."""
    d = _case(n, prec)
    p = O.params(d)
    psi0 = _state(d, sum(n))
    ref = O.evolve(psi0, p, 0.1, 2)
    got = _gpu(lib, d, psi0, 0.1, 2)
    rel, elem = bounds(prec, 2)
    assert_parity(got, ref, rel, elem, f"{n} {prec}")


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_2d_x512_partial_tile_matches_oracle(lib, prec):
    """2D at n = (512, 24): 24 lines, so the second 16-line tile of the packed
    n_x = 512 x passes holds 8 lines (the rest of the tile is not read or written)."""
    d = dict(dim=2, n=(512, 24), lo=(-16.0, -6.0), hi=(16.0, 6.0), s=0.7, m=0.0, omega=0.5, beta=60.0,
             lam=10.0, dt=1e-3, kernel="coulomb", gamma=(1.0, 1.5), prec=prec)
    p = O.params(d)
    psi0 = _state(d, 24)
    ref = O.evolve(psi0, p, 0.0, 3)
    got = _gpu(lib, d, psi0, 0.0, 3)
    rel, elem = bounds(prec, 3)
    assert_parity(got, ref, rel, elem, f"2d (512, 24) {prec}")


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_2d_512_matches_oracle(lib, prec):
    """2D at n = 512: padded y transforms of length 1024, x passes at n_x = 512."""
    d = dict(dim=2, n=(512, 512), lo=(-16.0, -16.0), hi=(16.0, 16.0), s=0.8, m=0.0, omega=0.6, beta=100.0,
             lam=10.0, dt=1e-3, kernel="coulomb", gamma=(1.0, 1.0), prec=prec)
    p = O.params(d)
    psi0 = _state(d, 512)
    ref = O.evolve(psi0, p, 0.0, 3)
    got = _gpu(lib, d, psi0, 0.0, 3)
    rel, elem = bounds(prec, 3)
    assert_parity(got, ref, rel, elem, f"2d 512 {prec}")


@pytest.fixture(scope="module")
def dipolar_256_oracle():
    """The FP64 oracle's two steps of the 256^3 benchmark workload (about a
    minute of CPU: the kernel transform, then four 512^3 FFTs per step)."""
    d = I.workload("3d_dipolar_256")
    p = O.params(d)
    psi0 = I.psi0("3d_dipolar_256")
    return d, psi0, O.evolve(psi0, p, 0.0, 2)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_3d_dipolar_256_two_steps_match_oracle(lib, dipolar_256_oracle, prec):
    """The benchmark workload in the benchmark's launch configuration (one
    fse_step call, merged kinetic half steps), every element against the oracle."""
    d, psi0, ref = dipolar_256_oracle
    got = _gpu(lib, dict(d, prec=prec), psi0, 0.0, 2)
    rel, elem = bounds(prec, 2)
    assert_parity(got, ref, rel, elem, f"3d_dipolar_256 {prec}")

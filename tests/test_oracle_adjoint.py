"""Pins of the oracle's adjoint recursion and of the shared input generators (no GPU).

The paper has no adjoint; the oracle's transpose of the real-linearised split
step is checked against central finite differences of the forward oracle.
"""
import math

import numpy as np

import fse_inputs as I
import oracle as O


def _setup(kernel="coulomb", dim=2):
    if dim == 2:
        p = O.Params(dim=2, n=(16, 16), lo=(-6.0, -6.0), hi=(6.0, 6.0), s=0.6, omega=0.7,
                     beta=50.0, lam=10.0, dt=2e-2, kernel=kernel, gamma=(1.0, 1.0))
    else:
        p = O.Params(dim=3, n=(8, 8, 8), lo=(-5.0,) * 3, hi=(5.0,) * 3, s=0.7, omega=0.8,
                     beta=50.0, lam=20.0, dt=2e-2, kernel=kernel, dip_n=(0.6, 0.0, 0.8),
                     gamma=(1.0, 1.2, 2.0))
    X = O.coords(p)
    r2 = sum((X[j] - (0.5 if j == 0 else 0.0)) ** 2 for j in range(dim))
    phi0 = np.exp(-r2 / 2 + 0.3j * X[1]).astype(complex)
    phi0 /= math.sqrt(O.mass(phi0, p))
    tgt = np.exp(-sum((X[j] - 0.3) ** 2 for j in range(dim)) / 2).astype(complex)
    return p, phi0, tgt


def _J(phi0, tgt, p, gam, nst):
    return O.objective_overlap(O.evolve(phi0, p, 0.1, nst, gam), tgt, p)


def test_adjoint_state_gradient_matches_finite_differences():
    p, phi0, tgt = _setup()
    nst = 4
    rng = np.random.default_rng(7)
    gam = 1.0 + 0.1 * rng.standard_normal((nst, 2))
    g, dg = O.gradient_adjoint(phi0, tgt, p, 0.1, nst, gam)
    for _ in range(3):
        d = rng.standard_normal(phi0.shape) + 1j * rng.standard_normal(phi0.shape)
        eps = 1e-6
        fd = (_J(phi0 + eps * d, tgt, p, gam, nst) - _J(phi0 - eps * d, tgt, p, gam, nst)) / (2 * eps)
        an = float(np.sum((np.conj(g) * d).real))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


def test_adjoint_trap_gradient_matches_finite_differences():
    p, phi0, tgt = _setup()
    nst = 4
    rng = np.random.default_rng(8)
    gam = 1.0 + 0.1 * rng.standard_normal((nst, 2))
    _, dg = O.gradient_adjoint(phi0, tgt, p, 0.1, nst, gam)
    for n in range(nst):
        for v in range(2):
            e = np.zeros_like(gam)
            e[n, v] = 1e-6
            fd = (_J(phi0, tgt, p, gam + e, nst) - _J(phi0, tgt, p, gam - e, nst)) / 2e-6
            assert abs(fd - dg[n, v]) < 1e-6 * max(1e-3, abs(dg[n, v])), (n, v, fd, dg[n, v])


def test_adjoint_3d_dipolar_state_gradient():
    p, phi0, tgt = _setup("ddi3d", 3)
    nst = 2
    g, _ = O.gradient_adjoint(phi0, tgt, p, 0.0, nst)
    rng = np.random.default_rng(9)
    d = rng.standard_normal(phi0.shape) + 1j * rng.standard_normal(phi0.shape)
    eps = 1e-6
    fd = (O.objective_overlap(O.evolve(phi0 + eps * d, p, 0.0, nst), tgt, p)
          - O.objective_overlap(O.evolve(phi0 - eps * d, p, 0.0, nst), tgt, p)) / (2 * eps)
    an = float(np.sum((np.conj(g) * d).real))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_splitmix64_reference_stream():
    """SplitMix64 with seed 0: published first output 0xE220A8397B1DCDAF; fast == scalar path."""
    g = I.SplitMix64(0)
    assert int(g.next_u64(1)[0]) == 0xE220A8397B1DCDAF
    a = I.SplitMix64(12345).next_u64(50)
    b = I.SplitMix64(12345).next_u64_fast(50)
    assert np.array_equal(a, b)
    u = I.SplitMix64(1).uniform(200000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 5e-3
    z = I.SplitMix64(2).normal(200000)
    assert abs(z.mean()) < 1e-2 and abs(z.std() - 1) < 1e-2


def test_workload_initial_states_have_unit_mass():
    for name in ("2d_coulomb_128", "adjoint_2d_256"):
        p = I.workload(name)
        assert abs(O.mass(I.psi0(name), p) - 1.0) < 1e-12
    p = I.workload("3d_dipolar_128", n=(32, 32, 32))
    assert abs(O.mass(I.psi0("3d_dipolar_128", n=(32, 32, 32)), p) - 1.0) < 1e-6
    p = I.workload("3d_dipolar_256", n=(48, 48, 48))
    psi = I.psi0("3d_dipolar_256", n=(48, 48, 48))
    assert abs(O.mass(psi, p) - 1.0) < 1e-12
    runs = I.batched_runs(16)
    assert all(r["n"][0] in (128, 192, 256, 384, 512) for r in runs)
    assert all(0.3 <= r["s"] <= 1.0 and 0.0 <= r["omega"] <= 0.95 for r in runs)

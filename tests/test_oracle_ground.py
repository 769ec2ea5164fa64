"""Pins of the oracle's GF-GauSum ground-state solver (Section 3.2), no GPU.

The inner BiCGStab solve is checked against a dense direct solve of the same
preconditioned system; the converged state against the lowest eigenvector of
the dense linear Hamiltonian, the exact harmonic ground state at s = 1, and
(nonlinear cases) the stationary equation H[phi] phi = mu phi it must satisfy.
"""
import math

import numpy as np
import pytest

import oracle as O


def _dense(apply, shape):
    n = int(np.prod(shape))
    M = np.empty((n, n), dtype=complex)
    e = np.zeros(n, dtype=complex)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        M[:, j] = apply(e.reshape(shape)).ravel()
    return M


def _gauss(p, c=(0.3, -0.2)):
    X = O.coords(p)
    return np.exp(-((X[0] - c[0]) ** 2 + 1.2 * (X[1] - c[1]) ** 2) / 2).astype(complex)


def test_bicgstab_solves_the_preconditioned_system():
    """(I + P_Delta A_TF) x = P_Delta phi / dt: BiCGStab against numpy.linalg.solve."""
    p = O.Params(dim=2, n=(8, 6), lo=(-3.0, -2.5), hi=(3.0, 2.5), s=0.7, omega=0.5, beta=30.0, lam=5.0,
                 kernel="coulomb", gamma=(1.0, 1.3), lat_amp=2.0, lat_k=(1.5, 1.0))
    phi = _gauss(p)
    phi /= math.sqrt(O.mass(phi, p))
    dtg = 0.2
    W = O.gf_potential(phi, p)
    b = O.gf_precond(phi / dtg, p, dtg)
    M = _dense(lambda v: O.gf_matvec(v, W, p, dtg), p.shape())
    ref = np.linalg.solve(M, b.ravel()).reshape(p.shape())
    x, it, res = O.bicgstab(lambda v: O.gf_matvec(v, W, p, dtg), b, phi, 1e-14, 200)
    assert res <= 1e-14
    assert np.max(np.abs(x - ref)) < 1e-12 * np.max(np.abs(ref))


def test_linear_ground_state_is_the_lowest_eigenvector():
    """beta = lambda = 0: GF-GauSum converges to the lowest eigenpair of the dense
    H = (-Lap)^s / 2 + V - Omega L_z (harmonic plus lattice, rotating)."""
    p = O.Params(dim=2, n=(16, 16), lo=(-5.0, -5.0), hi=(5.0, 5.0), s=0.85, omega=0.25, kernel="none",
                 gamma=(1.0, 1.2), lat_amp=2.0, lat_k=(math.pi / 2, math.pi / 2))
    H = _dense(lambda v: O.gf_hamiltonian(v, p), p.shape())
    assert np.max(np.abs(H - H.conj().T)) < 1e-12 * np.max(np.abs(H))
    lam, vec = np.linalg.eigh(0.5 * (H + H.conj().T))
    phi, n, inner, change = O.ground_state(_gauss(p), p, 0.5, 3000, tol=1e-12)
    assert change <= 1e-12
    hd = float(np.prod(O.mesh_size(p)))
    u = phi.ravel() * math.sqrt(hd)                       # unit vector in l2
    assert abs(abs(np.vdot(vec[:, 0], u)) - 1.0) < 1e-10
    assert abs(np.vdot(u, H @ u).real - lam[0]) < 1e-10 * abs(lam[0])
    assert lam[1] - lam[0] > 1e-3                         # simple lowest eigenvalue


def test_harmonic_s1_ground_state_is_the_gaussian():
    """s = 1, Omega = 0, gamma = 1, no interaction: phi_g = pi^{-1/2} e^{-r^2/2}, E = 1 (2D)."""
    p = O.Params(dim=2, n=(32, 32), lo=(-8.0, -8.0), hi=(8.0, 8.0), s=1.0, kernel="none", gamma=(1.0, 1.0))
    phi, n, inner, change = O.ground_state(_gauss(p), p, 0.5, 3000, tol=1e-12)
    X = O.coords(p)
    ex = np.exp(-(X[0] ** 2 + X[1] ** 2) / 2) / math.sqrt(math.pi)
    phase = np.vdot(ex, phi) / abs(np.vdot(ex, phi))
    assert np.max(np.abs(phi / phase - ex)) < 1e-9
    assert abs(O.observables(phi, p, 0.0)["energy"] - 1.0) < 1e-9


@pytest.mark.parametrize("s,omega,kernel", [(0.8, 0.0, "coulomb"), (1.0, 0.4, "coulomb")])
def test_nonlinear_ground_state_is_stationary(s, omega, kernel):
    """beta, lambda > 0: the converged state solves H[phi] phi = mu phi (Eq. gf-eq1 at rest)."""
    p = O.Params(dim=2, n=(32, 32), lo=(-7.0, -7.0), hi=(7.0, 7.0), s=s, omega=omega, beta=40.0, lam=8.0,
                 kernel=kernel, gamma=(1.0, 1.0))
    phi, n, inner, change = O.ground_state(_gauss(p), p, 0.2, 4000, tol=1e-10)
    assert change <= 1e-10
    Hphi = O.gf_hamiltonian(phi, p)
    hd = float(np.prod(O.mesh_size(p)))
    mu = hd * np.vdot(phi, Hphi).real
    res = math.sqrt(hd * float(np.sum(np.abs(Hphi - mu * phi) ** 2)))
    assert res < 1e-8 * abs(mu)
    # the energy of the ground state is below that of the starting state
    g0 = _gauss(p) / math.sqrt(O.mass(_gauss(p), p))
    assert O.observables(phi, p, 0.0)["energy"] < O.observables(g0, p, 0.0)["energy"]


def test_shift_kick():
    """Eq. ini_dyn: a grid-multiple shift is np.roll exactly; a fractional shift of a
    Gaussian is the shifted Gaussian; the kick multiplies by exp(i k.x)."""
    p = O.Params(dim=2, n=(32, 24), lo=(-8.0, -6.0), hi=(8.0, 6.0), kernel="none")
    rng = np.random.default_rng(4)
    phi = rng.standard_normal(p.shape()) + 1j * rng.standard_normal(p.shape())
    h = O.mesh_size(p)
    got = O.shift_kick(phi, p, x0=(3 * h[0], -2 * h[1]))
    assert np.max(np.abs(got - np.roll(phi, (-2, 3), axis=(0, 1)))) < 1e-12
    p = O.Params(dim=2, n=(64, 48), lo=(-8.0, -6.0), hi=(8.0, 6.0), kernel="none")   # band-limited Gaussian
    X = O.coords(p)
    g = np.exp(-((X[0] - 0.4) ** 2 + (X[1] + 0.3) ** 2))
    x0 = (0.37, -0.21)
    ex = np.exp(-((X[0] - 0.4 - x0[0]) ** 2 + (X[1] + 0.3 - x0[1]) ** 2))
    assert np.max(np.abs(O.shift_kick(g, p, x0=x0) - ex)) < 1e-12
    k = (0.8, 0.5)
    got = O.shift_kick(g, p, k=k)
    assert np.max(np.abs(got - g * np.exp(1j * (0.8 * X[0] + 0.5 * X[1])))) < 1e-15

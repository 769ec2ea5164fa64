"""Pins of the oracle's kinetic step and whole split step (no GPU).

Each test checks the oracle against something other than itself: the explicit
sum of Eq. tssp1, exact solutions of the free and harmonic problems at s=1,
the centre-of-mass laws (Eqs. classical_CoM and PCoM2), the conservation
laws (Eq. MassEnerg, Lemma on <L_z>) and time reversibility of the symmetric
splitting.
"""
import math

import numpy as np
import pytest

import oracle as O


def _p(**kw):
    base = dict(dim=2, n=(32, 32), lo=(-8.0, -8.0), hi=(8.0, 8.0), s=0.8, omega=0.0,
                beta=0.0, lam=0.0, dt=1e-3, kernel="none", gamma=(0.0, 0.0))
    base.update(kw)
    return O.Params(**base)


@pytest.mark.parametrize("m", [0.0, 0.8])
def test_kinetic_step_is_the_tssp1_sum(m):
    """Eq. tssp1 written as explicit sums over p, q with W_pq(x_l, y_m), mass m of (-Lap + m^2)^s."""
    L, M = 6, 8
    p = _p(n=(L, M), lo=(-1.0, -2.0), hi=(2.0, 1.5), s=0.65, dt=0.37, m=m)
    rng = np.random.default_rng(1)
    phi = rng.standard_normal((M, L)) + 1j * rng.standard_normal((M, L))
    hx = (p.hi[0] - p.lo[0]) / L
    hy = (p.hi[1] - p.lo[1]) / M
    xs = p.lo[0] + hx * np.arange(L)
    ys = p.lo[1] + hy * np.arange(M)
    ps = np.arange(-L // 2, L // 2)
    qs = np.arange(-M // 2, M // 2)
    mux = 2 * np.pi * ps / (p.hi[0] - p.lo[0])
    muy = 2 * np.pi * qs / (p.hi[1] - p.lo[1])
    out = np.zeros((M, L), dtype=complex)
    for a, pp in enumerate(ps):
        for b, qq in enumerate(qs):
            # discrete Fourier coefficient (1/(LM)) sum phi W_pq^*
            Wpq = np.exp(1j * mux[a] * (xs[None, :] - p.lo[0])) * np.exp(1j * muy[b] * (ys[:, None] - p.lo[1]))
            coef = np.sum(phi * np.conj(Wpq)) / (L * M)
            ph = np.exp(-1j * p.dt / 4 * (mux[a] ** 2 + muy[b] ** 2 + p.m ** 2) ** p.s)
            out += ph * coef * Wpq
    got = O.kinetic_step(phi, p, 0.5 * p.dt)
    assert np.max(np.abs(got - out)) < 1e-12


def test_free_gaussian_s1_exact():
    """s=1, V=beta=lambda=0: psi = (1+it)^{-1} pi^{-1/2} exp(-|x|^2/(2(1+it))) (2D)."""
    p = _p(n=(64, 64), lo=(-12.0, -12.0), hi=(12.0, 12.0), s=1.0, dt=0.01)
    X = O.coords(p)
    r2 = X[0] ** 2 + X[1] ** 2
    phi = (np.pi ** -0.5 * np.exp(-r2 / 2)).astype(complex)
    out = O.evolve(phi, p, 0.0, 100)
    ex = (1 + 1j) ** -1 * np.pi ** -0.5 * np.exp(-r2 / (2 * (1 + 1j)))
    assert np.max(np.abs(out - ex)) < 1e-12


def test_free_propagator_any_s_and_omega():
    """V=beta=lambda=0: the split step is exp(-i dt/2 |k|^{2s}) exactly, for any s, Omega."""
    p = _p(n=(16, 12), s=0.55, omega=0.9, dt=0.05, gamma=(0.0, 0.0))
    rng = np.random.default_rng(2)
    phi = rng.standard_normal((12, 16)) + 1j * rng.standard_normal((12, 16))
    # dense DFT matrices, independent of numpy.fft
    def dft(n):
        j = np.arange(n)
        return np.exp(-2j * np.pi * np.outer(j, j) / n)
    Fx, Fy = dft(16), dft(12)
    kx = 2 * np.pi * np.where(np.arange(16) < 8, np.arange(16), np.arange(16) - 16) / 16.0
    ky = 2 * np.pi * np.where(np.arange(12) < 6, np.arange(12), np.arange(12) - 12) / 16.0
    sym = (ky[:, None] ** 2 + kx[None, :] ** 2) ** 0.55
    hat = Fy @ phi @ Fx.T
    ex = np.conj(Fy).T @ (np.exp(-0.5j * p.dt * sym) * hat) @ np.conj(Fx) / (16 * 12)
    got = O.split_step(phi, p, 0.3)
    assert np.max(np.abs(got - ex)) < 1e-12


def _coherent(X, q, pm, t, d):
    """Harmonic coherent state pi^{-d/4} exp(-|x-q|^2/2 + i p.x - i p.q/2 - i d t/2)."""
    e = -0.5 * sum((X[j] - q[j]) ** 2 for j in range(d))
    e = e + 1j * sum(pm[j] * X[j] for j in range(d)) - 0.5j * float(np.dot(pm, q)) - 0.5j * d * t
    return np.pi ** (-d / 4) * np.exp(e)


@pytest.mark.parametrize("omega", [0.0, 0.7])
def test_coherent_state_s1_second_order(omega):
    """s=1 isotropic harmonic trap: exact coherent state; splitting error O(dt^2)."""
    errs = []
    for dt in (0.02, 0.01):
        p = _p(n=(64, 64), lo=(-10.0, -10.0), hi=(10.0, 10.0), s=1.0, omega=omega,
               dt=dt, gamma=(1.0, 1.0))
        X = O.coords(p)
        q0 = np.array([1.5, -0.5])
        phi = _coherent(X, q0, np.zeros(2), 0.0, 2)
        T = 1.0
        out = O.evolve(phi, p, 0.0, int(round(T / dt)))
        q = q0 * math.cos(T)
        pm = -q0 * math.sin(T)
        errs.append(np.max(np.abs(out - _coherent(X, q, pm, T, 2))))
    assert errs[1] < 2e-4
    assert 3.5 < errs[0] / errs[1] < 4.5


def _rk4(f, y, t0, t1, n):
    h = (t1 - t0) / n
    t = t0
    for _ in range(n):
        k1 = f(t, y)
        k2 = f(t + h / 2, y + h / 2 * k1)
        k3 = f(t + h / 2, y + h / 2 * k2)
        k4 = f(t + h, y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        t += h
    return y


def test_classical_com_law_s1_rotating_anisotropic_coulomb():
    """Eq. classical_CoM: x_c'' - 2 Omega J x_c' + (Omega^2 J^2 + Lambda) x_c = 0 (s=1).

    Holds with the Coulomb interaction and the cubic term; the oracle runs in
    the rotating Lagrangian frame, so this pins the frame map x = A(t) x~, the
    time-dependent trap integral and the sign conventions of A and J.
    """
    om, gx, gy = 0.6, 1.0, 1.4
    p = _p(n=(64, 64), lo=(-10.0, -10.0), hi=(10.0, 10.0), s=1.0, omega=om, dt=2e-3,
           gamma=(gx, gy), beta=5.0, lam=3.0, kernel="coulomb")
    X = O.coords(p)
    x0 = np.array([1.0, 0.5])
    phi = (np.pi ** -0.5 * np.exp(-((X[0] - x0[0]) ** 2 + (X[1] - x0[1]) ** 2) / 2)).astype(complex)
    T = 1.0
    nst = int(round(T / p.dt))
    out = O.evolve(phi, p, 0.0, nst)
    xc = O.observables(out, p, T)["xc"]
    J = np.array([[0.0, 1.0], [-1.0, 0.0]])
    Lam = np.diag([gx * gx, gy * gy])
    Mx = om * om * J @ J + Lam

    def f(t, y):
        x, v = y[:2], y[2:]
        return np.concatenate([v, 2 * om * J @ v - Mx @ x])
    # at t=0 the state is real: x~_c' = 0, so x_c' = A'(0) x~_c = Omega J x_c
    y = _rk4(f, np.concatenate([x0, om * J @ x0]), 0.0, T, 2000)
    assert np.max(np.abs(xc - y[:2])) < 2e-5


def test_com_spectral_law_fractional():
    """Eq. PCoM2 (rotating Lagrangian frame, no rotation term) for s=0.6 with a moving packet."""
    p = _p(n=(64, 64), lo=(-10.0, -10.0), hi=(10.0, 10.0), s=0.6, omega=0.4, dt=1e-4,
           gamma=(1.0, 1.3), beta=10.0, lam=2.0, kernel="coulomb")
    X = O.coords(p)
    # a fast, wide packet keeps the spectrum away from the cusp of |k|^{2s} at k = 0,
    # where the discrete commutator [x, |k|^{2s}] departs from its continuum limit
    phi = (np.exp(-((X[0] - 1) ** 2 + X[1] ** 2) / 4.5
                  + 1j * (4.0 * X[0] + 2.5 * X[1]))).astype(complex)
    phi /= math.sqrt(O.mass(phi, p))
    t0 = 0.2
    a = O.evolve(phi, p, t0, 1)
    b = O.evolve(a, p, t0 + p.dt, 1)
    hd = np.prod(O.mesh_size(p))
    xt = lambda f: np.array([hd * np.sum(X[j] * np.abs(f) ** 2) for j in range(2)])
    vel_fd = (xt(b) - xt(phi)) / (2 * p.dt)
    vel = O.com_velocity_spectral(a, p)
    assert np.max(np.abs(vel_fd - vel)) < 1e-6 * max(1.0, np.max(np.abs(vel)))
    # a wrong fractional order would move the packet at a visibly different speed
    wrong = O.com_velocity_spectral(a, O.Params(**dict(vars(p), s=0.62)))
    assert np.max(np.abs(wrong - vel)) > 1e-3


def test_mass_conserved_each_step():
    p = _p(n=(48, 48), s=0.7, omega=0.8, beta=100.0, lam=10.0, kernel="coulomb",
           gamma=(1.0, 1.2), dt=1e-2)
    X = O.coords(p)
    phi = (np.pi ** -0.5 * np.exp(-((X[0] - 1) ** 2 + X[1] ** 2) / 2)).astype(complex)
    m0 = O.mass(phi, p)
    for n in range(5):
        phi = O.split_step(phi, p, n * p.dt)
        assert abs(O.mass(phi, p) - m0) < 1e-13


def test_reversibility():
    """Stepping back with -dt from t_{n+1} returns phi^n (symmetric splitting)."""
    p = O.Params(dim=3, n=(16, 16, 16), lo=(-6.0,) * 3, hi=(6.0,) * 3, s=0.7, omega=0.8,
                 beta=50.0, lam=20.0, dt=5e-3, kernel="ddi3d", dip_n=(0.6, 0.0, 0.8),
                 gamma=(1.0, 1.2, 2.0))
    X = O.coords(p)
    rng = np.random.default_rng(3)
    phi = np.exp(-(X[0] ** 2 + 1.2 * X[1] ** 2 + 2 * X[2] ** 2) / 2) * np.exp(1j * 0.1 * rng.standard_normal(X[0].shape))
    t = 0.4
    fwd = O.split_step(phi, p, t)
    back = O.split_step(fwd, O.Params(**dict(vars(p), dt=-p.dt)), t + p.dt)
    assert np.max(np.abs(back - phi)) < 1e-12


def test_energy_drift_second_order():
    """Eq. MassEnerg: E(T) - E(0) -> 0 like dt^2 for the split step."""
    drift = []
    for dt in (4e-3, 2e-3):
        p = _p(n=(48, 48), lo=(-8.0, -8.0), hi=(8.0, 8.0), s=0.8, omega=0.6, beta=20.0,
               lam=5.0, kernel="coulomb", gamma=(1.0, 1.3), dt=dt)
        X = O.coords(p)
        phi = (np.pi ** -0.5 * np.exp(-((X[0] - 1) ** 2 + X[1] ** 2) / 2)).astype(complex)
        e0 = O.observables(phi, p, 0.0)["energy"]
        T = 0.4
        out = O.evolve(phi, p, 0.0, int(round(T / dt)))
        drift.append(abs(O.observables(out, p, T)["energy"] - e0))
    assert drift[1] < 1e-4
    assert 3.0 < drift[0] / drift[1] < 5.0


def test_angular_momentum_conserved_isotropic_coulomb():
    """Lemma on <L_z>: conserved for an isotropic trap with the Coulomb interaction."""
    # the square grid breaks rotation symmetry at the level of its spectral error
    # (3.8e-6 at n=64, 2.4e-8 at n=96 and n=128 on this machine)
    p = _p(n=(96, 96), lo=(-10.0, -10.0), hi=(10.0, 10.0), s=0.7, omega=0.5, beta=20.0,
           lam=5.0, kernel="coulomb", gamma=(1.0, 1.0), dt=2e-3)
    X = O.coords(p)
    phi = (np.pi ** -0.5 * np.exp(-((X[0] - 1) ** 2 + X[1] ** 2) / 2 + 0.7j * X[1])).astype(complex)
    l0 = O.observables(phi, p, 0.0)["lz"]
    out = O.evolve(phi, p, 0.0, 200)
    l1 = O.observables(out, p, 200 * p.dt)["lz"]
    assert abs(l0) > 0.3
    assert abs(l1 - l0) < 1e-7
    # an anisotropic trap changes it (the law has a non-zero right-hand side)
    q = O.Params(**dict(vars(p), gamma=(1.0, 1.5, 1.0)))
    l2 = O.observables(O.evolve(phi, q, 0.0, 200), q, 200 * p.dt)["lz"]
    assert abs(l2 - l0) > 1e-3


# --- fourth-order composition (triple jump of TS2-GauSum sub-steps) -------------

def test_triple_jump_weights():
    """w1 = 1/(2 - 2^{1/3}), w0 = 1 - 2 w1: the weights sum to one and their cubes cancel."""
    w1, w0 = O.TRIPLE_JUMP_W1, O.TRIPLE_JUMP_W0
    assert abs(2 * w1 + w0 - 1.0) < 1e-15
    assert abs(2 * w1 ** 3 + w0 ** 3) < 1e-14


@pytest.mark.parametrize("omega", [0.0, 0.7])
def test_coherent_state_s1_fourth_order(omega):
    """s=1 isotropic harmonic trap (exact coherent state): order 4 error ratio ~16."""
    errs = []
    for dt in (0.1, 0.05):
        p = _p(n=(64, 64), lo=(-10.0, -10.0), hi=(10.0, 10.0), s=1.0, omega=omega,
               dt=dt, gamma=(1.0, 1.0), order=4)
        X = O.coords(p)
        q0 = np.array([1.5, -0.5])
        phi = _coherent(X, q0, np.zeros(2), 0.0, 2)
        T = 1.0
        out = O.evolve(phi, p, 0.0, int(round(T / dt)))
        q = q0 * math.cos(T)
        pm = -q0 * math.sin(T)
        errs.append(np.max(np.abs(out - _coherent(X, q, pm, T, 2))))
    assert errs[1] < 1e-5
    assert 13.0 < errs[0] / errs[1] < 19.0


def test_fourth_order_nonlinear_convergence():
    """Fractional, rotating, anisotropic trap, cubic and Coulomb terms: errors
    against a fine run shrink ~16x per halving of dt (order 2 shrinks ~4x)."""
    base = dict(n=(32, 32), lo=(-6.0, -6.0), hi=(6.0, 6.0), s=0.8, omega=0.6, beta=20.0, lam=5.0,
                kernel="coulomb", gamma=(1.0, 1.3))
    X = O.coords(_p(**base))
    phi0 = (np.pi ** -0.5 * np.exp(-((X[0] - 0.5) ** 2 + X[1] ** 2) / 2)).astype(complex)
    T = 0.4
    ref = O.evolve(phi0, _p(dt=T / 160, order=4, **base), 0.0, 160)
    e4, e2 = [], []
    for nst in (10, 20):
        e4.append(np.max(np.abs(O.evolve(phi0, _p(dt=T / nst, order=4, **base), 0.0, nst) - ref)))
        e2.append(np.max(np.abs(O.evolve(phi0, _p(dt=T / nst, order=2, **base), 0.0, nst) - ref)))
    assert 12.0 < e4[0] / e4[1] < 20.0
    assert 3.5 < e2[0] / e2[1] < 4.5
    assert e4[1] < e2[1] / 10


def test_fourth_order_reversible_and_free():
    """Symmetric composition: stepping back with -dt restores the state; with
    V = beta = lambda = 0 the step is the exact free propagator."""
    base = dict(n=(24, 16), lo=(-5.0, -4.0), hi=(5.0, 4.0), s=0.7, omega=0.8, beta=30.0, lam=8.0,
                kernel="coulomb", gamma=(1.0, 1.4), order=4)
    X = O.coords(_p(**base))
    phi = (np.exp(-((X[0] - 0.3) ** 2 + 1.3 * X[1] ** 2) / 2 + 0.4j * X[0])).astype(complex)
    fw = O.evolve(phi, _p(dt=0.05, **base), 0.2, 3)
    back = O.evolve(fw, _p(dt=-0.05, **base), 0.35, 3)
    assert np.max(np.abs(back - phi)) < 1e-12 * np.max(np.abs(phi))
    free = dict(base, beta=0.0, lam=0.0, kernel="none", gamma=(0.0, 0.0))
    p = _p(dt=0.07, **free)
    got = O.evolve(phi, p, 0.1, 1)
    ex = np.fft.ifftn(np.exp(-0.5j * p.dt * O.kinetic_symbol(p)) * np.fft.fftn(phi))
    assert np.max(np.abs(got - ex)) < 1e-13


def _naive_fft(x):
    """Recursive mixed-radix decimation-in-time DFT (radix 2 and 3), twiddles
    from math.cos / math.sin, written from the DFT's definition
    X_k = sum_j x_j exp(-2 pi i j k / N)."""
    n = len(x)
    if n == 1:
        return [complex(x[0])]
    r = 2 if n % 2 == 0 else 3
    assert n % r == 0
    m = n // r
    subs = [_naive_fft(x[q::r]) for q in range(r)]
    out = [0j] * n
    for k in range(n):
        acc = 0j
        for q in range(r):
            a = -2.0 * math.pi * q * k / n
            acc += subs[q][k % m] * complex(math.cos(a), math.sin(a))
        out[k] = acc
    return out


@pytest.mark.parametrize("n", [8, 12, 48, 96, 256])
def test_library_fft_matches_naive_recursive_fft(n):
    """The oracle's one library primitive (numpy's FFT, forward unnormalised and
    inverse 1/N, reading 6) against a naive recursive radix-2/3 FFT and, for the
    short lengths, the O(N^2) sum of the DFT's definition."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.array(_naive_fft(list(x)))
    got = np.fft.fft(x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    back = np.fft.ifft(got)
    assert np.max(np.abs(back - x)) <= 1e-13 * np.max(np.abs(x))
    if n <= 48:
        j = np.arange(n)
        dft = np.exp(-2j * np.pi * np.outer(j, j) / n) @ x
        assert np.max(np.abs(got - dft)) <= 1e-12 * np.max(np.abs(dft))

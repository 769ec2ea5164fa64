"""Pins of the oracle's nonlocal solver and per-step integrals (no GPU).

The Gaussian-sum transform C^ is checked against an independent brute-force
evaluation of the cube-truncated kernel transform (polar/spherical
coordinates, no Gaussians), the whole padded convolution against an O(N^2)
direct sum and against closed-form potentials of Gaussian densities (Coulomb
in 2D and 3D, 3D dipolar), the Gaussian-sum fit against 1/r on the fitting
interval (Section 2, Eq. GS-Gene), the near-field integrals against their
closed forms, and the time integrals of trap and dipole axis against
adaptive quadrature.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O


def _edge_nodes(W, nodes=48, panels=6):
    xg, wg = np.polynomial.legendre.leggauss(nodes)
    e = np.linspace(-W, W, panels + 1)
    a, b = e[:-1, None], e[1:, None]
    return (0.5 * (b - a) * xg + 0.5 * (a + b)).ravel(), (0.5 * (b - a) * wg).ravel()


def cref_2d(k, W):
    """int_{[-W,W]^2} e^{-ik.y}/(2 pi |y|) dy = (1/2pi) sum_edges int W sin(k.y)/((k.y)|y|) du."""
    u, wu = _edge_nodes(W)
    tot = 0.0
    for ax in range(2):
        for sg in (-1.0, 1.0):
            y = [None, None]
            y[ax] = sg * W * np.ones_like(u)
            y[1 - ax] = u
            ry = np.hypot(y[0], y[1])
            z = k[0] * y[0] + k[1] * y[1]
            f = np.where(np.abs(z) > 1e-6, np.sin(z) / np.where(z == 0, 1, z), 1 - z * z / 6)
            tot += np.sum(wu * W * f / ry)
    return tot / (2 * math.pi)


def cref_3d(k, W, nodes=32, panels=4):
    """int_{[-W,W]^3} e^{-ik.y}/(4 pi |y|) dy by faces: (1/4pi) sum int int W/|y| [sin z/z + (cos z-1)/z^2]."""
    u, wu = _edge_nodes(W, nodes, panels)
    U, V = np.meshgrid(u, u, indexing="ij")
    WW = np.outer(wu, wu)
    tot = 0.0
    for ax in range(3):
        oth = [a for a in range(3) if a != ax]
        for sg in (-1.0, 1.0):
            y = [None] * 3
            y[ax] = sg * W * np.ones_like(U)
            y[oth[0]], y[oth[1]] = U, V
            ry = np.sqrt(y[0] ** 2 + y[1] ** 2 + y[2] ** 2)
            z = k[0] * y[0] + k[1] * y[1] + k[2] * y[2]
            zz = np.where(np.abs(z) > 1e-3, z, 1.0)
            f = np.where(np.abs(z) > 1e-3, np.sin(zz) / zz + (np.cos(zz) - 1) / zz ** 2,
                         0.5 - z * z / 8 + z ** 4 / 144)
            tot += np.sum(WW * W * f / ry)
    return tot / (4 * math.pi)


def test_gausum_fit_accuracy():
    """U_GS within 1e-14 (relative) of the kernel on [delta, 2 sqrt(d)] (Section 2, Eq. GS-Gene)."""
    for d in (2, 3):
        p = O.Params(dim=d, n=(16,) * d, lo=(-1.0,) * d, hi=(1.0,) * d, kernel="coulomb")
        w, tau = O.gausum_nodes(p)
        r = np.geomspace(p.gs_delta, 2 * math.sqrt(d), 400)
        ugs = np.exp(-np.outer(r * r, tau * tau)) @ w
        u = 1.0 / (2 ** (d - 1) * math.pi * r)
        assert np.max(np.abs(ugs / u - 1)) < 5e-15
        assert 340 <= w.size <= 380


@pytest.mark.parametrize("d", [2, 3])
def test_near_field_integrals_closed_form(d):
    """I0, I2 against closed-form radial integrals of the kernel and each Gaussian (40 digits)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    p = O.Params(dim=d, n=(16,) * d, lo=(-3.0,) * d, hi=(3.0,) * d, kernel="coulomb")
    w, tau = O.gausum_nodes(p)
    I0, I2 = O.near_field(p, w, tau)
    dl = mp.mpf(p.gs_delta) * 3

    def gint(j, t):
        # int_0^dl r^j exp(-t^2 r^2) dr = gamma_inc((j+1)/2, 0, t^2 dl^2) / (2 t^{j+1})
        t = mp.mpf(t)
        return mp.gammainc(mp.mpf(j + 1) / 2, 0, (t * dl) ** 2) / (2 * t ** (j + 1))
    if d == 2:
        e0 = dl - 2 * mp.pi * mp.fsum(mp.mpf(wq) * gint(1, tq) for wq, tq in zip(w, tau))
        e2 = dl ** 3 / 3 - 2 * mp.pi * mp.fsum(mp.mpf(wq) * gint(3, tq) for wq, tq in zip(w, tau))
    else:
        e0 = dl ** 2 / 2 - 4 * mp.pi * mp.fsum(mp.mpf(wq) * gint(2, tq) for wq, tq in zip(w, tau))
        e2 = dl ** 4 / 4 - 4 * mp.pi * mp.fsum(mp.mpf(wq) * gint(4, tq) for wq, tq in zip(w, tau))
    e0, e2 = float(e0), float(e2)
    # the correction is a difference of nearly equal terms: compare against their size
    scale0 = float(dl) if d == 2 else float(dl) ** 2 / 2
    scale2 = float(dl) ** 3 / 3 if d == 2 else float(dl) ** 4 / 4
    assert abs(I0 - e0) < 1e-13 * scale0
    assert abs(I2 - e2) < 1e-13 * scale2


def test_gausum_2d_matches_bruteforce_transform():
    p = O.Params(dim=2, n=(16, 16), lo=(-2.0, -2.0), hi=(2.0, 2.0), kernel="coulomb")
    oc = O.gausum_octant(p)
    W = 4.0
    dk = 2 * math.pi / (2 * W)
    for px, py in [(0, 0), (1, 0), (0, 3), (2, 5), (7, 7), (16, 0), (16, 16), (11, 4)]:
        ref = cref_2d((px * dk, py * dk), W)
        assert abs(oc[py, px] - ref) < 1e-13 * max(1.0, abs(ref)), (px, py)


def test_gausum_3d_matches_bruteforce_transform():
    p = O.Params(dim=3, n=(8, 8, 8), lo=(-1.0,) * 3, hi=(1.0,) * 3, kernel="coulomb")
    oc = O.gausum_octant(p)
    W = 2.0
    dk = 2 * math.pi / (2 * W)
    for pp in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (3, 2, 1), (8, 8, 8), (8, 0, 3), (5, 7, 2)]:
        ref = cref_3d([v * dk for v in pp], W)
        assert abs(oc[pp[2], pp[1], pp[0]] - ref) < 2e-13 * max(1.0, abs(ref)), pp


def test_padded_convolution_matches_direct_sum():
    """nonlocal_potential == direct O(N^2) evaluation of sum_k rho^_k C_ref(k) e^{ik.x}/N."""
    p = O.Params(dim=2, n=(8, 6), lo=(-1.0, -1.5), hi=(1.0, 1.5), kernel="coulomb")
    rng = np.random.default_rng(5)
    rho = rng.random((6, 8))
    nx, ny = 16, 12
    Wx, Wy = 2 * 2.0, 2 * 3.0     # padded periods
    # direct DFT of the zero-padded density
    xs = np.arange(nx)
    ys = np.arange(ny)
    pxs = np.where(xs < nx // 2, xs, xs - nx)
    pys = np.where(ys < ny // 2, ys, ys - ny)
    out = np.zeros((6, 8))
    coef = {}
    for a in pxs:
        for b in pys:
            c = 0j
            for j in range(6):
                for i in range(8):
                    c += rho[j, i] * np.exp(-2j * math.pi * (a * i / nx + b * j / ny))
            coef[(a, b)] = c
    # brute-force truncated transform on the rectangle [-2,2]x[-3,3]
    def cref_rect(kx, ky):
        # polar: integrate in r analytically per angle, over the rectangle's boundary
        def g(th):
            c, s = math.cos(th), math.sin(th)
            R = min(2.0 / abs(c) if abs(c) > 1e-300 else 1e300, 3.0 / abs(s) if abs(s) > 1e-300 else 1e300)
            al = kx * c + ky * s
            return R if abs(al) < 1e-14 else math.sin(al * R) / al
        ths = [math.atan2(3, 2), math.pi - math.atan2(3, 2), math.pi + math.atan2(3, 2), 2 * math.pi - math.atan2(3, 2)]
        brk = [0.0] + ths + [2 * math.pi]
        tot = sum(integrate.quad(g, brk[i], brk[i + 1], epsabs=1e-15, epsrel=1e-14, limit=200)[0]
                  for i in range(len(brk) - 1))
        return tot / (2 * math.pi)
    C = {}
    for a in pxs:
        for b in pys:
            key = (abs(a), abs(b))
            if key not in C:
                C[key] = cref_rect(2 * math.pi * a / Wx, 2 * math.pi * b / Wy)
    for j in range(6):
        for i in range(8):
            v = 0j
            for a in pxs:
                for b in pys:
                    v += coef[(a, b)] * C[(abs(a), abs(b))] * np.exp(2j * math.pi * (a * i / nx + b * j / ny))
            out[j, i] = (v / (nx * ny)).real
    got = O.nonlocal_potential(rho, p, O.gausum_multiplier(p))
    assert np.max(np.abs(got - out)) < 1e-12 * np.max(np.abs(out))


def test_coulomb_2d_gaussian_closed_form():
    """U=1/(2 pi|x|), rho=e^{-r^2}/pi: Phi = e^{-r^2/2} I0(r^2/2)/(2 sqrt(pi))."""
    p = O.Params(dim=2, n=(64, 64), lo=(-8.0, -8.0), hi=(8.0, 8.0), kernel="coulomb")
    X = O.coords(p)
    r2 = X[0] ** 2 + X[1] ** 2
    Phi = O.nonlocal_potential(np.exp(-r2) / math.pi, p, O.gausum_multiplier(p))
    ex = special.i0e(r2 / 2) / (2 * math.sqrt(math.pi))
    assert abs(Phi[32, 32] - 0.28209479177387814) < 1e-14
    assert np.max(np.abs(Phi - ex)) < 1e-13


def test_coulomb_3d_gaussian_closed_form():
    """U=1/(4 pi|x|), rho=pi^{-3/2} e^{-r^2}: Phi = erf(r)/(4 pi r)."""
    p = O.Params(dim=3, n=(48, 48, 48), lo=(-6.0,) * 3, hi=(6.0,) * 3, kernel="coulomb")
    X = O.coords(p)
    r = np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2)
    Phi = O.nonlocal_potential(math.pi ** -1.5 * np.exp(-r * r), p, O.gausum_multiplier(p))
    rr = np.where(r > 0, r, 1.0)
    ex = np.where(r > 0, special.erf(rr) / (4 * math.pi * rr), 1 / (2 * math.pi ** 1.5))
    assert np.max(np.abs(Phi - ex)) < 1e-13


def test_ddi_3d_gaussian_closed_form():
    """3D DDI: Phi = -rho - 3 d_nn f, f = erf(r)/(4 pi r) (Eq. Kernel, Fourier form)."""
    nvec = np.array([0.6, 0.0, 0.8])
    p = O.Params(dim=3, n=(48, 48, 48), lo=(-6.0,) * 3, hi=(6.0,) * 3, kernel="ddi3d",
                 dip_n=tuple(nvec), omega=0.0)
    X = O.coords(p)
    r = np.sqrt(X[0] ** 2 + X[1] ** 2 + X[2] ** 2)
    rho = math.pi ** -1.5 * np.exp(-r * r)
    Phi = O.nonlocal_potential(rho, p, O.kernel_multiplier_instant(p, 0.0))
    m = r > 0.3
    rr = r[m]
    c = (nvec[0] * X[0][m] + nvec[1] * X[1][m] + nvec[2] * X[2][m]) / rr
    e = np.exp(-rr * rr)
    erf = special.erf(rr)
    sp = 2 / math.sqrt(math.pi)
    g1 = sp * e / rr - erf / rr ** 2                     # (erf r / r)'
    g2 = -2 * sp * e - 2 * sp * e / rr ** 2 + 2 * erf / rr ** 3   # (erf r / r)''
    dnn = (g2 * c * c + g1 / rr * (1 - c * c)) / (4 * math.pi)
    ex = -rho[m] - 3 * dnn
    assert np.max(np.abs(Phi[m] - ex)) < 1e-12
    # isotropic density: Phi(0) = 0 for any axis
    assert abs(Phi[24, 24, 24]) < 1e-12


def test_trap_integral_quadrature():
    p = O.Params(dim=3, n=(4, 4, 4), lo=(-3.0,) * 3, hi=(3.0,) * 3, omega=0.9, gamma=(1.0, 1.2, 2.0))
    ta, tb = 0.37, 0.37 + 0.05
    P = O.trap_integral(p, ta, tb)
    X = O.coords(p)
    for idx in [(0, 0, 0), (1, 2, 3), (3, 3, 1)]:
        x = np.array([X[j][idx] for j in range(3)])
        f = lambda t: 0.5 * sum(p.gamma[v] ** 2 * (O.rotation(p.omega, t, 3) @ x)[v] ** 2 for v in range(3))
        ref = integrate.quad(f, ta, tb, epsabs=1e-17, epsrel=1e-14)[0]
        assert abs(P[idx] - ref) < 1e-14 * max(1, abs(ref))
    iso = O.Params(**dict(vars(p), gamma=(1.3, 1.3, 0.7)))
    V = sum(0.5 * g * g * x * x for g, x in zip(iso.gamma, X))
    assert np.max(np.abs(O.trap_integral(iso, ta, tb) - (tb - ta) * V)) < 1e-14


def test_dipole_integral_quadrature():
    p = O.Params(dim=3, n=(4, 4, 4), lo=(-1.0,) * 3, hi=(1.0,) * 3, omega=0.8,
                 dip_n=(1 / math.sqrt(2), 0.0, 1 / math.sqrt(2)), kernel="ddi3d")
    ta, tb = 1.3, 1.3 + 0.2
    M = O.dipole_integral(p, ta, tb)
    for i in range(3):
        for j in range(3):
            ref = integrate.quad(lambda t: O.dipole_axis(p, t)[i] * O.dipole_axis(p, t)[j], ta, tb,
                                 epsabs=1e-16, epsrel=1e-14)[0]
            assert abs(M[i, j] - ref) < 1e-15
    assert abs(np.trace(M) - (tb - ta)) < 1e-15
    # m(t) = A(t)^{-1} n rotates the in-plane part backwards
    m = O.dipole_axis(p, math.pi / (2 * p.omega))
    assert np.allclose(m, [0.0, 1 / math.sqrt(2), 1 / math.sqrt(2)], atol=1e-15)


# --- Coulomb-type kernels 1/|x|^mu, 0 < mu <= d - 1 (Eq. Kernel) --------------------

MU_CASES = [(2, 0.5), (2, 1.0), (3, 0.5), (3, 1.5), (3, 2.0)]


@pytest.mark.parametrize("d,mu", MU_CASES)
def test_gausum_fit_accuracy_mu(d, mu):
    """U_GS within 1e-13 (relative) of 1/(2^{d-1} pi r^mu) on [delta, 2 sqrt(d)] (Eq. GS-Gene)."""
    p = O.Params(dim=d, n=(16,) * d, lo=(-1.0,) * d, hi=(1.0,) * d, kernel="coulomb", mu=mu)
    w, tau = O.gausum_nodes(p)
    r = np.geomspace(p.gs_delta, 2 * math.sqrt(d), 400)
    ugs = np.exp(-np.outer(r * r, tau * tau)) @ w
    u = 1.0 / (2 ** (d - 1) * math.pi * r ** mu)
    assert np.max(np.abs(ugs / u - 1)) < 1e-13


@pytest.mark.parametrize("d,mu", MU_CASES)
def test_near_field_integrals_closed_form_mu(d, mu):
    """I0, I2 for 1/|x|^mu against exact radial integrals (incomplete gamma, 40 digits)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    p = O.Params(dim=d, n=(16,) * d, lo=(-3.0,) * d, hi=(3.0,) * d, kernel="coulomb", mu=mu)
    w, tau = O.gausum_nodes(p)
    I0, I2 = O.near_field(p, w, tau)
    dl = mp.mpf(p.gs_delta) * 3
    S = 2 * mp.pi if d == 2 else 4 * mp.pi
    pref = 1 / (2 ** (d - 1) * mp.pi)
    m = mp.mpf(mu)

    def gint(j, t):
        t = mp.mpf(t)
        return mp.gammainc(mp.mpf(j + 1) / 2, 0, (t * dl) ** 2) / (2 * t ** (j + 1))
    u0 = pref * S * dl ** (d - m) / (d - m)
    u2 = pref * S * dl ** (d + 2 - m) / (d + 2 - m)
    e0 = u0 - S * mp.fsum(mp.mpf(wq) * gint(d - 1, tq) for wq, tq in zip(w, tau))
    e2 = u2 - S * mp.fsum(mp.mpf(wq) * gint(d + 1, tq) for wq, tq in zip(w, tau))
    assert abs(I0 - float(e0)) < 1e-12 * float(u0)
    assert abs(I2 - float(e2)) < 1e-12 * float(u2)


@pytest.mark.parametrize("d,mu,n,L", [(2, 0.5, 64, 8.0), (3, 1.5, 48, 6.0), (3, 0.5, 48, 6.0)])
def test_riesz_potential_of_gaussian_closed_form(d, mu, n, L):
    """rho = pi^{-d/2} e^{-r^2}: int rho(y)/|x-y|^mu dy = Gamma((d-mu)/2)/Gamma(d/2) 1F1(mu/2; d/2; -r^2).

    At mu = 1 this is erf(r)/r (3D) and sqrt(pi) e^{-r^2/2} I0(r^2/2) (2D),
    the two Coulomb closed forms above."""
    p = O.Params(dim=d, n=(n,) * d, lo=(-L,) * d, hi=(L,) * d, kernel="coulomb", mu=mu)
    X = O.coords(p)
    r2 = sum(X[j] ** 2 for j in range(d))
    rho = math.pi ** (-d / 2) * np.exp(-r2)
    Phi = O.nonlocal_potential(rho, p, O.gausum_multiplier(p))
    ex = (special.gamma((d - mu) / 2) / special.gamma(d / 2) * special.hyp1f1(mu / 2, d / 2, -r2)
          / (2 ** (d - 1) * math.pi))
    assert np.max(np.abs(Phi - ex)) < 1e-12 * np.max(np.abs(ex))


def test_kernel_exponent_range():
    """Eq. Kernel: 0 < mu <= d - 1 for the Coulomb type; the dipolar kernel uses mu = 1."""
    base = dict(n=(8, 8), lo=(-1.0, -1.0), hi=(1.0, 1.0), kernel="coulomb")
    for bad in (0.0, 1.5, -1.0):
        with pytest.raises(ValueError):
            O.Params(dim=2, mu=bad, **base)
    assert O.Params(dim=2, mu=1.0, **base).gs_tmin == -36.0
    assert O.Params(dim=2, mu=0.5, **base).gs_tmin == -72.0
    with pytest.raises(ValueError):
        O.Params(dim=3, n=(8,) * 3, lo=(-1.0,) * 3, hi=(1.0,) * 3, kernel="ddi3d", mu=0.5)


def test_ddi_2d_gaussian_closed_form():
    """2D DDI (Eq. Kernel): Phi = -3/2 (d_{n_perp n_perp} - n_3^2 Lap) f with
    f = (1/(2 pi|x|)) * rho = e^{-r^2/2} I0(r^2/2) / (2 sqrt(pi)) for rho = e^{-r^2}/pi."""
    nvec = np.array([0.48, -0.36, 0.8])
    p = O.Params(dim=2, n=(64, 64), lo=(-8.0, -8.0), hi=(8.0, 8.0), kernel="ddi2d", dip_n=tuple(nvec))
    X = O.coords(p)
    r2 = X[0] ** 2 + X[1] ** 2
    rho = np.exp(-r2) / math.pi
    Phi = O.nonlocal_potential(rho, p, O.kernel_multiplier_instant(p, 0.0))
    u = r2 / 2
    r = np.sqrt(r2)
    c = 1.0 / (2 * math.sqrt(math.pi))
    g1 = special.i1e(u) - special.i0e(u)                                  # G'(u), G = e^{-u} I0(u)
    i1_over_u = np.where(u > 1e-12, special.i1e(u) / np.where(u > 0, u, 1.0), 0.5)
    g2 = 2 * special.i0e(u) - 2 * special.i1e(u) - i1_over_u              # G''(u)
    f1_over_r = c * g1                                                    # f'(r)/r
    f2 = c * (g2 * r2 + g1)                                               # f''(r)
    npp = nvec[:2]
    nx = np.where(r > 0, (npp[0] * X[0] + npp[1] * X[1]) / np.where(r > 0, r, 1.0), 0.0)
    dnn = nx ** 2 * f2 + (npp @ npp - nx ** 2) * f1_over_r                # d_{n_perp n_perp} f
    lap = f2 + f1_over_r
    ex = -1.5 * (dnn - nvec[2] ** 2 * lap)
    assert np.max(np.abs(Phi - ex)) < 1e-12 * np.max(np.abs(ex))


def test_ddi_2d_integrated_kernel_matches_instant_quadrature():
    """K^ over [ta, tb] is the time integral of the instantaneous multiplier (Eq. Kernel_Rot)."""
    p = O.Params(dim=2, n=(8, 8), lo=(-2.0, -2.0), hi=(2.0, 2.0), kernel="ddi2d", omega=1.3,
                 dip_n=(0.6, 0.0, 0.8))
    C = O.gausum_multiplier(p)
    ta, tb = 0.2, 0.9
    got = O.kernel_multiplier(p, ta, tb, C)
    tq, wq = np.polynomial.legendre.leggauss(24)
    t = 0.5 * (tb - ta) * tq + 0.5 * (ta + tb)
    ref = sum(0.5 * (tb - ta) * w * O.kernel_multiplier_instant(p, tt, C) for tt, w in zip(t, wq))
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_lattice_trap_integral_quadrature():
    """Harmonic plus optical lattice V = sum_v (gamma_v^2 x_v^2/2 + A sin^2(k_v x_v)) in the
    rotating frame: P = int V(A(tau) x~) dtau against adaptive quadrature (Section 4.2,
    quadrature for a general V); Omega = 0 gives dt V; the Section 3.3 example's V."""
    p = O.Params(dim=3, n=(6, 6, 4), lo=(-3.0,) * 3, hi=(3.0,) * 3, omega=1.1, gamma=(1.0, 1.2, 2.0),
                 lat_amp=10.0, lat_k=(math.pi, 0.8 * math.pi, 0.5 * math.pi))
    ta, tb = 0.21, 0.21 + 0.07
    P = O.trap_integral(p, ta, tb)
    X = O.coords(p)
    for idx in [(0, 0, 0), (1, 2, 3), (3, 5, 1), (2, 4, 5)]:
        x = np.array([X[j][idx] for j in range(3)])

        def f(t):
            y = O.rotation(p.omega, t, 3) @ x
            return sum(0.5 * p.gamma[v] ** 2 * y[v] ** 2 + p.lat_amp * math.sin(p.lat_k[v] * y[v]) ** 2
                       for v in range(3))
        ref = integrate.quad(f, ta, tb, epsabs=1e-17, epsrel=1e-14)[0]
        assert abs(P[idx] - ref) < 1e-14 * max(1, abs(ref))
    still = O.Params(dim=2, n=(8, 8), lo=(-2.0, -2.0), hi=(2.0, 2.0), omega=0.0, gamma=(1.0, 1.0),
                     lat_amp=10.0, lat_k=(math.pi, math.pi))
    X = O.coords(still)
    V = (X[0] ** 2 + X[1] ** 2) / 2 + 10 * (np.sin(math.pi * X[0]) ** 2 + np.sin(math.pi * X[1]) ** 2)
    assert np.max(np.abs(O.trap_potential(still, 0.0) - V)) < 1e-13
    assert np.max(np.abs(O.trap_integral(still, 0.3, 0.35) - 0.05 * V)) < 1e-13

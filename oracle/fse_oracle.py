"""FP64 CPU oracle of the TS2-GauSum split step -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use this module; the CUDA library never calls it and shares
no code with it.

What it computes, in the paper's order (Antoine, Tang & Zhang, arXiv
1512.03210, Section 4.2 "Numerical method"):

* the rotating Lagrangian frame (Eqs. Amatrix, transform, FSE1_Rot,
  Kernel_Rot): the unknown is phi(x~, t) = psi(A(t) x~, t) on the box B;
* the Strang split step TS2-GauSum (Eqs. tssp1-tssp3): a kinetic half step
  exp(-i dt/4 (|k|^2+m^2)^s) in Fourier space (Eq. 1step), the exactly
  integrated potential step (Eqs. 2stepA/B, solu_step2, solu_step2_conv,
  int_poten), and a second kinetic half step;
* the nonlocal term by the Gaussian-sum method (Section 2, Eqs. key_form00,
  GS-Gene, FourSeriB3, tensor, taylor) with the DDI rewritten as Coulomb
  acting on a differentiated density (Section 2, end);
* the observables of Section 1 and 4.1 (Eqs. mass, energy, AME, CoM,
  ConWidth) and the spectral centre-of-mass law (Eq. PCoM2, Appendix B);
* the GF-GauSum ground-state iteration of Section 3.2 (backward-Euler
  gradient flow with discrete normalisation, BiCGStab on the system
  preconditioned by P_Delta, Eq. precond_type1).

Readings where the paper is silent or ambiguous (each pinned by a test):

1. Eq. tssp2 prints |phi^n|^2; the potential sub-step conserves the density
   of its own input, so rho = |phi^(1)|^2 (the output of the first kinetic
   half step) is used, for rho and for the nonlocal density.
2. The density is zero-padded by a factor 2 per axis (period 2W for a box of
   width W) instead of to B3 (factor 3): for x, y in B, x - y lies in one
   period, so the cube-truncated kernel never aliases.
3. The Gaussian-sum fit (sinc quadrature, deferred by the paper to its
   reference on GauSum) uses step h_s, t in [t_min, ln(7/delta)], in units
   where the box is [-1,1]^d; it is fitted on [delta, 2 sqrt(d)] (the cube
   corners) rather than [delta, 2].
4. The printed 3D DDI reformulation drops a factor -3; the Fourier form
   -1 + 3 (n.k)^2/|k|^2 of Eq. Kernel is followed.
5. Odd spectral factors (k_j in cross terms, derivatives) vanish at the
   Nyquist index; forward DFT unnormalised, inverse 1/N.
6. The grid is n points per axis, x_l = lo + l h, l = 0..n-1 (the printed
   index set duplicates the periodic endpoint). m = 0 unless given.
7. Coulomb-type kernels 1/|x|^mu, 0 < mu <= d - 1 (Eq. Kernel): the same
   sinc quadrature with exponent mu, lower end t_min = -36/mu by default.
8. Order 4 (``order=4``): the symmetric triple jump of three TS2-GauSum
   sub-steps, the higher-order extension that Section 4.2 mentions.
9. 2D DDI (``kernel="ddi2d"``): Eq. Kernel_Rot prints only
   -3/2 L~_2 (1/(2 pi|x|)); the rotation-invariant term -3/2 (-n_3^2 Lap) of
   Eq. Kernel and of the Section 2 reformulation is kept, integrated over the
   window: K^ = 3/2 (k^T M_perp k - n_3^2 (tb-ta) |k|^2) C^.
10. A general V (Section 4.2: P by numerical quadrature): the harmonic trap
   plus an optical lattice lat_amp sum_v sin^2(lat_k_v x_v) in the lab frame,
   the potential of the harmonic-plus-lattice example of Section 3.3.
11. Eq. ini_dyn shifts a ground state by x0 off the grid: the translation is
   spectral, and the Nyquist mode of each axis takes cos(k_N x0_j).

The time-integrated trap P (Eq. int_poten) and dipole matrix
M = int m m^T dtau (Eq. Kernel_Rot / solu_step2_conv) are computed here by
Gauss-Legendre quadrature of their definitions, not by closed forms.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "Params", "params", "mesh_size", "coords", "wavenumbers", "kinetic_symbol",
    "kinetic_step", "rotation", "trap_potential", "trap_integral", "dipole_axis",
    "dipole_integral", "gausum_nodes", "gausum_g_table", "near_field",
    "gausum_octant", "gausum_multiplier", "kernel_multiplier", "kernel_multiplier_instant",
    "split_step4", "TRIPLE_JUMP_W1", "TRIPLE_JUMP_W0",
    "pad", "crop", "nonlocal_potential", "potential_step", "split_step", "evolve",
    "observables", "com_velocity_spectral", "mass",
    "adjoint_split_step", "evolve_with_states", "objective_overlap", "gradient_adjoint",
    "gf_lz", "gf_potential", "gf_precond", "gf_matvec", "bicgstab", "gf_step", "ground_state",
    "gf_hamiltonian", "shift_kick",
]


class Params:
    """Plain parameter record (the fields of Eq. SFSE, Eq. Kernel, Eq. harm_poten)."""

    FIELDS = dict(dim=2, n=None, lo=None, hi=None, s=1.0, m=0.0, omega=0.0, beta=0.0,
                  lam=0.0, dt=1e-3, kernel="coulomb", mu=1.0, dip_n=(0.0, 0.0, 1.0),
                  gamma=(1.0, 1.0, 1.0), gs_delta=1e-3, gs_h=0.125, gs_tmin=None, order=2,
                  lat_amp=0.0, lat_k=(0.0, 0.0, 0.0))

    def __init__(self, **kw):
        for k, v in self.FIELDS.items():
            setattr(self, k, kw.get(k, v))
        self.n = tuple(int(v) for v in self.n)
        self.lo = tuple(float(v) for v in self.lo)
        self.hi = tuple(float(v) for v in self.hi)
        g = tuple(float(v) for v in self.gamma)
        self.gamma = g + (1.0,) * (3 - len(g))
        lk = tuple(float(v) for v in self.lat_k)
        self.lat_k = lk + (0.0,) * (3 - len(lk))
        if self.kernel == "ddi3d" and self.dim != 3:
            raise ValueError("the 3D dipolar kernel needs dim=3")
        if self.kernel == "ddi3d" and self.mu != 1.0:
            raise ValueError("the 3D dipolar kernel is built on 1/|x| (mu = 1)")
        if self.kernel == "ddi2d" and (self.dim != 2 or self.mu != 1.0):
            raise ValueError("the 2D dipolar kernel needs dim=2 and is built on 1/(2 pi |x|)")
        if self.kernel == "coulomb" and not (0.0 < self.mu <= self.dim - 1):
            raise ValueError("Coulomb-type kernel 1/|x|^mu needs 0 < mu <= d - 1 (Eq. Kernel)")
        if self.order not in (2, 4):
            raise ValueError("splitting order 2 (Strang, Eqs. tssp1-tssp3) or 4 (triple jump)")
        if not self.gs_tmin:
            # lower end of the sinc quadrature: the dropped tail is ~ e^{mu t_min} / mu
            self.gs_tmin = -36.0 / self.mu

    def shape(self):
        """Array shape, x fastest: (ny, nx) or (nz, ny, nx)."""
        return tuple(reversed(self.n))


def params(p) -> Params:
    if isinstance(p, Params):
        return p
    return Params(**{k: v for k, v in dict(p).items() if k in Params.FIELDS})


def mesh_size(p):
    p = params(p)
    return [(p.hi[j] - p.lo[j]) / p.n[j] for j in range(p.dim)]


def coords(p):
    """Grid coordinates x~_l = lo + l h (reading 6) as arrays of the field's shape.

    Returns [X, Y] or [X, Y, Z] (vector index order x, y, z).
    """
    p = params(p)
    h = mesh_size(p)
    ax = [p.lo[j] + h[j] * np.arange(p.n[j]) for j in range(p.dim)]
    grids = np.meshgrid(*reversed(ax), indexing="ij")     # [z][y][x] order
    return list(reversed(grids))


def _index(n):
    """Signed integer mode numbers p in numpy FFT order: 0..n/2-1, -n/2..-1 (n even)."""
    i = np.arange(n)
    return np.where(i < n // 2, i, i - n)


def _freq(n, width):
    """Signed wavenumbers 2 pi p / width, p in numpy FFT order (Section 4.2, mu_p)."""
    return 2 * np.pi * _index(n) / width


def _odd(k):
    """Copy of a 1D wavenumber array with the Nyquist entry zeroed (reading 5)."""
    k = k.copy()
    if k.size % 2 == 0:
        k[k.size // 2] = 0.0
    return k


def wavenumbers(p, padded=False, odd=False):
    """Per-axis wavenumber arrays broadcast to the (padded) grid, vector order x,y,z."""
    p = params(p)
    out = []
    for j in range(p.dim):
        w = p.hi[j] - p.lo[j]
        n = p.n[j]
        k = _freq(2 * n, 2 * w) if padded else _freq(n, w)
        if odd:
            k = _odd(k)
        shape = [1] * p.dim
        shape[p.dim - 1 - j] = k.size
        out.append(k.reshape(shape))
    return out


def kinetic_symbol(p):
    """(|k|^2 + m^2)^s on the grid (Section 1, definition of the fractional operator)."""
    p = params(p)
    k2 = sum(k * k for k in wavenumbers(p))
    return (k2 + p.m * p.m) ** p.s


def kinetic_step(phi, p, tau):
    """Exact solution of Eq. 1step over time tau with periodic conditions on B.

    phi <- F^-1[ exp(-i tau/2 (|k|^2+m^2)^s) F phi ]; tau = dt/2 gives the
    half step of Eq. tssp1 / tssp3 (phase dt/4 (|k|^2+m^2)^s).
    """
    p = params(p)
    return np.fft.ifftn(np.exp(-0.5j * tau * kinetic_symbol(p)) * np.fft.fftn(phi))


def rotation(omega, t, dim):
    """A(t) of Eq. Amatrix."""
    c, s = math.cos(omega * t), math.sin(omega * t)
    if dim == 2:
        return np.array([[c, s], [-s, c]])
    return np.array([[c, s, 0.0], [-s, c, 0.0], [0.0, 0.0, 1.0]])


def _gl(a, b, nodes=20):
    x, w = np.polynomial.legendre.leggauss(nodes)
    return 0.5 * (b - a) * x + 0.5 * (a + b), 0.5 * (b - a) * w


def trap_potential(p, t, gamma=None):
    """W(x~, t) = V(A(t) x~) (Eq. FSE1_Rot) with V the harmonic trap of Eq. harm_poten,
    plus an optical lattice lat_amp sum_v sin^2(lat_k_v x_v) when lat_amp != 0 (the
    harmonic-plus-lattice potential of the Section 3.3 example; reading 10)."""
    p = params(p)
    g = p.gamma if gamma is None else tuple(gamma) + p.gamma[len(gamma):]
    X = coords(p)
    A = rotation(p.omega, t, p.dim)
    V = 0.0
    for v in range(p.dim):
        xv = sum(A[v, j] * X[j] for j in range(p.dim))
        V = V + 0.5 * g[v] ** 2 * xv * xv
        if p.lat_amp != 0.0:
            V = V + p.lat_amp * np.sin(p.lat_k[v] * xv) ** 2
    return V


def trap_integral(p, ta, tb, gamma=None, nodes=16):
    """P(x~) = int_{ta}^{tb} V(A(tau) x~) dtau (Eq. int_poten) by Gauss-Legendre (the
    numerical quadrature that Section 4.2 names for a general V)."""
    tq, wq = _gl(ta, tb, nodes)
    return sum(w * trap_potential(p, t, gamma) for t, w in zip(tq, wq))


def dipole_axis(p, t):
    """m(t) = A(t)^{-1} n (Section 4.2, below Eq. Kernel_Rot)."""
    p = params(p)
    n = np.asarray(p.dip_n, dtype=float)
    return rotation(p.omega, t, 3).T @ n


def dipole_integral(p, ta, tb, nodes=16):
    """M = int_{ta}^{tb} m(tau) m(tau)^T dtau (the operator L~_3 of Section 4.2)."""
    tq, wq = _gl(ta, tb, nodes)
    M = np.zeros((3, 3))
    for t, w in zip(tq, wq):
        m = dipole_axis(p, t)
        M += w * np.outer(m, m)
    return M


def _kernel_prefactor(p):
    """U(x) = 1/(2^{d-1} pi |x|^mu) (Eq. Kernel, Coulomb-type)."""
    return 1.0 / (2 ** (p.dim - 1) * math.pi)


def _box_scale(p):
    """Length of one unit of the unit box B1 = [-1,1]^d (Section 2): half the box width."""
    widths = [p.hi[j] - p.lo[j] for j in range(p.dim)]
    return 0.5 * max(widths)


def gausum_nodes(p):
    """Weights and nodes (w_q, tau_q) of U_GS (Eq. GS-Gene), physical units.

    Sinc quadrature of r^-mu = (2/Gamma(mu/2)) int exp(mu t - r^2 e^{2t}) dt
    with step h_s on [t_min, ln(7/delta)] in unit-box units (reading 3), then
    scaled to physical lengths and multiplied by the kernel prefactor.
    """
    p = params(p)
    sc = _box_scale(p)
    tmax = math.log(7.0 / p.gs_delta)
    nq = int(math.ceil((tmax - p.gs_tmin) / p.gs_h)) + 1
    t = p.gs_tmin + p.gs_h * np.arange(nq)
    # 1/|x|^mu with |x| = sc * r: sc^-mu * sum c_q exp(-(|x|/sc)^2 e^{2t_q})
    w = (2 * p.gs_h / math.gamma(p.mu / 2)) * np.exp(p.mu * t) * sc ** (-p.mu)
    tau = np.exp(t) / sc
    return w * _kernel_prefactor(p), tau


def gausum_g_table(tau, k, W, nodes=24):
    """g_q(k) = int_{-W}^{W} exp(-tau_q^2 y^2) cos(k y) dy (Eq. tensor), one row per q.

    Composite Gauss-Legendre on [0, Y_q], Y_q = min(W, 9/tau_q) (beyond it the
    integrand is below e^-81), panels sized to both the Gaussian and the
    highest oscillation.
    """
    k = np.asarray(k, dtype=float)
    out = np.empty((tau.size, k.size))
    xg, wg = np.polynomial.legendre.leggauss(nodes)
    kmax = float(np.max(np.abs(k))) if k.size else 0.0
    for q, tq in enumerate(tau):
        Y = min(W, 9.0 / tq)
        npan = int(max(4, math.ceil(kmax * Y / math.pi) + 4, math.ceil(tq * Y)))
        edges = np.linspace(0.0, Y, npan + 1)
        a, b = edges[:-1, None], edges[1:, None]
        y = (0.5 * (b - a) * xg[None, :] + 0.5 * (a + b)).ravel()
        wy = (0.5 * (b - a) * wg[None, :]).ravel()
        f = wy * np.exp(-(tq * y) ** 2)
        out[q] = 2.0 * (f @ np.cos(np.outer(y, k)))
    return out


def near_field(p, w, tau, panels=16, nodes=20):
    """I0 = int_{B_delta} (U - U_GS) and I2 = int_{B_delta} |y|^2 (U - U_GS).

    The two radial integrals of the near-field correction (Eq. taylor), by
    composite Gauss-Legendre with the d-dimensional Jacobian, in u with
    r = delta u^2 so that r^{d-1-mu} dr stays smooth for non-integer mu.
    """
    p = params(p)
    delta = p.gs_delta * _box_scale(p)
    edges = np.linspace(0.0, 1.0, panels + 1)
    xg, wg = np.polynomial.legendre.leggauss(nodes)
    a, b = edges[:-1, None], edges[1:, None]
    u = (0.5 * (b - a) * xg[None, :] + 0.5 * (a + b)).ravel()
    r = delta * u * u
    wr = (0.5 * (b - a) * wg[None, :]).ravel() * 2.0 * delta * u
    surf = 2 * math.pi * r if p.dim == 2 else 4 * math.pi * r * r
    U = _kernel_prefactor(p) * r ** (-p.mu)
    Ugs = np.exp(-np.outer(r * r, tau * tau)) @ w
    f = (U - Ugs) * surf * wr
    return float(np.sum(f)), float(np.sum(f * r * r))


def gausum_octant(p):
    """C^(k) on the non-negative padded frequencies |p_j| = 0..n_j, shape reversed(n+1).

    C^(k) = sum_q w_q prod_j g_q(k_j) + I0 - I2 |k|^2/(2d): the regular
    integral I1 of the zero-padded Fourier series (Eqs. FourSeriB3, tensor)
    plus the near-field Taylor correction (Eq. taylor; Delta rho <-> -|k|^2).
    """
    p = params(p)
    w, tau = gausum_nodes(p)
    tabs, ks = [], []
    for j in range(p.dim):
        W = p.hi[j] - p.lo[j]
        k = 2 * np.pi * np.arange(p.n[j] + 1) / (2 * W)
        ks.append(k)
        tabs.append(gausum_g_table(tau, k, W))
    if p.dim == 2:
        C = np.einsum("q,qy,qx->yx", w, tabs[1], tabs[0])
        k2 = ks[1][:, None] ** 2 + ks[0][None, :] ** 2
    else:
        C = np.einsum("q,qz,qy,qx->zyx", w, tabs[2], tabs[1], tabs[0], optimize=True)
        k2 = ks[2][:, None, None] ** 2 + ks[1][None, :, None] ** 2 + ks[0][None, None, :] ** 2
    I0, I2 = near_field(p, w, tau)
    return C + I0 - I2 * k2 / (2 * p.dim)


def gausum_multiplier(p, octant=None):
    """C^ on the full padded grid (numpy FFT order), from the octant by |p_j|."""
    p = params(p)
    oc = gausum_octant(p) if octant is None else octant
    idx = [np.abs(_index(2 * p.n[j])) for j in range(p.dim)]
    return oc[np.ix_(*reversed(idx))]


def _quad_form(p, M, Chat, factor=3.0):
    """factor (k^T M k) C^ over the grid's axes, odd factors zeroed at the Nyquist index (reading 5)."""
    k = wavenumbers(p, padded=True)
    ko = wavenumbers(p, padded=True, odd=True)
    q = 0.0
    for i in range(p.dim):
        q = q + M[i, i] * k[i] * k[i]
        for j in range(i + 1, p.dim):
            q = q + 2 * M[i, j] * ko[i] * ko[j]
    return factor * q * Chat


def _ksq(p):
    k = wavenumbers(p, padded=True)
    return sum(k[j] * k[j] for j in range(p.dim))


def kernel_multiplier(p, ta, tb, Chat=None):
    """Transform of the time-integrated kernel K~ over [ta, tb] (Eq. solu_step2_conv).

    Coulomb: (tb-ta) C^.  3D DDI: -(tb-ta) + 3 k^T M k C^ with M the integral
    of m m^T (the operator L~_3 applied to 1/(4 pi|x|)).  2D DDI:
    3/2 (k^T M_perp k - n_3^2 (tb-ta) |k|^2) C^ with C^ the transform of
    1/(2 pi|x|) and M_perp the in-plane block of M (Eq. Kernel, 2D DDI row).
    """
    p = params(p)
    C = gausum_multiplier(p) if Chat is None else Chat
    if p.kernel == "coulomb":
        return (tb - ta) * C
    if p.kernel == "ddi3d":
        return -(tb - ta) + _quad_form(p, dipole_integral(p, ta, tb), C)
    if p.kernel == "ddi2d":
        # -3/2 L~_2 (1/(2 pi|x|)) plus the rotation-invariant -3/2 (-n_3^2 Lap) part
        # of Eq. Kernel, integrated over the window (reading 9)
        n3 = float(p.dip_n[2])
        return _quad_form(p, dipole_integral(p, ta, tb), C, 1.5) - 1.5 * n3 * n3 * (tb - ta) * _ksq(p) * C
    return np.zeros_like(C)


def kernel_multiplier_instant(p, t, Chat=None):
    """Transform of U~(., t) (Eq. Kernel_Rot): C^ or -1 + 3 (m(t).k)^2 C^."""
    p = params(p)
    C = gausum_multiplier(p) if Chat is None else Chat
    if p.kernel == "coulomb":
        return C
    if p.kernel == "ddi3d":
        m = dipole_axis(p, t)
        return -1.0 + _quad_form(p, np.outer(m, m), C)
    if p.kernel == "ddi2d":
        m = dipole_axis(p, t)
        n3 = float(p.dip_n[2])
        return _quad_form(p, np.outer(m, m), C, 1.5) - 1.5 * n3 * n3 * _ksq(p) * C
    return np.zeros_like(C)


def pad(rho, p):
    """Zero-pad rho (on B) into the corner of the doubled grid (Section 2, reading 2)."""
    p = params(p)
    out = np.zeros(tuple(2 * v for v in p.shape()), dtype=rho.dtype)
    out[tuple(slice(0, v) for v in p.shape())] = rho
    return out


def crop(arr, p):
    p = params(p)
    return arr[tuple(slice(0, v) for v in p.shape())]


def nonlocal_potential(rho, p, khat):
    """int K(y) rho(x-y) dy on B: pad, FFT, multiply by the kernel transform, IFFT, crop."""
    return crop(np.fft.ifftn(np.fft.fftn(pad(rho, p)) * khat), p).real


def potential_step(u1, p, ta, tb, gamma=None, Chat=None):
    """Exact potential sub-step (Eqs. 2stepA/B, solu_step2) from ta to tb.

    u2 = u1 exp(-i [(tb-ta) beta rho + lambda varphi + P]), rho = |u1|^2 (reading 1),
    varphi = K~ * rho (Eq. solu_step2_conv), P from Eq. int_poten.
    """
    p = params(p)
    rho = np.abs(u1) ** 2
    theta = (tb - ta) * p.beta * rho + trap_integral(p, ta, tb, gamma)
    if p.kernel != "none" and p.lam != 0.0:
        theta = theta + p.lam * nonlocal_potential(rho, p, kernel_multiplier(p, ta, tb, Chat))
    return u1 * np.exp(-1j * theta)


def split_step(phi, p, tn, gamma=None, Chat=None):
    """One TS2-GauSum step from t_n to t_n + dt (Eqs. tssp1-tssp3)."""
    p = params(p)
    u1 = kinetic_step(phi, p, 0.5 * p.dt)
    u2 = potential_step(u1, p, tn, tn + p.dt, gamma, Chat)
    return kinetic_step(u2, p, 0.5 * p.dt)


# Fourth-order symmetric composition of three Strang steps ("triple jump",
# Yoshida 1990): S4(dt) = S2(w1 dt) S2(w0 dt) S2(w1 dt) with w1 = 1/(2 - 2^{1/3})
# and w0 = 1 - 2 w1 < 0 (the middle sub-step runs backwards in time). This is
# the extension of TS2-GauSum to higher-order splitting that Section 4.2 notes.
TRIPLE_JUMP_W1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
TRIPLE_JUMP_W0 = 1.0 - 2.0 * TRIPLE_JUMP_W1


def split_step4(phi, p, tn, gamma=None, Chat=None):
    """One fourth-order step from t_n to t_n + dt: three TS2-GauSum sub-steps
    of lengths w1 dt, w0 dt, w1 dt over consecutive windows."""
    p = params(p)
    t = tn
    for w in (TRIPLE_JUMP_W1, TRIPLE_JUMP_W0, TRIPLE_JUMP_W1):
        tau = w * p.dt
        u1 = kinetic_step(phi, p, 0.5 * tau)
        u2 = potential_step(u1, p, t, t + tau, gamma, Chat)
        phi = kinetic_step(u2, p, 0.5 * tau)
        t = t + tau
    return phi


def evolve(phi, p, t0, nsteps, gammas=None, Chat=None):
    """nsteps steps of order p.order; gammas (optional) is [nsteps][dim] per-step trap frequencies."""
    p = params(p)
    if Chat is None and p.kernel != "none":
        Chat = gausum_multiplier(p)
    step = split_step4 if p.order == 4 else split_step
    for n in range(nsteps):
        phi = step(phi, p, t0 + n * p.dt, None if gammas is None else gammas[n], Chat)
    return phi


def mass(phi, p):
    """N = int |phi|^2 (Eq. mass), rectangle rule on the periodic grid."""
    return float(np.prod(mesh_size(p)) * np.sum(np.abs(phi) ** 2))


def _spectral_deriv(phi, p, j):
    k = wavenumbers(p, odd=True)[j]
    return np.fft.ifftn(1j * k * np.fft.fftn(phi))


def observables(phi, p, t, gamma=None, Chat=None):
    """Mass, energy parts (Eq. energy), <L_z> (Eq. AME), centre of mass (Eq. CoM), widths (Eq. ConWidth).

    phi lives in the rotating Lagrangian frame at time t; the energy is that of
    Eq. SFSE (rotation term included), evaluated in x~ since the kinetic term,
    the interactions and L_z are invariant under the frame rotation and
    V(A(t) x~) = W(x~, t). Centre of mass and widths are returned in the
    frame of Eq. SFSE, x = A(t) x~.
    """
    p = params(p)
    hd = float(np.prod(mesh_size(p)))
    rho = np.abs(phi) ** 2
    ph = np.fft.fftn(phi)
    ntot = phi.size
    out = {}
    out["mass"] = hd * float(np.sum(rho))
    out["e_kin"] = 0.5 * hd / ntot * float(np.sum(kinetic_symbol(p) * np.abs(ph) ** 2))
    out["e_pot"] = hd * float(np.sum(trap_potential(p, t, gamma) * rho))
    out["e_int"] = 0.5 * p.beta * hd * float(np.sum(rho * rho))
    if p.kernel != "none":
        Phi = nonlocal_potential(rho, p, kernel_multiplier_instant(p, t, Chat))
        out["e_non"] = 0.5 * p.lam * hd * float(np.sum(Phi * rho))
    else:
        out["e_non"] = 0.0
    X = coords(p)
    dx = _spectral_deriv(phi, p, 0)
    dy = _spectral_deriv(phi, p, 1)
    lz = hd * np.sum(np.conj(phi) * (-1j) * (X[0] * dy - X[1] * dx))
    out["lz"] = float(lz.real)
    out["e_rot"] = -p.omega * out["lz"]
    out["energy"] = out["e_kin"] + out["e_pot"] + out["e_int"] + out["e_non"] + out["e_rot"]
    A = rotation(p.omega, t, p.dim)
    xt = np.array([hd * float(np.sum(X[j] * rho)) for j in range(p.dim)])
    out["xc"] = A @ xt
    S = np.array([[hd * float(np.sum(X[i] * X[j] * rho)) for j in range(p.dim)]
                  for i in range(p.dim)])
    out["width"] = np.diag(A @ S @ A.T).copy()
    return out


def com_velocity_spectral(phi, p):
    """Right side of Eq. PCoM2 in the rotating Lagrangian frame (no rotation term).

    d x~_c/dt = s (2 pi)^-d <(|k|^2+m^2)^{s-1} k phi^, phi^>, discretised as
    s (h^d / N) sum_k (|k|^2+m^2)^{s-1} k |DFT(phi)_k|^2 (k = 0 term is zero).
    """
    p = params(p)
    hd = float(np.prod(mesh_size(p)))
    k = wavenumbers(p)
    ko = wavenumbers(p, odd=True)
    k2 = sum(v * v for v in k) + p.m * p.m
    with np.errstate(divide="ignore", invalid="ignore"):
        fac = np.where(k2 > 0, k2 ** (p.s - 1.0), 0.0)
    a = np.abs(np.fft.fftn(phi)) ** 2
    return np.array([p.s * hd / phi.size * float(np.sum(fac * ko[j] * a)) for j in range(p.dim)])


# ---------------------------------------------------------------------------
# Adjoint of the split step (the paper has no adjoint; this is the transpose of
# the real-linearised map of Eqs. tssp1-tssp3, used by the gradient tests).
# Cotangents follow g = dJ/dRe(psi) + i dJ/dIm(psi).
# ---------------------------------------------------------------------------

def _kinetic_adjoint(g, p, tau):
    """Transpose of the unitary kinetic map: its conjugate phase."""
    p = params(p)
    return np.fft.ifftn(np.exp(0.5j * tau * kinetic_symbol(p)) * np.fft.fftn(g))


def _nonlocal_linear(r, p, ta, tb, Chat):
    return nonlocal_potential(r, p, kernel_multiplier(p, ta, tb, Chat))


def adjoint_split_step(phi_n, g_next, p, tn, gamma=None, Chat=None):
    """Pull a cotangent back through one split step.

    Forward: u1 = K phi_n, rho = |u1|^2, Theta = dt beta rho + lambda Kc rho + P,
    u2 = u1 exp(-i Theta), phi_{n+1} = K u2. Returns (g_n, dJ/dgamma_n) with
    dJ/dgamma_v = sum_x r dP/dgamma_v, r = Im(conj(g_u2) u2), the time integral
    of the trap being linear in gamma_v^2.
    """
    p = params(p)
    ta, tb = tn, tn + p.dt
    u1 = kinetic_step(phi_n, p, 0.5 * p.dt)
    rho = np.abs(u1) ** 2
    theta = (tb - ta) * p.beta * rho + trap_integral(p, ta, tb, gamma)
    if p.kernel != "none" and p.lam != 0.0:
        theta = theta + p.lam * _nonlocal_linear(rho, p, ta, tb, Chat)
    u2 = u1 * np.exp(-1j * theta)
    g_u2 = _kinetic_adjoint(g_next, p, 0.5 * p.dt)
    r = np.imag(np.conj(g_u2) * u2)
    q = (tb - ta) * p.beta * r
    if p.kernel != "none" and p.lam != 0.0:
        q = q + p.lam * _nonlocal_linear(r, p, ta, tb, Chat)
    g_u1 = np.exp(1j * theta) * g_u2 + 2.0 * q * u1
    g_n = _kinetic_adjoint(g_u1, p, 0.5 * p.dt)
    dgam = np.zeros(p.dim)
    g = p.gamma if gamma is None else tuple(gamma) + p.gamma[len(gamma):]
    for v in range(p.dim):
        one = [0.0] * 3
        one[v] = 1.0
        # dP/dgamma_v = gamma_v * int (A x~)_v^2 dtau = 2/gamma_v * (part of P)
        unit = params(dict(vars(p), gamma=tuple(one)))
        dP = 2.0 * g[v] * trap_integral(unit, ta, tb, None)
        dgam[v] = float(np.sum(r * dP))
    return g_n, dgam


def evolve_with_states(phi, p, t0, nsteps, gammas=None, Chat=None):
    """Forward run keeping every state phi_0..phi_T (for the oracle adjoint)."""
    p = params(p)
    if Chat is None and p.kernel != "none":
        Chat = gausum_multiplier(p)
    states = [phi]
    for n in range(nsteps):
        phi = split_step(phi, p, t0 + n * p.dt, None if gammas is None else gammas[n], Chat)
        states.append(phi)
    return states


def objective_overlap(phiT, target, p):
    """J = |<phi_T, target>|^2 with <f, g> = h^d sum f conj(g)."""
    hd = float(np.prod(mesh_size(p)))
    c = hd * np.sum(phiT * np.conj(target))
    return float(abs(c) ** 2)


def gradient_adjoint(phi0, target, p, t0, nsteps, gammas=None):
    """dJ/dphi0 (as dJ/dRe + i dJ/dIm) and dJ/dgamma [nsteps][dim] by the adjoint recursion."""
    p = params(p)
    Chat = gausum_multiplier(p) if p.kernel != "none" else None
    states = evolve_with_states(phi0, p, t0, nsteps, gammas, Chat)
    hd = float(np.prod(mesh_size(p)))
    c = hd * np.sum(states[-1] * np.conj(target))
    g = 2.0 * hd * c * target
    dgam = np.zeros((nsteps, p.dim))
    for n in range(nsteps - 1, -1, -1):
        g, dg = adjoint_split_step(states[n], g, p, t0 + n * p.dt,
                                   None if gammas is None else gammas[n], Chat)
        dgam[n] = dg
    return g, dgam


# ---------------------------------------------------------------------------
# Ground state by GF-GauSum (Section 3.2, Eqs. gf-eq2, gf-colb2, gffg33): the
# gradient flow with discrete normalisation, each backward-Euler step solved
# with BiCGStab on the left-preconditioned system of Eq. precond_type1,
#   (I + P_Delta A_TF) phi^(1) = P_Delta phi^n / dt,
#   P_Delta = [1/dt + (-Lap + m^2)^s / 2]^-1,  A_TF = V + beta|phi^n|^2 + lambda Phi^n - Omega L_z,
# followed by phi^{n+1} = phi^(1) / ||phi^(1)||. The problem is posed in the
# laboratory frame (no rotating coordinates): V is the trap at t = 0 and the
# dipole axis is n.
# ---------------------------------------------------------------------------

def gf_lz(v, p):
    """L_z v = -i (x d_y v - y d_x v) with spectral derivatives (Eq. AME)."""
    X = coords(p)
    return -1j * (X[0] * _spectral_deriv(v, p, 1) - X[1] * _spectral_deriv(v, p, 0))


def gf_potential(phi, p, Chat=None):
    """W = V + beta |phi|^2 + lambda Phi, Phi = U * |phi|^2 (Eq. gf-colb2)."""
    p = params(p)
    rho = np.abs(phi) ** 2
    W = trap_potential(p, 0.0) + p.beta * rho
    if p.kernel != "none" and p.lam != 0.0:
        W = W + p.lam * nonlocal_potential(rho, p, kernel_multiplier_instant(p, 0.0, Chat))
    return W


def gf_precond(v, p, dtg):
    """P_Delta v = F^-1 [F v / (1/dt + (|k|^2 + m^2)^s / 2)]."""
    return np.fft.ifftn(np.fft.fftn(v) / (1.0 / dtg + 0.5 * kinetic_symbol(p)))


def gf_matvec(v, W, p, dtg):
    """(I + P_Delta A_TF) v (left system of Eq. precond_type1)."""
    return v + gf_precond(W * v - p.omega * gf_lz(v, p), p, dtg)


def bicgstab(apply, b, x0, tol, maxit):
    """BiCGStab (van der Vorst 1992) for complex systems, inner product sum conj(a) b.

    Stops when ||r|| <= tol ||b||; returns (x, iterations, ||r|| / ||b||)."""
    dot = lambda a, c: np.vdot(a, c)
    x = x0.copy()
    r = b - apply(x)
    rh = r.copy()
    bn = math.sqrt(dot(b, b).real)
    rho_prev = alpha = omega = 1.0
    v = np.zeros_like(b)
    pp = np.zeros_like(b)
    it = 0
    res = math.sqrt(dot(r, r).real) / bn
    while it < maxit and res > tol:
        rho = dot(rh, r)
        beta = (rho / rho_prev) * (alpha / omega)
        pp = r + beta * (pp - omega * v)
        v = apply(pp)
        alpha = rho / dot(rh, v)
        s = r - alpha * v
        t = apply(s)
        omega = dot(t, s) / dot(t, t)
        x = x + alpha * pp + omega * s
        r = s - omega * t
        rho_prev = rho
        it += 1
        res = math.sqrt(dot(r, r).real) / bn
    return x, it, res


def gf_step(phi, p, dtg, Chat=None, inner_tol=1e-13, max_inner=500):
    """One GFDN step: backward-Euler solve, then normalisation (Eqs. gf-eq2, gffg33)."""
    p = params(p)
    W = gf_potential(phi, p, Chat)
    b = gf_precond(phi / dtg, p, dtg)
    x, it, _ = bicgstab(lambda v: gf_matvec(v, W, p, dtg), b, phi, inner_tol, max_inner)
    return x / math.sqrt(mass(x, p)), it


def ground_state(phi0, p, dtg, max_outer, tol=0.0, inner_tol=1e-13, max_inner=500):
    """GF-GauSum iterations from phi0 until max|phi^{n+1} - phi^n| / dt <= tol or max_outer steps.

    Returns (phi, outer steps, total inner iterations, last change)."""
    p = params(p)
    Chat = gausum_multiplier(p) if p.kernel != "none" else None
    phi = phi0 / math.sqrt(mass(phi0, p))
    inner, change, n = 0, float("inf"), 0
    while n < max_outer:
        nxt, it = gf_step(phi, p, dtg, Chat, inner_tol, max_inner)
        inner += it
        change = float(np.max(np.abs(nxt - phi))) / dtg
        phi = nxt
        n += 1
        if change <= tol:
            break
    return phi, n, inner, change


def gf_hamiltonian(phi, p, Chat=None):
    """H[phi] phi = (-Lap+m^2)^s phi / 2 + W phi - Omega L_z phi (the operator of Eq. gf-eq1)."""
    p = params(p)
    kin = 0.5 * np.fft.ifftn(kinetic_symbol(p) * np.fft.fftn(phi))
    return kin + gf_potential(phi, p, Chat) * phi - p.omega * gf_lz(phi, p)


def shift_kick(phi, p, x0=None, k=None):
    """phi(x - x0) exp(i k.x): the shifted and kicked initial data of Eq. ini_dyn.

    The translation uses the shift theorem on the periodic grid (reading 11);
    at the Nyquist index of each axis the factor is cos(k_N x0_j), the mean of
    the two aliases +-k_N. The kick multiplies pointwise."""
    p = params(p)
    out = np.asarray(phi, dtype=complex)
    if x0 is not None and any(x0[j] != 0.0 for j in range(p.dim)):
        fac = 1.0
        for j in range(p.dim):
            n = p.n[j]
            kj = _freq(n, p.hi[j] - p.lo[j])
            f = np.exp(-1j * kj * x0[j])
            f[n // 2] = math.cos(kj[n // 2] * x0[j])
            shape = [1] * p.dim
            shape[p.dim - 1 - j] = n
            fac = fac * f.reshape(shape)
        out = np.fft.ifftn(fac * np.fft.fftn(out))
    if k is not None and any(k[j] != 0.0 for j in range(p.dim)):
        X = coords(p)
        out = out * np.exp(1j * sum(k[j] * X[j] for j in range(p.dim)))
    return out

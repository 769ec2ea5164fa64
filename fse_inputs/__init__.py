"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the split-step method. It only defines
(a) a counter-free SplitMix64 stream (Steele, Lea & Flood 2014) with uniform
and Box-Muller normal draws, (b) the parameter sets of the workloads and
(c) their initial wave functions, all in float64 on the host.

Workloads (named by what they are):

* ``2d_coulomb_128``   -- 2D, 128x128 on [-8,8]^2, s=0.8, Omega=0.6, Coulomb mu=1.
* ``3d_dipolar_128``   -- 3D, 128^3 on [-8,8]^3, s=0.7, Omega=0.8, dipolar.
* ``batched_2d``       -- 256 independent 2D Coulomb runs of mixed sizes.
* ``adjoint_2d_256``   -- 2D, 256^2, per-step trap frequencies.
* ``3d_dipolar_256``   -- 3D, 256^3 on [-12,12]^3, s=0.6, Omega=0.9, dipolar,
                          16-vortex Thomas-Fermi-like initial state.

The paper's own dynamics start from ground states (Section 4.3), which do not
exist for 0<s<1 with Omega>0 (Theorem 3.1); synthetic states of the same
shapes stand in for them.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "SplitMix64", "WORKLOADS", "workload", "grid_axes", "psi0",
    "batched_runs", "adjoint_gammas", "adjoint_target",
]

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator; ``next_u64`` follows the published constants."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self, count: int) -> np.ndarray:
        out = np.empty(count, dtype=np.uint64)
        st = self.state
        for i in range(count):
            st = (st + 0x9E3779B97F4A7C15) & _MASK
            z = st
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
            out[i] = z ^ (z >> 31)
        self.state = st
        return out

    def next_u64_fast(self, count: int) -> np.ndarray:
        """Vectorised equivalent of ``next_u64`` (same stream)."""
        with np.errstate(over="ignore"):
            idx = np.arange(1, count + 1, dtype=np.uint64)
            st = np.uint64(self.state) + idx * np.uint64(0x9E3779B97F4A7C15)
            z = st.copy()
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + count * 0x9E3779B97F4A7C15) & _MASK
        return z

    def uniform(self, count: int) -> np.ndarray:
        """Uniform doubles in [0, 1) from the top 53 bits."""
        return (self.next_u64_fast(count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, count: int) -> np.ndarray:
        """Standard normal doubles by the Box-Muller transform."""
        m = (count + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))          # 1-u1 in (0,1]
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:count]


_SQ = 1.0 / math.sqrt(2.0)

# Parameter sets. Keys mirror the fields of fse_params in include/fse.h.
WORKLOADS = {
    "2d_coulomb_128": dict(
        dim=2, n=(128, 128), lo=(-8.0, -8.0), hi=(8.0, 8.0), s=0.8, m=0.0, omega=0.6,
        beta=100.0, lam=10.0, dt=1e-3, kernel="coulomb", mu=1.0, dip_n=(0.0, 0.0, 1.0),
        gamma=(1.0, 1.0), steps=100, seed=0, prec="f64"),
    "3d_dipolar_128": dict(
        dim=3, n=(128, 128, 128), lo=(-8.0,) * 3, hi=(8.0,) * 3, s=0.7, m=0.0, omega=0.8,
        beta=200.0, lam=60.0, dt=5e-4, kernel="ddi3d", mu=1.0, dip_n=(_SQ, 0.0, _SQ),
        gamma=(1.0, 1.2, 2.0), steps=1000, seed=1, prec="f32"),
    "batched_2d": dict(
        dim=2, runs=256, sizes=(128, 192, 256, 384, 512), lo=(-8.0, -8.0), hi=(8.0, 8.0),
        m=0.0, lam=10.0, dt=1e-3, kernel="coulomb", mu=1.0, gamma=(1.0, 1.0),
        steps=500, seed=2, prec="f32"),
    "adjoint_2d_256": dict(
        dim=2, n=(256, 256), lo=(-8.0, -8.0), hi=(8.0, 8.0), s=0.6, m=0.0, omega=0.7,
        beta=100.0, lam=10.0, dt=1e-3, kernel="coulomb", mu=1.0, dip_n=(0.0, 0.0, 1.0),
        gamma=(1.0, 1.0), steps=200, seed=3, prec="f32"),
    "gs_2d_512": dict(
        dim=2, n=(512, 512), lo=(-32.0, -32.0), hi=(32.0, 32.0), s=0.8, m=0.0, omega=0.0,
        beta=10.0, lam=10.0, dt=1e-3, kernel="coulomb", mu=1.0, dip_n=(0.0, 0.0, 1.0),
        gamma=(1.0, 1.0), steps=20, seed=5, prec="f64", init="gs_guess"),
    "3d_dipolar_256": dict(
        dim=3, n=(256, 256, 256), lo=(-12.0,) * 3, hi=(12.0,) * 3, s=0.6, m=0.0, omega=0.9,
        beta=500.0, lam=100.0, dt=2.5e-4, kernel="ddi3d", mu=1.0, dip_n=(_SQ, 0.0, _SQ),
        gamma=(1.0, 1.2, 2.0), steps=2000, seed=4, prec="f32"),
}


def workload(name: str, **override) -> dict:
    """Copy of a named parameter set with optional overrides (e.g. a smaller n)."""
    w = dict(WORKLOADS[name])
    w.update(override)
    return w


def grid_axes(p: dict):
    """Per-axis node coordinates lo + i*h, i=0..n-1, ordered (x, y[, z])."""
    return [p["lo"][j] + (p["hi"][j] - p["lo"][j]) / p["n"][j] * np.arange(p["n"][j])
            for j in range(p["dim"])]


def _mesh(p: dict):
    ax = grid_axes(p)
    if p["dim"] == 2:
        Y, X = np.meshgrid(ax[1], ax[0], indexing="ij")
        return X, Y, None
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def _mass(p: dict, psi: np.ndarray) -> float:
    h = np.prod([(p["hi"][j] - p["lo"][j]) / p["n"][j] for j in range(p["dim"])])
    return float(h * np.sum(np.abs(psi) ** 2))


def psi0(name_or_params, **override) -> np.ndarray:
    """Initial wave function (complex128, shape [nz][ny][nx] or [ny][nx], x fastest).

    * 2D workloads: pi^{-1/2} exp(-((x-1)^2+y^2)/2) (unit mass).
    * ``gs_2d_512`` (ground state): ((1-Omega) phi_ho + Omega phi^v_ho) / norm with
      phi_ho = pi^{-1/2} e^{-|x|^2/2}, phi^v_ho = (x+iy) phi_ho (the shape of the
      paper's initial guess for its ground-state runs).
    * ``3d_dipolar_128``: anisotropic Gaussian (gx gy gz)^{1/4} pi^{-3/4}
      exp(-sum g_v v^2/2) times exp(i 1e-3 xi), xi i.i.d. N(0,1) per point.
    * ``3d_dipolar_256``: Thomas-Fermi-like envelope sqrt(max(0,1-sum (v/R_v)^2)),
      R_v = 5/g_v, smoothed by a Gaussian of width 2h (spectrally), times 16
      phase vortices along z on a jittered 4x4 lattice (spacing 1.5, jitter
      U[-0.2,0.2]); normalised to unit mass.
    """
    if isinstance(name_or_params, str):
        p = workload(name_or_params, **override)
        kind = name_or_params
    else:
        p = dict(name_or_params)
        p.update(override)
        kind = p.get("init", "gauss2d" if p["dim"] == 2 else "gauss3d")
    X, Y, Z = _mesh(p)
    rng = SplitMix64(p.get("seed", 0))
    if p["dim"] == 2 and (kind == "gs_2d_512" or p.get("init") == "gs_guess"):
        # ground-state initial guess ((1-Omega) phi_ho + Omega phi^v_ho), normalised
        om = p.get("omega", 0.0)
        ho = np.pi ** -0.5 * np.exp(-(X ** 2 + Y ** 2) / 2)
        psi = ((1 - om) * ho + om * (X + 1j * Y) * ho).astype(np.complex128)
        return psi / math.sqrt(_mass(p, psi))
    if p["dim"] == 2 and kind != "vortex3d":
        x0 = p.get("x0", (1.0, 0.0))
        return (np.pi ** -0.5 * np.exp(-((X - x0[0]) ** 2 + (Y - x0[1]) ** 2) / 2)).astype(np.complex128)
    g = p["gamma"]
    if kind in ("3d_dipolar_256", "vortex3d"):
        R = [5.0 / g[0], 5.0 / g[1], 5.0 / g[2]]
        env = np.sqrt(np.maximum(0.0, 1 - (X / R[0]) ** 2 - (Y / R[1]) ** 2 - (Z / R[2]) ** 2))
        # Gaussian smoothing of width 2h, applied as a spectral multiplier.
        h = [(p["hi"][j] - p["lo"][j]) / p["n"][j] for j in range(3)]
        ks = [2 * np.pi * np.fft.fftfreq(p["n"][j], d=h[j]) for j in range(3)]
        KZ, KY, KX = np.meshgrid(ks[2], ks[1], ks[0], indexing="ij")
        w = 2 * h[0]
        env = np.fft.ifftn(np.fft.fftn(env) * np.exp(-0.5 * w * w * (KX ** 2 + KY ** 2 + KZ ** 2))).real
        jit = rng.uniform(32) * 0.4 - 0.2
        psi = env.astype(np.complex128)
        c = 0
        for a in range(4):
            for b in range(4):
                xj = (a - 1.5) * 1.5 + jit[c]
                yj = (b - 1.5) * 1.5 + jit[c + 16]
                c += 1
                z = (X - xj) + 1j * (Y - yj)
                mag = np.abs(z)
                psi *= np.where(mag > 0, z / np.where(mag > 0, mag, 1.0), 0.0)
        return psi / math.sqrt(_mass(p, psi))
    amp = (g[0] * g[1] * g[2]) ** 0.25 * np.pi ** -0.75
    psi = amp * np.exp(-(g[0] * X ** 2 + g[1] * Y ** 2 + g[2] * Z ** 2) / 2)
    noise = p.get("phase_noise", 1e-3)
    if noise:
        xi = rng.normal(psi.size).reshape(psi.shape)
        psi = psi * np.exp(1j * noise * xi)
    return psi.astype(np.complex128)


def batched_runs(count: int | None = None, seed: int = 2) -> list:
    """Per-run parameters of the batched 2D workload (sizes, s, Omega, beta)."""
    base = WORKLOADS["batched_2d"]
    count = base["runs"] if count is None else count
    rng = SplitMix64(seed)
    u = rng.uniform(4 * count).reshape(count, 4)
    runs = []
    for r in range(count):
        n = base["sizes"][min(int(u[r, 0] * len(base["sizes"])), len(base["sizes"]) - 1)]
        runs.append(dict(
            dim=2, n=(n, n), lo=base["lo"], hi=base["hi"], s=0.3 + 0.7 * u[r, 1], m=0.0,
            omega=0.95 * u[r, 2], beta=50.0 + 450.0 * u[r, 3], lam=base["lam"], dt=base["dt"],
            kernel="coulomb", mu=1.0, dip_n=(0.0, 0.0, 1.0), gamma=base["gamma"],
            steps=base["steps"], seed=1000 + r, prec="f32"))
    return runs


def adjoint_gammas(nsteps: int = 200, seed: int = 3) -> np.ndarray:
    """Per-step trap frequencies [nsteps][2]: 1 + 0.2 sum_j (a_j/j) sin(2 pi j n/T + phi_j)."""
    rng = SplitMix64(seed)
    a = rng.uniform(8).reshape(2, 4) * 2 - 1
    ph = rng.uniform(8).reshape(2, 4) * 2 * np.pi
    nn = np.arange(nsteps)
    out = np.ones((nsteps, 2))
    for v in range(2):
        for j in range(1, 5):
            out[:, v] += 0.2 * a[v, j - 1] / j * np.sin(2 * np.pi * j * nn / nsteps + ph[v, j - 1])
    return out


def adjoint_target(p: dict, seed: int = 3) -> np.ndarray:
    """Target state pi^{-1/2} exp(-|x-x_t|^2/2), x_t ~ U[-1,1]^2."""
    rng = SplitMix64(seed + 100)
    xt = rng.uniform(2) * 2 - 1
    X, Y, _ = _mesh(p)
    return (np.pi ** -0.5 * np.exp(-((X - xt[0]) ** 2 + (Y - xt[1]) ** 2) / 2)).astype(np.complex128)

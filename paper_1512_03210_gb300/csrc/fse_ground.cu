// fse_ground.cu -- ground state by GF-GauSum (Section 3.2, Eqs. gf-eq2, gf-colb2, gffg33),
// and the shifted and kicked initial data of the dynamics runs (Section 4.3, Eq. ini_dyn).
//
// Gradient flow with discrete normalisation, discretised by backward Euler:
//   (1/dt + (-Lap + m^2)^s / 2 + W_n - Omega L_z) phi^(1) = phi^n / dt,
//   W_n = V + beta |phi^n|^2 + lambda Phi^n,  Phi^n = U * |phi^n|^2,
//   phi^{n+1} = phi^(1) / ||phi^(1)||,
// each step solved by BiCGStab on the left system of Eq. precond_type1,
//   (I + P_Delta A_TF) phi^(1) = P_Delta phi^n / dt,
//   P_Delta = [1/dt + (|k|^2 + m^2)^s / 2]^-1,  A_TF = W_n - Omega L_z,
// with L_z = -i (x d_y - y d_x) by spectral derivatives. The problem is posed
// in the laboratory frame: V is the trap (harmonic plus optional lattice) and
// the dipole axis is n. Every transform runs through the plan's FFT passes;
// the BiCGStab vectors live in a caller-supplied workspace, and its scalars
// (inner products, alpha, omega, beta, the residual) stay on the device: the
// host reads them one iteration behind the GPU to stop the solve.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstring>

#include "fse.h"
#include "fse_internal.h"
#include "fse_passes.cuh"

namespace fse {
namespace {

constexpr int kGsBlocks = 1024;  // reduction partials per value

struct GsGrid {
  int nx, ny, nz;
  double lo[3], h[3], dk[3];
};

__device__ __forceinline__ void gs_index(long long i, const GsGrid& g, int& ix, int& iy, int& iz) {
  ix = (int)(i % g.nx);
  const long long r = i / g.nx;
  iy = (int)(r % g.ny);
  iz = (int)(r / g.ny);
}

// P_Delta / N on the spectrum: 1 / (N (1/dt + (|k|^2 + m^2)^s / 2)), k signed (Nyquist -n/2)
template <typename Real>
__global__ void k_gs_precond_table(Real* pk, GsGrid g, double inv_dt, double s, double m2, double inv_n) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    gs_index(i, g, ix, iy, iz);
    const int px = ix < g.nx / 2 ? ix : ix - g.nx, py = iy < g.ny / 2 ? iy : iy - g.ny;
    const int pz = g.nz > 1 ? (iz < g.nz / 2 ? iz : iz - g.nz) : 0;
    const double kx = g.dk[0] * px, ky = g.dk[1] * py, kz = g.dk[2] * pz;
    const double k2 = kx * kx + ky * ky + kz * kz + m2;
    pk[i] = Real(inv_n / (inv_dt + 0.5 * (k2 > 0.0 ? pow(k2, s) : 0.0)));
  }
}

// W = V + beta |phi|^2 + lambda Phi, V = sum_v gamma_v^2 x_v^2 / 2 + lat_amp sum_v sin^2(lat_k_v x_v)
template <typename Real>
__global__ void k_gs_potential(const typename Cplx<Real>::T* __restrict__ phi, const Real* __restrict__ Phi,
                               Real* __restrict__ W, GsGrid g, double3 g2, double beta, double lam, double lat_amp,
                               double3 lk) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    gs_index(i, g, ix, iy, iz);
    const double x = g.lo[0] + g.h[0] * ix, y = g.lo[1] + g.h[1] * iy, z = g.lo[2] + g.h[2] * iz;
    double v = g2.x * x * x + g2.y * y * y + g2.z * z * z;
    if (lat_amp != 0.0) {
      const double sx = sin(lk.x * x), sy = sin(lk.y * y), sz = sin(lk.z * z);
      v += lat_amp * (sx * sx + sy * sy + sz * sz);
    }
    const typename Cplx<Real>::T u = phi[i];
    v += beta * ((double)u.x * u.x + (double)u.y * u.y);
    if (Phi) v += lam * (double)Phi[i];
    W[i] = Real(v);
  }
}

// d = i k_axis sp / N, the odd factor zero at the Nyquist index
template <typename Real>
__global__ void k_gs_ik(const typename Cplx<Real>::T* __restrict__ sp, typename Cplx<Real>::T* __restrict__ d,
                        GsGrid g, int axis, double inv_n) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    gs_index(i, g, ix, iy, iz);
    const int idx = axis == 0 ? ix : iy, n = axis == 0 ? g.nx : g.ny;
    const Real k = (2 * idx == n) ? Real(0) : Real(g.dk[axis] * inv_n) * Real(wrap_index(idx, n));
    const typename Cplx<Real>::T u = sp[i];
    d[i] = mk(-k * u.y, k * u.x);
  }
}

// out = A_TF u = W u - Omega L_z u = W u + i Omega (x d_y u - y d_x u)
template <typename Real>
__global__ void k_gs_atf(const typename Cplx<Real>::T* __restrict__ u, const typename Cplx<Real>::T* __restrict__ dx,
                         const typename Cplx<Real>::T* __restrict__ dy, const Real* __restrict__ W,
                         typename Cplx<Real>::T* __restrict__ out, GsGrid g, double omega) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const typename Cplx<Real>::T a = u[i];
    const Real w = W[i];
    Real re = w * a.x, im = w * a.y;
    if (omega != 0.0) {
      int ix, iy, iz;
      gs_index(i, g, ix, iy, iz);
      const Real x = Real(g.lo[0] + g.h[0] * ix), y = Real(g.lo[1] + g.h[1] * iy);
      const typename Cplx<Real>::T bx = dx[i], by = dy[i];
      const Real lr = x * by.x - y * bx.x, li = x * by.y - y * bx.y;  // x d_y u - y d_x u
      re -= Real(omega) * li;                                          // i Omega (lr + i li)
      im += Real(omega) * lr;
    }
    out[i] = mk(re, im);
  }
}

template <typename Real>
__global__ void k_gs_scale_real(typename Cplx<Real>::T* __restrict__ d, const Real* __restrict__ pk, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const typename Cplx<Real>::T u = d[i];
    const Real f = pk[i];
    d[i] = mk(f * u.x, f * u.y);
  }
}

// out = ca A + cb B + cc Cc (complex coefficients; a null operand counts as zero)
template <typename Real>
__global__ void k_gs_lincomb(typename Cplx<Real>::T* out, const typename Cplx<Real>::T* A, double2 ca,
                             const typename Cplx<Real>::T* B, double2 cb, const typename Cplx<Real>::T* Cc, double2 cc,
                             long long N) {
  typedef typename Cplx<Real>::T C;
  const C a = mk(Real(ca.x), Real(ca.y)), b = mk(Real(cb.x), Real(cb.y)), c = mk(Real(cc.x), Real(cc.y));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    C r = mk(Real(0), Real(0));
    if (A) r = cadd(r, cmul(A[i], a));
    if (B) r = cadd(r, cmul(B[i], b));
    if (Cc) r = cadd(r, cmul(Cc[i], c));
    out[i] = r;
  }
}

// block partials of sum conj(a1) b1 and sum conj(a2) b2 (float64): part[v * kGsBlocks + block], v = 0..3
template <typename Real>
__global__ void __launch_bounds__(256) k_gs_dot2(const typename Cplx<Real>::T* a1, const typename Cplx<Real>::T* b1,
                                                 const typename Cplx<Real>::T* a2, const typename Cplx<Real>::T* b2,
                                                 long long N, double* part) {
  __shared__ double red[32];
  double acc[4] = {0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const typename Cplx<Real>::T x1 = a1[i], y1 = b1[i], x2 = a2[i], y2 = b2[i];
    acc[0] += (double)x1.x * y1.x + (double)x1.y * y1.y;
    acc[1] += (double)x1.x * y1.y - (double)x1.y * y1.x;
    acc[2] += (double)x2.x * y2.x + (double)x2.y * y2.y;
    acc[3] += (double)x2.x * y2.y - (double)x2.y * y2.x;
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const double t = block_sum(acc[v], red);
    if (threadIdx.x == 0) part[v * kGsBlocks + blockIdx.x] = t;
  }
}

// block partials of max |a - b|
template <typename Real>
__global__ void __launch_bounds__(256) k_gs_maxdiff(const typename Cplx<Real>::T* a, const typename Cplx<Real>::T* b,
                                                    long long N, double* part) {
  __shared__ double red[256];
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const double dx = (double)a[i].x - b[i].x, dy = (double)a[i].y - b[i].y;
    m = fmax(m, sqrt(dx * dx + dy * dy));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// out[v] = sum (max = 1: max) over the count partials of value v (one block per value)
__global__ void __launch_bounds__(256) k_gs_final(const double* part, int count, int max, double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const double v = part[blockIdx.x * kGsBlocks + i];
    acc = max ? fmax(acc, v) : acc + v;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      red[threadIdx.x] = max ? fmax(red[threadIdx.x], red[threadIdx.x + o]) : red[threadIdx.x] + red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
// BiCGStab scalars on the device. The state sc[] holds, in float64,
//   rho (complex, sc[0..1]), rho_prev (sc[2..3]), alpha (sc[4..5]),
//   omega (sc[6..7]), beta (sc[8..9]), ||b|| (sc[10]), ||r|| / ||b|| (sc[11]),
//   done (sc[12]: converged or broken down), iterations (sc[13]), tol (sc[14]).
// One-thread kernels update it from the inner products in out[] (written by
// k_gs_final), and the vector updates read their coefficients from it, so an
// inner iteration needs no host round trip. Once done is set, every update
// leaves its output untouched.
// ---------------------------------------------------------------------------
enum { SC_RHO = 0, SC_RHOP = 2, SC_ALPHA = 4, SC_OM = 6, SC_BETA = 8, SC_BN = 10, SC_RES = 11, SC_DONE = 12,
       SC_IT = 13, SC_TOL = 14, SC_SIZE = 16 };

__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 ld2(const double* p) { return make_double2(p[0], p[1]); }
__device__ __forceinline__ void st2(double* p, double2 v) {
  p[0] = v.x;
  p[1] = v.y;
}

// after <s, s>, <r, r> (s = b, r = b - M x, rh = r): the start of an inner solve
__global__ void k_gs_sc_init(double* sc, const double* out, double tol) {
  const double bn = sqrt(out[0]);
  const double res = bn > 0.0 ? sqrt(out[2]) / bn : 0.0;
  st2(sc + SC_RHO, make_double2(out[2], out[3]));
  st2(sc + SC_RHOP, make_double2(1.0, 0.0));
  st2(sc + SC_ALPHA, make_double2(1.0, 0.0));
  st2(sc + SC_OM, make_double2(1.0, 0.0));
  st2(sc + SC_BETA, make_double2(0.0, 0.0));
  sc[SC_BN] = bn;
  sc[SC_RES] = res;
  sc[SC_TOL] = tol;
  sc[SC_IT] = 0.0;
  sc[SC_DONE] = (!(res > tol) || (out[2] == 0.0 && out[3] == 0.0)) ? 1.0 : 0.0;
}

// after <rh, v>: alpha = rho / <rh, v> (breakdown when it vanishes)
__global__ void k_gs_sc_alpha(double* sc, const double* out) {
  if (sc[SC_DONE] != 0.0) return;
  const double2 rv = make_double2(out[0], out[1]);
  if (rv.x == 0.0 && rv.y == 0.0) {
    sc[SC_DONE] = 1.0;
    return;
  }
  st2(sc + SC_ALPHA, zdiv(ld2(sc + SC_RHO), rv));
}

// after <t, s>, <t, t>: omega = <t, s> / <t, t> (0 if <t, t> = 0)
__global__ void k_gs_sc_omega(double* sc, const double* out) {
  if (sc[SC_DONE] != 0.0) return;
  st2(sc + SC_OM, out[2] > 0.0 ? make_double2(out[0] / out[2], out[1] / out[2]) : make_double2(0.0, 0.0));
}

// after <rh, r>, <r, r>: the end of an iteration
__global__ void k_gs_sc_rho(double* sc, const double* out) {
  if (sc[SC_DONE] != 0.0) return;
  const double2 rho_prev = ld2(sc + SC_RHO), rho = make_double2(out[0], out[1]);
  const double2 alpha = ld2(sc + SC_ALPHA), om = ld2(sc + SC_OM);
  st2(sc + SC_RHOP, rho_prev);
  st2(sc + SC_RHO, rho);
  const double res = sqrt(out[2]) / sc[SC_BN];
  sc[SC_RES] = res;
  sc[SC_IT] += 1.0;
  const bool om0 = om.x == 0.0 && om.y == 0.0, rho0 = rho.x == 0.0 && rho.y == 0.0;
  if (om0 || rho0 || !(res > sc[SC_TOL])) {
    sc[SC_DONE] = 1.0;
    return;
  }
  // beta of the next iteration: (rho / rho_prev) (alpha / omega)
  st2(sc + SC_BETA, zmul(zdiv(rho, rho_prev), zdiv(alpha, om)));
}

enum { GS_P = 0, GS_S = 1, GS_X = 2, GS_R = 3 };
// The BiCGStab vector updates with coefficients from sc (nothing when done):
//   GS_P: o = A + beta (o - omega Cc)   (o = A on the first iteration)
//   GS_S: o = A - alpha Cc               GS_X: o = o + alpha A + omega Cc
//   GS_R: o = A - omega Cc
template <typename Real, int MODE>
__global__ void k_gs_update(typename Cplx<Real>::T* o, const typename Cplx<Real>::T* A,
                            const typename Cplx<Real>::T* Cc, const double* sc, long long N) {
  typedef typename Cplx<Real>::T C;
  if (sc[SC_DONE] != 0.0) return;
  const double2 al = ld2(sc + SC_ALPHA), om = ld2(sc + SC_OM), be = ld2(sc + SC_BETA);
  const bool first = sc[SC_IT] == 0.0;
  C c1, c2;
  if (MODE == GS_P) {
    c1 = mk(Real(be.x), Real(be.y));
    const double2 bo = zmul(be, om);
    c2 = mk(Real(-bo.x), Real(-bo.y));
  } else if (MODE == GS_S) {
    c2 = mk(Real(-al.x), Real(-al.y));
  } else if (MODE == GS_X) {
    c1 = mk(Real(al.x), Real(al.y));
    c2 = mk(Real(om.x), Real(om.y));
  } else {
    c2 = mk(Real(-om.x), Real(-om.y));
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    C r;
    if (MODE == GS_P) r = first ? A[i] : cadd(A[i], cadd(cmul(o[i], c1), cmul(Cc[i], c2)));
    else if (MODE == GS_X) r = cadd(o[i], cadd(cmul(A[i], c1), cmul(Cc[i], c2)));
    else r = cadd(A[i], cmul(Cc[i], c2));
    o[i] = r;
  }
}

// Spectral translation by x0 (the Nyquist mode takes cos(k_N x0), the mean of
// its two aliases) and 1/N for the unnormalised inverse.
template <typename Real>
__global__ void k_gs_shift(typename Cplx<Real>::T* __restrict__ sp, GsGrid g, double3 x0, double inv_n) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    gs_index(i, g, ix, iy, iz);
    const int nn[3] = {g.nx, g.ny, g.nz};
    const int id[3] = {ix, iy, iz};
    const double xs[3] = {x0.x, x0.y, x0.z};
    double re = inv_n, im = 0.0;
    for (int j = 0; j < 3; ++j) {
      if (nn[j] == 1 || xs[j] == 0.0) continue;
      const double k = g.dk[j] * wrap_index(id[j], nn[j]);
      double c, s;
      if (2 * id[j] == nn[j]) {
        c = cos(k * xs[j]);
        s = 0.0;
      } else {
        sincos(-k * xs[j], &s, &c);
      }
      const double r2 = re * c - im * s, i2 = re * s + im * c;
      re = r2;
      im = i2;
    }
    const typename Cplx<Real>::T u = sp[i];
    sp[i] = mk(Real(re * u.x - im * u.y), Real(re * u.y + im * u.x));
  }
}

// psi *= exp(i k . x)
template <typename Real>
__global__ void k_gs_kick(typename Cplx<Real>::T* __restrict__ psi, GsGrid g, double3 kv) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    int ix, iy, iz;
    gs_index(i, g, ix, iy, iz);
    const double ph = kv.x * (g.lo[0] + g.h[0] * ix) + kv.y * (g.lo[1] + g.h[1] * iy) + kv.z * (g.lo[2] + g.h[2] * iz);
    double s, c;
    sincos(ph, &s, &c);
    const typename Cplx<Real>::T u = psi[i];
    psi[i] = mk(Real(c * u.x - s * u.y), Real(c * u.y + s * u.x));
  }
}

GsGrid gs_grid(const fse_plan* P) {
  GsGrid g;
  g.nx = P->nx;
  g.ny = P->ny;
  g.nz = P->nz;
  for (int j = 0; j < 3; ++j) {
    g.lo[j] = j < P->dim ? P->p.lo[j] : 0.0;
    g.h[j] = j < P->dim ? P->h[j] : 0.0;
    g.dk[j] = j < P->dim ? 2 * kPi / (P->p.hi[j] - P->p.lo[j]) : 0.0;
  }
  return g;
}

template <typename Real>
fse_status shift_kick(fse_plan* P, void* psi, const double* x0, const double* kv) {
  const GsGrid g = gs_grid(P);
  const long long N = (long long)P->nx * P->ny * P->nz;
  const int blocks = (int)std::min<long long>(kGsBlocks, (N + 255) / 256);
  fse_status st;
  if (x0 && (x0[0] != 0.0 || x0[1] != 0.0 || (P->dim == 3 && x0[2] != 0.0))) {
    if ((st = fft_full<Real>(P, psi, -1)) != FSE_OK) return st;
    k_gs_shift<Real><<<blocks, 256, 0, P->stream>>>(static_cast<typename Cplx<Real>::T*>(psi), g,
                                                    make_double3(x0[0], x0[1], P->dim == 3 ? x0[2] : 0.0),
                                                    1.0 / (double)N);
    if ((st = launched(P, cudaGetLastError(), "shift")) != FSE_OK) return st;
    if ((st = fft_full<Real>(P, psi, +1)) != FSE_OK) return st;
  }
  if (kv && (kv[0] != 0.0 || kv[1] != 0.0 || (P->dim == 3 && kv[2] != 0.0))) {
    k_gs_kick<Real><<<blocks, 256, 0, P->stream>>>(static_cast<typename Cplx<Real>::T*>(psi), g,
                                                   make_double3(kv[0], kv[1], P->dim == 3 ? kv[2] : 0.0));
    if ((st = launched(P, cudaGetLastError(), "kick")) != FSE_OK) return st;
  }
  return FSE_OK;
}

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

// workspace: 10 complex fields, 3 real fields, reduction partials and results
struct GsLayout {
  size_t cplx[10], real[3], part, out, sc, total;
};
GsLayout gs_layout(const fse_plan* P) {
  GsLayout L;
  const size_t N = (size_t)P->nx * P->ny * P->nz;
  size_t off = 0;
  for (int i = 0; i < 10; ++i) {
    L.cplx[i] = off;
    off = al256(off + N * P->csize);
  }
  for (int i = 0; i < 3; ++i) {
    L.real[i] = off;
    off = al256(off + N * P->rsize);
  }
  L.part = off;
  off = al256(off + sizeof(double) * 4 * kGsBlocks);
  L.out = off;
  off = al256(off + sizeof(double) * 8);
  L.sc = off;
  off = al256(off + sizeof(double) * SC_SIZE);
  L.total = off;
  return L;
}

template <typename Real>
struct Gs {
  typedef typename Cplx<Real>::T C;
  fse_plan* P;
  cudaStream_t st;
  long long N;
  int blocks;
  GsGrid g;
  C *phin, *r, *rh, *p, *v, *s, *t, *t1, *t2, *t3;
  Real *W, *pk, *Phi;
  double *part, *out, *sc;
  double omega;

  fse_status chk(const char* w) { return launched(P, cudaGetLastError(), w); }

  fse_status copy(C* dst, const C* src) {
    cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)N * sizeof(C), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? FSE_OK : cuda_fail(P, e, "ground state copy");
  }
  fse_status lincomb(C* o, const C* A, std::complex<double> a, const C* B = nullptr,
                     std::complex<double> b = 0.0, const C* Cc = nullptr, std::complex<double> c = 0.0) {
    k_gs_lincomb<Real><<<blocks, 256, 0, st>>>(o, A, make_double2(a.real(), a.imag()), B,
                                               make_double2(b.real(), b.imag()), Cc, make_double2(c.real(), c.imag()), N);
    return chk("ground state update");
  }
  // two complex inner products sum conj(a) b, read back to the host (synchronises)
  fse_status dot2(const C* a1, const C* b1, const C* a2, const C* b2, std::complex<double>& d1,
                  std::complex<double>& d2) {
    k_gs_dot2<Real><<<blocks, 256, 0, st>>>(a1, b1, a2, b2, N, part);
    fse_status s0 = chk("ground state reduction");
    if (s0 != FSE_OK) return s0;
    k_gs_final<<<4, 256, 0, st>>>(part, blocks, 0, out);
    if ((s0 = chk("ground state reduction")) != FSE_OK) return s0;
    double h[4];
    cudaError_t e = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(P, e, "ground state reduction");
    d1 = std::complex<double>(h[0], h[1]);
    d2 = std::complex<double>(h[2], h[3]);
    return FSE_OK;
  }
  // the same two inner products into out[0..3], left on the device
  fse_status dot2_dev(const C* a1, const C* b1, const C* a2, const C* b2) {
    k_gs_dot2<Real><<<blocks, 256, 0, st>>>(a1, b1, a2, b2, N, part);
    fse_status s0 = chk("ground state reduction");
    if (s0 != FSE_OK) return s0;
    k_gs_final<<<4, 256, 0, st>>>(part, blocks, 0, out);
    return chk("ground state reduction");
  }
  template <int MODE> fse_status update(C* o, const C* A, const C* Cc) {
    k_gs_update<Real, MODE><<<blocks, 256, 0, st>>>(o, A, Cc, sc, N);
    return chk("ground state update");
  }
  fse_status maxdiff(const C* a, const C* b, double& m) {
    k_gs_maxdiff<Real><<<blocks, 256, 0, st>>>(a, b, N, part);
    fse_status s0 = chk("ground state reduction");
    if (s0 != FSE_OK) return s0;
    k_gs_final<<<1, 256, 0, st>>>(part, blocks, 1, out);
    if ((s0 = chk("ground state reduction")) != FSE_OK) return s0;
    cudaError_t e = cudaMemcpyAsync(&m, out, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? FSE_OK : cuda_fail(P, e, "ground state reduction");
  }
  // y = (I + P_Delta A_TF) u   (u and y distinct; t1..t3 scratch)
  fse_status matvec(const C* u, C* y) {
    fse_status s0;
    if ((s0 = copy(t1, u)) != FSE_OK) return s0;
    if (omega != 0.0) {
      if ((s0 = fft_full<Real>(P, t1, -1)) != FSE_OK) return s0;
      const double inv_n = 1.0 / (double)N;
      k_gs_ik<Real><<<blocks, 256, 0, st>>>(t1, t2, g, 0, inv_n);
      if ((s0 = chk("ground state derivative")) != FSE_OK) return s0;
      k_gs_ik<Real><<<blocks, 256, 0, st>>>(t1, t3, g, 1, inv_n);
      if ((s0 = chk("ground state derivative")) != FSE_OK) return s0;
      if ((s0 = fft_full<Real>(P, t2, +1)) != FSE_OK) return s0;
      if ((s0 = fft_full<Real>(P, t3, +1)) != FSE_OK) return s0;
    }
    k_gs_atf<Real><<<blocks, 256, 0, st>>>(u, t2, t3, W, t1, g, omega);
    if ((s0 = chk("ground state operator")) != FSE_OK) return s0;
    if ((s0 = precond(t1)) != FSE_OK) return s0;
    return lincomb(y, u, 1.0, t1, 1.0);
  }
  // w <- P_Delta w (in place)
  fse_status precond(C* w) {
    fse_status s0;
    if ((s0 = fft_full<Real>(P, w, -1)) != FSE_OK) return s0;
    k_gs_scale_real<Real><<<blocks, 256, 0, st>>>(w, pk, N);
    if ((s0 = chk("ground state preconditioner")) != FSE_OK) return s0;
    return fft_full<Real>(P, w, +1);
  }
};

template <typename Real>
fse_status ground_state(fse_plan* P, void* psi_v, void* ws, const fse_gs_opts& o, fse_gs_info* info) {
  typedef typename Cplx<Real>::T C;
  const GsLayout L = gs_layout(P);
  char* base = static_cast<char*>(ws);
  Gs<Real> G;
  G.P = P;
  G.st = P->stream;
  G.N = (long long)P->nx * P->ny * P->nz;
  G.blocks = (int)std::min<long long>(kGsBlocks, (G.N + 255) / 256);
  G.g = gs_grid(P);
  C** cp[10] = {&G.phin, &G.r, &G.rh, &G.p, &G.v, &G.s, &G.t, &G.t1, &G.t2, &G.t3};
  for (int i = 0; i < 10; ++i) *cp[i] = reinterpret_cast<C*>(base + L.cplx[i]);
  G.W = reinterpret_cast<Real*>(base + L.real[0]);
  G.pk = reinterpret_cast<Real*>(base + L.real[1]);
  G.Phi = reinterpret_cast<Real*>(base + L.real[2]);
  G.part = reinterpret_cast<double*>(base + L.part);
  G.out = reinterpret_cast<double*>(base + L.out);
  G.sc = reinterpret_cast<double*>(base + L.sc);
  G.omega = P->p.omega;
  C* x = static_cast<C*>(psi_v);
  const double hd = P->h[0] * P->h[1] * (P->dim == 3 ? P->h[2] : 1.0);
  const bool nl = has_nonlocal(P);
  fse_status st;

  k_gs_precond_table<Real><<<G.blocks, 256, 0, G.st>>>(G.pk, G.g, 1.0 / o.dt, P->p.s, P->p.m * P->p.m,
                                                       1.0 / (double)G.N);
  if ((st = G.chk("ground state preconditioner")) != FSE_OK) return st;
  std::complex<double> m2, dummy;
  if ((st = G.dot2(x, x, x, x, m2, dummy)) != FSE_OK) return st;
  if (!(m2.real() > 0.0)) return fail(P, FSE_ERR_INVALID, "ground state: zero initial field");
  if ((st = G.lincomb(x, x, 1.0 / std::sqrt(hd * m2.real()))) != FSE_OK) return st;

  const double3 g2 = make_double3(0.5 * P->p.gamma[0] * P->p.gamma[0], 0.5 * P->p.gamma[1] * P->p.gamma[1],
                                  P->dim == 3 ? 0.5 * P->p.gamma[2] * P->p.gamma[2] : 0.0);
  const double3 lk = make_double3(P->p.lat_k[0], P->p.lat_k[1], P->dim == 3 ? P->p.lat_k[2] : 0.0);
  // one BiCGStab iteration: every operand and coefficient is on the device, so
  // the launches are captured once per call as a CUDA graph and replayed
  auto iteration = [&]() -> fse_status {
    fse_status s0;
    if ((s0 = G.template update<GS_P>(G.p, G.r, G.v)) != FSE_OK) return s0;
    if ((s0 = G.matvec(G.p, G.v)) != FSE_OK) return s0;
    if ((s0 = G.dot2_dev(G.rh, G.v, G.rh, G.v)) != FSE_OK) return s0;
    k_gs_sc_alpha<<<1, 1, 0, G.st>>>(G.sc, G.out);
    if ((s0 = G.chk("ground state scalars")) != FSE_OK) return s0;
    if ((s0 = G.template update<GS_S>(G.s, G.r, G.v)) != FSE_OK) return s0;
    if ((s0 = G.matvec(G.s, G.t)) != FSE_OK) return s0;
    if ((s0 = G.dot2_dev(G.t, G.s, G.t, G.t)) != FSE_OK) return s0;
    k_gs_sc_omega<<<1, 1, 0, G.st>>>(G.sc, G.out);
    if ((s0 = G.chk("ground state scalars")) != FSE_OK) return s0;
    if ((s0 = G.template update<GS_X>(x, G.p, G.s)) != FSE_OK) return s0;
    if ((s0 = G.template update<GS_R>(G.r, G.s, G.t)) != FSE_OK) return s0;
    if ((s0 = G.dot2_dev(G.rh, G.r, G.r, G.r)) != FSE_OK) return s0;
    k_gs_sc_rho<<<1, 1, 0, G.st>>>(G.sc, G.out);
    return G.chk("ground state scalars");
  };
  cudaGraphExec_t iter_exec = nullptr;
  long long iter_launches = 0;
  if (o.max_inner > 0 && o.max_outer > 0) {
    // capture on the solve's own stream; if capture is refused (e.g. the
    // thread is capturing another stream) the iterations are launched directly
    const long long l0 = P->launches;
    if (cudaStreamBeginCapture(G.st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const fse_status sq = iteration();
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(G.st, &graph);
      if (sq != FSE_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return sq != FSE_OK ? sq : cuda_fail(P, e, "ground state capture");
      }
      const cudaError_t ei = cudaGraphInstantiate(&iter_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) return cuda_fail(P, ei, "ground state capture");
      iter_launches = P->launches - l0;
      P->launches = l0;
    } else {
      cudaGetLastError();
    }
  }
  struct ExecGuard {
    cudaGraphExec_t* e;
    ~ExecGuard() {
      if (*e) cudaGraphExecDestroy(*e);
    }
  } exec_guard{&iter_exec};
  int outer = 0;
  long long inner = 0;
  double change = 0.0, res = 0.0;
  while (outer < o.max_outer) {
    if ((st = G.copy(G.phin, x)) != FSE_OK) return st;
    if (nl && (st = nonlocal_field(P, x, nullptr, G.Phi)) != FSE_OK) return st;
    k_gs_potential<Real><<<G.blocks, 256, 0, G.st>>>(x, nl ? G.Phi : nullptr, G.W, G.g, g2, P->p.beta, P->p.lambda,
                                                      P->p.lat_amp, lk);
    if ((st = G.chk("ground state potential")) != FSE_OK) return st;
    // b = P_Delta phi^n / dt (held in s), r = b - M x, rh = r
    if ((st = G.lincomb(G.s, G.phin, 1.0 / o.dt)) != FSE_OK) return st;
    if ((st = G.precond(G.s)) != FSE_OK) return st;
    if ((st = G.matvec(x, G.v)) != FSE_OK) return st;
    if ((st = G.lincomb(G.r, G.s, 1.0, G.v, -1.0)) != FSE_OK) return st;
    if ((st = G.copy(G.rh, G.r)) != FSE_OK) return st;
    if ((st = G.dot2_dev(G.s, G.s, G.r, G.r)) != FSE_OK) return st;
    k_gs_sc_init<<<1, 1, 0, G.st>>>(G.sc, G.out, o.inner_tol);
    if ((st = G.chk("ground state scalars")) != FSE_OK) return st;
    // Iterations are queued one ahead of the host: after queueing iteration
    // it, the host waits for the scalars of iteration it - 1 (copied to pinned
    // host memory behind it) and stops once they say done, so the GPU never
    // idles on a read-back; the extra iteration then changes nothing.
    double* hs = P->gs_host;
    int it = 0;
    for (; it < o.max_inner; ++it) {
      if (iter_exec) {
        cudaError_t e = cudaGraphLaunch(iter_exec, G.st);
        if (e != cudaSuccess) return cuda_fail(P, e, "ground state iteration");
        P->launches += iter_launches;
      } else if ((st = iteration()) != FSE_OK) {
        return st;
      }
      cudaError_t e = cudaMemcpyAsync(hs + (it & 1) * SC_SIZE, G.sc, sizeof(double) * SC_SIZE,
                                      cudaMemcpyDeviceToHost, G.st);
      if (e == cudaSuccess) e = cudaEventRecord(P->gs_ev[it & 1], G.st);
      if (e != cudaSuccess) return cuda_fail(P, e, "ground state scalars");
      if (it >= 1) {
        if ((e = cudaEventSynchronize(P->gs_ev[(it - 1) & 1])) != cudaSuccess)
          return cuda_fail(P, e, "ground state scalars");
        if (hs[((it - 1) & 1) * SC_SIZE + SC_DONE] != 0.0) break;
      }
    }
    // the scalars after the last queued iteration (iteration count, residual)
    {
      cudaError_t e = cudaMemcpyAsync(hs, G.sc, sizeof(double) * SC_SIZE, cudaMemcpyDeviceToHost, G.st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(G.st);
      if (e != cudaSuccess) return cuda_fail(P, e, "ground state scalars");
    }
    it = (int)hs[SC_IT];
    res = hs[SC_RES];
    inner += it;
    // phi^{n+1} = phi^(1) / ||phi^(1)||
    if ((st = G.dot2(x, x, x, x, m2, dummy)) != FSE_OK) return st;
    if (!(m2.real() > 0.0)) return fail(P, FSE_ERR_NONFINITE, "ground state: zero field");
    if ((st = G.lincomb(x, x, 1.0 / std::sqrt(hd * m2.real()))) != FSE_OK) return st;
    if ((st = G.maxdiff(x, G.phin, change)) != FSE_OK) return st;
    change /= o.dt;
    ++outer;
    if (!std::isfinite(change)) return fail(P, FSE_ERR_NONFINITE, "ground state: non-finite iterate");
    if (change <= o.tol) break;
  }
  if (info) {
    info->outer = outer;
    info->inner = (int)std::min<long long>(inner, 0x7fffffff);
    info->change = change;
    info->residual = res;
  }
  return FSE_OK;
}

}  // namespace
}  // namespace fse

using namespace fse;

extern "C" fse_status fse_ground_state_workspace(fse_plan_t P, size_t* bytes) {
  if (!P || !bytes) return FSE_ERR_INVALID;
  *bytes = gs_layout(P).total;
  return FSE_OK;
}

extern "C" fse_status fse_ground_state(fse_plan_t P, void* psi, void* workspace, size_t bytes,
                                       const fse_gs_opts* opts, fse_gs_info* info) {
  if (!P || !psi || !workspace || !opts) return FSE_ERR_INVALID;
  if (!P->ws || !P->precomputed) return fail(P, FSE_ERR_INVALID, "fse_kernel_precompute has not run");
  if (reinterpret_cast<uintptr_t>(psi) % P->csize != 0 || reinterpret_cast<uintptr_t>(workspace) % 256 != 0)
    return fail(P, FSE_ERR_INVALID, "misaligned buffer");
  if (bytes < gs_layout(P).total) return fail(P, FSE_ERR_NOMEM, "ground-state workspace too small");
  if (!(opts->dt > 0.0) || opts->max_outer < 0 || opts->max_inner < 0 || !(opts->tol >= 0.0) ||
      !(opts->inner_tol >= 0.0))
    return fail(P, FSE_ERR_INVALID, "ground state: bad options");
  if (!P->gs_host) {
    void* h = nullptr;
    cudaError_t e = cudaMallocHost(&h, sizeof(double) * 2 * SC_SIZE);
    if (e != cudaSuccess) return cuda_fail(P, e, "ground state host scalars");
    P->gs_host = static_cast<double*>(h);
  }
  for (auto& ev : P->gs_ev) {
    if (ev) continue;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(P, e, "ground state events");
  }
  if (!P->gs_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&P->gs_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->gs_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->gs_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(P, e, "ground state stream");
  }
  // the solve runs on a stream of the plan's own (capturable, unlike the
  // legacy default stream), after and before the caller's stream
  cudaStream_t user = P->stream;
  cudaError_t e = cudaEventRecord(P->gs_fork, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->gs_stream, P->gs_fork, 0);
  if (e != cudaSuccess) return cuda_fail(P, e, "ground state fork");
  P->stream = P->gs_stream;
  const fse_status st = P->prec == FSE_F32 ? ground_state<float>(P, psi, workspace, *opts, info)
                                           : ground_state<double>(P, psi, workspace, *opts, info);
  P->stream = user;
  e = cudaEventRecord(P->gs_join, P->gs_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, P->gs_join, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(user);
  if (st == FSE_OK && e != cudaSuccess) return cuda_fail(P, e, "ground state join");
  return st;
}

extern "C" fse_status fse_shift_kick(fse_plan_t P, void* psi, const double* x0, const double* k) {
  if (!P || !psi) return FSE_ERR_INVALID;
  if (!P->ws || !P->precomputed) return fail(P, FSE_ERR_INVALID, "fse_kernel_precompute has not run");
  if (reinterpret_cast<uintptr_t>(psi) % P->csize != 0) return fail(P, FSE_ERR_INVALID, "misaligned buffer");
  for (int j = 0; j < P->dim; ++j)
    if ((x0 && !std::isfinite(x0[j])) || (k && !std::isfinite(k[j])))
      return fail(P, FSE_ERR_INVALID, "shift or kick not finite");
  return P->prec == FSE_F32 ? shift_kick<float>(P, psi, x0, k) : shift_kick<double>(P, psi, x0, k);
}

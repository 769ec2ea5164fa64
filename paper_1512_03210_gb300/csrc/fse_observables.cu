// fse_observables.cu -- float64 observables on the device (Section 1, Eqs. mass, energy;
// Section 4.1, Eqs. AME, CoM, ConWidth).
//
// phi lives in the rotating Lagrangian frame at time t. The energy is that of
// Eq. SFSE (rotation term included); the kinetic term, the interactions and
// L_z are invariant under the frame rotation and V(A(t) x~) = W(x~, t), so
// every term is evaluated in x~. Centre of mass and widths are returned in
// the frame of Eq. SFSE, x = A(t) x~.
//
// Reductions: each block accumulates in float64 and writes one partial per
// slot; one block per slot then sums the partials in a fixed order, so the
// result does not depend on scheduling.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "fse.h"
#include "fse_internal.h"
#include "fse_passes.cuh"

namespace fse {

enum {
  SL_MASS = 0, SL_RHO2, SL_WRHO, SL_X, SL_Y, SL_Z, SL_XX, SL_YY, SL_ZZ, SL_XY,
  SL_KIN, SL_LZY, SL_LZX, SL_NON, NSLOT
};
constexpr int kPartStride = 65536;  // partials per slot (>= x-pass blocks of the largest grid)
constexpr int kRedBlocks = 1024;

struct ObsArgs {
  int nx, ny, nz;
  double lo[3], h[3];
  double g2[3];  // gamma_v^2 / 2
  double c, s;   // cos, sin of Omega t
  double lat_amp, lat_k[3];  // optical lattice lat_amp sum_v sin^2(lat_k[v] x_v)
};

template <typename Real>
__global__ void __launch_bounds__(256) k_obs_phys(const typename Cplx<Real>::T* __restrict__ psi, ObsArgs o,
                                                  double* part) {
  __shared__ double red[32];
  const long long N = (long long)o.nx * o.ny * o.nz;
  double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % o.nx);
    const long long r = i / o.nx;
    const int iy = (int)(r % o.ny), iz = (int)(r / o.ny);
    const double x = o.lo[0] + o.h[0] * ix, y = o.lo[1] + o.h[1] * iy, z = o.lo[2] + o.h[2] * iz;
    const typename Cplx<Real>::T u = psi[i];
    const double rho = (double)u.x * u.x + (double)u.y * u.y;
    const double X = o.c * x + o.s * y, Y = -o.s * x + o.c * y;
    double W = o.g2[0] * X * X + o.g2[1] * Y * Y + o.g2[2] * z * z;
    if (o.lat_amp != 0.0) {
      const double sx = sin(o.lat_k[0] * X), sy = sin(o.lat_k[1] * Y), sz = sin(o.lat_k[2] * z);
      W += o.lat_amp * (sx * sx + sy * sy + sz * sz);
    }
    acc[0] += rho;
    acc[1] += rho * rho;
    acc[2] += W * rho;
    acc[3] += x * rho;
    acc[4] += y * rho;
    acc[5] += z * rho;
    acc[6] += x * x * rho;
    acc[7] += y * y * rho;
    acc[8] += z * z * rho;
    acc[9] += x * y * rho;
  }
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const double v = block_sum(acc[k], red);
    if (threadIdx.x == 0) part[k * kPartStride + blockIdx.x] = v;
  }
}

// sum over the spectrum of (|k|^2 + m^2)^s |phi^_k|^2 (unnormalised DFT)
template <typename Real>
__global__ void __launch_bounds__(256) k_obs_kin(const typename Cplx<Real>::T* __restrict__ sp, ObsArgs o,
                                                 double dkx, double dky, double dkz, double s, double m2,
                                                 double* part) {
  __shared__ double red[32];
  const long long N = (long long)o.nx * o.ny * o.nz;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % o.nx);
    const long long r = i / o.nx;
    const int iy = (int)(r % o.ny), iz = (int)(r / o.ny);
    const Real kx = Real(dkx) * Real(wrap_index(ix, o.nx));
    const Real ky = Real(dky) * Real(wrap_index(iy, o.ny));
    const Real kz = o.nz > 1 ? Real(dkz) * Real(wrap_index(iz, o.nz)) : Real(0);
    const Real k2 = kx * kx + ky * ky + kz * kz + Real(m2);
    const typename Cplx<Real>::T u = sp[i];
    acc += (double)pow(k2, Real(s)) * ((double)u.x * u.x + (double)u.y * u.y);
  }
  const double v = block_sum(acc, red);
  if (threadIdx.x == 0) part[SL_KIN * kPartStride + blockIdx.x] = v;
}

// d = i k_axis phi^ / N (odd factor zero at the Nyquist index)
template <typename Real>
__global__ void __launch_bounds__(256) k_mul_ik(const typename Cplx<Real>::T* __restrict__ sp,
                                                typename Cplx<Real>::T* __restrict__ d, ObsArgs o, int axis,
                                                double dk, double inv_n) {
  const long long N = (long long)o.nx * o.ny * o.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % o.nx);
    const int iy = (int)((i / o.nx) % o.ny);
    const int idx = axis == 0 ? ix : iy;
    const int n = axis == 0 ? o.nx : o.ny;
    const Real k = (2 * idx == n) ? Real(0) : Real(dk * inv_n) * Real(wrap_index(idx, n));
    const typename Cplx<Real>::T u = sp[i];
    d[i] = mk(-k * u.y, k * u.x);
  }
}

// sum of c(x) Im(conj(psi) d): with c = x the y-derivative term, with c = -y the x-derivative term of
// <psi, -i (x d_y - y d_x) psi>
template <typename Real>
__global__ void __launch_bounds__(256) k_obs_lz(const typename Cplx<Real>::T* __restrict__ psi,
                                                const typename Cplx<Real>::T* __restrict__ d, ObsArgs o, int axis,
                                                int slot, double* part) {
  __shared__ double red[32];
  const long long N = (long long)o.nx * o.ny * o.nz;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % o.nx);
    const int iy = (int)((i / o.nx) % o.ny);
    const double c = axis == 1 ? (o.lo[0] + o.h[0] * ix) : -(o.lo[1] + o.h[1] * iy);
    const typename Cplx<Real>::T u = psi[i], v = d[i];
    acc += c * ((double)u.x * v.y - (double)u.y * v.x);
  }
  const double v = block_sum(acc, red);
  if (threadIdx.x == 0) part[slot * kPartStride + blockIdx.x] = v;
}

struct SlotCounts {
  int n[NSLOT];
};

__global__ void __launch_bounds__(256) k_sum_slots(const double* part, SlotCounts cnt, double* out) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < cnt.n[s]; i += blockDim.x) acc += part[s * kPartStride + i];
  const double v = block_sum(acc, red);
  if (threadIdx.x == 0) out[s] = v;
}

// ---------------------------------------------------------------------------
// Optional float64 renormalisation of the float32 path (not part of the
// paper's scheme): hold the mass at its value at the start of each fse_step
// call. Pass E (or XI) writes per-tile partial masses, k_renorm turns them
// into sqrt(N0 / N), pass A multiplies u2 by it.
// ---------------------------------------------------------------------------
constexpr int kRenormSlot = 15;
constexpr long long kScalarBase = 16LL * kPartStride;

template <typename Real>
__global__ void __launch_bounds__(256) k_sumsq(const typename Cplx<Real>::T* __restrict__ psi, long long N,
                                               double* part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const typename Cplx<Real>::T u = psi[i];
    acc += (double)u.x * u.x + (double)u.y * u.y;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(256) k_renorm(const double* part, int count, double* scal, int init) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    if (init) scal[0] = acc;
    else scal[1] = acc > 0.0 ? sqrt(scal[0] / acc) : 1.0;
  }
}

double* renorm_part(fse_plan* P) {
  return reinterpret_cast<double*>(P->ws_ptr(P->off_red)) + kRenormSlot * kPartStride;
}
const double* renorm_scale(fse_plan* P) {
  return reinterpret_cast<double*>(P->ws_ptr(P->off_red)) + kScalarBase + 1;
}

fse_status renorm_begin(fse_plan* P, const void* psi) {
  const long long N = (long long)P->nx * P->ny * P->nz;
  const int blocks = (int)std::min<long long>(kRedBlocks, (N + 255) / 256);
  double* scal = reinterpret_cast<double*>(P->ws_ptr(P->off_red)) + kScalarBase;
  cudaEvent_t ev = prof_begin(P);
  if (P->prec == FSE_F32)
    k_sumsq<float><<<blocks, 256, 0, P->stream>>>(reinterpret_cast<const float2*>(psi), N, renorm_part(P));
  else
    k_sumsq<double><<<blocks, 256, 0, P->stream>>>(reinterpret_cast<const double2*>(psi), N, renorm_part(P));
  prof_end(P, FSE_PASS_OTHER, ev);
  fse_status st = launched(P, cudaGetLastError(), "renormalisation");
  if (st != FSE_OK) return st;
  k_renorm<<<1, 256, 0, P->stream>>>(renorm_part(P), blocks, scal, 1);
  return launched(P, cudaGetLastError(), "renormalisation");
}

fse_status renorm_step(fse_plan* P, int count) {
  if (count > kPartStride) return fail(P, FSE_ERR_UNSUPPORTED, "renormalisation: grid too large");
  double* scal = reinterpret_cast<double*>(P->ws_ptr(P->off_red)) + kScalarBase;
  cudaEvent_t ev = prof_begin(P);
  k_renorm<<<1, 256, 0, P->stream>>>(renorm_part(P), count, scal, 0);
  prof_end(P, FSE_PASS_OTHER, ev);
  return launched(P, cudaGetLastError(), "renormalisation");
}

template <typename Real>
fse_status fft_full(fse_plan* P, void* buf, int dir) {
  MulArgs m;
  std::memset(&m, 0, sizeof(m));
  XArgs xa = x_args(P, buf, nullptr);
  fse_status st;
  ColArgs ay{buf, (long long)P->nx * P->ny, P->nx, P->nz, P->nx, P->ny, P->ny, tiles(P, P->ny, P->nx)};
  ColArgs az{buf, P->nx, (long long)P->nx * P->ny, P->ny, P->nx, P->nz, P->nz, tiles(P, P->nz, P->nx)};
  if (dir < 0) {
    if ((st = xpass(P, XP_FWD, xa)) != FSE_OK) return st;
    if ((st = col(P, FSE_PASS_OTHER, P->ny, COL_FWD, ay, m)) != FSE_OK) return st;
    if (P->dim == 3 && (st = col(P, FSE_PASS_OTHER, P->nz, COL_FWD, az, m)) != FSE_OK) return st;
    return FSE_OK;
  }
  if (P->dim == 3 && (st = col(P, FSE_PASS_OTHER, P->nz, COL_INV, az, m)) != FSE_OK) return st;
  if ((st = col(P, FSE_PASS_OTHER, P->ny, COL_INV, ay, m)) != FSE_OK) return st;
  return xpass(P, XP_INV, xa);
}

template fse_status fft_full<float>(fse_plan*, void*, int);
template fse_status fft_full<double>(fse_plan*, void*, int);

fse_status nonlocal_field(fse_plan* P, const void* psi, const double* mdir, void* phi) {
  void* tmp = P->ws_ptr(P->off_tmp);
  void* spec = P->ws_ptr(P->off_spec);
  cudaError_t e;
  fse_status st;
  if ((e = cudaMemcpyAsync(tmp, psi, P->psi_bytes, cudaMemcpyDeviceToDevice, P->stream)) != cudaSuccess)
    return cuda_fail(P, e, "nonlocal field copy");
  XArgs xa = x_args(P, tmp, spec);
  if ((st = xpass(P, XP_FWD, xa)) != FSE_OK) return st;
  if ((st = xpass(P, XP_E, xa)) != FSE_OK) return st;  // S = R2C of nx^2 rho
  const double* md = mdir ? mdir : P->p.dip_n;
  if ((st = nonlocal_yz(P, spec, 0.0, 0.0, false, md, 1.0 / ((double)P->nx * P->nx))) != FSE_OK) return st;
  XArgs xr = x_args(P, const_cast<void*>(psi), spec);
  xr.out = phi;
  return xpass(P, XP_R, xr);
}

template <typename Real>
fse_status observables(fse_plan* P, const void* psi_in, double t, const double* gam, fse_obs* out) {
  typedef typename Cplx<Real>::T C;
  const C* psi = reinterpret_cast<const C*>(psi_in);
  C* tmp = reinterpret_cast<C*>(P->ws_ptr(P->off_tmp));
  C* spec = reinterpret_cast<C*>(P->ws_ptr(P->off_spec));
  double* part = reinterpret_cast<double*>(P->ws_ptr(P->off_red));
  double* sums = part + NSLOT * kPartStride;
  cudaError_t e;
  fse_status st;
  SlotCounts cnt;
  for (int k = 0; k < NSLOT; ++k) cnt.n[k] = 0;

  ObsArgs o;
  o.nx = P->nx;
  o.ny = P->ny;
  o.nz = P->nz;
  for (int j = 0; j < 3; ++j) {
    o.lo[j] = j < P->dim ? P->p.lo[j] : 0.0;
    o.h[j] = P->h[j];
    const double g = j < P->dim ? (gam ? gam[j] : P->p.gamma[j]) : 0.0;
    o.g2[j] = 0.5 * g * g;
    o.lat_k[j] = j < P->dim ? P->p.lat_k[j] : 0.0;
  }
  o.c = std::cos(P->p.omega * t);
  o.s = std::sin(P->p.omega * t);
  o.lat_amp = P->p.lat_amp;
  const long long N = (long long)P->nx * P->ny * P->nz;
  const int blocks = (int)std::min<long long>(kRedBlocks, (N + 255) / 256);

  // nonlocal energy density: Phi = U~(., t) * rho (un-integrated kernel at time t)
  if (has_nonlocal(P)) {
    if ((e = cudaMemcpyAsync(tmp, psi, P->psi_bytes, cudaMemcpyDeviceToDevice, P->stream)) != cudaSuccess)
      return cuda_fail(P, e, "observables copy");
    XArgs xa = x_args(P, tmp, spec);
    if ((st = xpass(P, XP_FWD, xa)) != FSE_OK) return st;
    if ((st = xpass(P, XP_E, xa)) != FSE_OK) return st;  // tmp = nx psi, S = R2C of nx^2 rho
    double mdir[3] = {0, 0, 0};
    if (P->p.kernel == FSE_KERNEL_DDI3D || P->p.kernel == FSE_KERNEL_DDI2D) {
      // m(t) = A(t)^T n
      const double n1 = P->p.dip_n[0], n2 = P->p.dip_n[1], n3 = P->p.dip_n[2];
      mdir[0] = o.c * n1 - o.s * n2;
      mdir[1] = o.s * n1 + o.c * n2;
      mdir[2] = n3;
    }
    if ((st = nonlocal_yz(P, spec, t, t, false, mdir, 1.0 / ((double)P->nx * P->nx))) != FSE_OK) return st;
    XArgs xr = x_args(P, const_cast<C*>(psi), spec);
    xr.part = part + SL_NON * kPartStride;
    const int ncx = P->prec == FSE_F32 ? xpass_ncol<float>(P->nx) : xpass_ncol<double>(P->nx);
    if ((xr.nlines + ncx - 1) / ncx > kPartStride) return fail(P, FSE_ERR_UNSUPPORTED, "observables: grid too large");
    if ((st = xpass(P, XP_R, xr)) != FSE_OK) return st;
    cnt.n[SL_NON] = (xr.nlines + ncx - 1) / ncx;
  }

  cudaEvent_t ev = prof_begin(P);
  k_obs_phys<Real><<<blocks, 256, 0, P->stream>>>(psi, o, part);
  prof_end(P, FSE_PASS_OTHER, ev);
  if ((st = launched(P, cudaGetLastError(), "observables")) != FSE_OK) return st;
  for (int k = SL_MASS; k <= SL_XY; ++k) cnt.n[k] = blocks;

  // spectrum of psi
  if ((e = cudaMemcpyAsync(tmp, psi, P->psi_bytes, cudaMemcpyDeviceToDevice, P->stream)) != cudaSuccess)
    return cuda_fail(P, e, "observables copy");
  if ((st = fft_full<Real>(P, tmp, -1)) != FSE_OK) return st;
  const double dkx = 2 * kPi / (P->p.hi[0] - P->p.lo[0]);
  const double dky = 2 * kPi / (P->p.hi[1] - P->p.lo[1]);
  const double dkz = P->dim == 3 ? 2 * kPi / (P->p.hi[2] - P->p.lo[2]) : 0.0;
  ev = prof_begin(P);
  k_obs_kin<Real><<<blocks, 256, 0, P->stream>>>(tmp, o, dkx, dky, dkz, P->p.s, P->p.m * P->p.m, part);
  prof_end(P, FSE_PASS_OTHER, ev);
  if ((st = launched(P, cudaGetLastError(), "observables")) != FSE_OK) return st;
  cnt.n[SL_KIN] = blocks;

  // <L_z>: spectral derivatives d_y psi (paired with x) and d_x psi (paired with -y)
  for (int axis = 1; axis >= 0; --axis) {
    ev = prof_begin(P);
    k_mul_ik<Real><<<blocks, 256, 0, P->stream>>>(tmp, spec, o, axis, axis == 0 ? dkx : dky, 1.0 / (double)N);
    prof_end(P, FSE_PASS_OTHER, ev);
    if ((st = launched(P, cudaGetLastError(), "observables")) != FSE_OK) return st;
    if ((st = fft_full<Real>(P, spec, +1)) != FSE_OK) return st;
    const int slot = axis == 1 ? SL_LZY : SL_LZX;
    ev = prof_begin(P);
    k_obs_lz<Real><<<blocks, 256, 0, P->stream>>>(psi, spec, o, axis, slot, part);
    prof_end(P, FSE_PASS_OTHER, ev);
    if ((st = launched(P, cudaGetLastError(), "observables")) != FSE_OK) return st;
    cnt.n[slot] = blocks;
  }

  k_sum_slots<<<NSLOT, 256, 0, P->stream>>>(part, cnt, sums);
  if ((st = launched(P, cudaGetLastError(), "observables")) != FSE_OK) return st;
  double h[NSLOT];
  if ((e = cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, P->stream)) != cudaSuccess)
    return cuda_fail(P, e, "observables read");
  if ((e = cudaStreamSynchronize(P->stream)) != cudaSuccess) return cuda_fail(P, e, "observables sync");

  double hd = 1.0;
  for (int j = 0; j < P->dim; ++j) hd *= P->h[j];
  std::memset(out, 0, sizeof(*out));
  out->mass = hd * h[SL_MASS];
  out->e_kin = 0.5 * hd / (double)N * h[SL_KIN];
  out->e_pot = hd * h[SL_WRHO];
  out->e_int = 0.5 * P->p.beta * hd * h[SL_RHO2];
  out->e_non = has_nonlocal(P) ? 0.5 * P->p.lambda * hd * h[SL_NON] : 0.0;
  out->lz = hd * (h[SL_LZY] + h[SL_LZX]);
  out->e_rot = -P->p.omega * out->lz;
  out->energy = out->e_kin + out->e_pot + out->e_int + out->e_non + out->e_rot;
  const double xt[3] = {hd * h[SL_X], hd * h[SL_Y], hd * h[SL_Z]};
  out->xc[0] = o.c * xt[0] + o.s * xt[1];
  out->xc[1] = -o.s * xt[0] + o.c * xt[1];
  out->xc[2] = P->dim == 3 ? xt[2] : 0.0;
  const double Sxx = hd * h[SL_XX], Syy = hd * h[SL_YY], Sxy = hd * h[SL_XY];
  out->width[0] = o.c * o.c * Sxx + 2 * o.c * o.s * Sxy + o.s * o.s * Syy;
  out->width[1] = o.s * o.s * Sxx - 2 * o.c * o.s * Sxy + o.c * o.c * Syy;
  out->width[2] = P->dim == 3 ? hd * h[SL_ZZ] : 0.0;
  if (!std::isfinite(out->mass) || !std::isfinite(out->energy))
    return fail(P, FSE_ERR_NONFINITE, "observables: non-finite mass or energy");
  return FSE_OK;
}

}  // namespace fse

using namespace fse;

extern "C" fse_status fse_observables(fse_plan_t P, const void* psi, double t, const double* gamma, fse_obs* out) {
  if (!P || !psi || !out) return FSE_ERR_INVALID;
  if (!P->ws || !P->precomputed) return fail(P, FSE_ERR_INVALID, "fse_kernel_precompute has not run");
  return P->prec == FSE_F32 ? observables<float>(P, psi, t, gamma, out) : observables<double>(P, psi, t, gamma, out);
}

// fse_adjoint.cu -- transpose of one split step (gradients; the paper has no adjoint).
//
// Forward step (Section 4.2, Eqs. tssp1-tssp3): u1 = K psi_n, rho = |u1|^2,
// Theta = dt beta rho + lambda Kc rho + P(gamma), u2 = u1 exp(-i Theta),
// psi_{n+1} = K u2, with K the kinetic half step and Kc the padded
// convolution with the time-integrated kernel (real, even multiplier, so Kc
// is symmetric). Cotangents are g = dJ/dRe + i dJ/dIm. Pulling g back:
//   g_u2 = K^H g                                    (conjugate kinetic phase)
//   h    = exp(+i Theta) g_u2,  r = Im(conj(g_u2) u2) = Im(conj(h) u1)
//   g_u1 = h + 2 (dt beta r + lambda Kc r) u1
//   g_n  = K^H g_u1
//   dJ/dgamma_v = sum_x r dP/dgamma_v
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "fse.h"
#include "fse_internal.h"
#include "fse_passes.cuh"

namespace fse {

constexpr long long kAdjStride = 65536;  // partials per gradient slot
constexpr long long kAdjBase = 0;         // slots 0..2 of the reduction region (shared with observables)
constexpr long long kAdjOut = 16LL * 65536 + 8;  // scalar results

__global__ void __launch_bounds__(256) k_sum3(const double* part, int count, long long stride, double* out) {
  __shared__ double red[32];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[s * stride + i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[s] = acc;
}

// K or K^H on a physical field: fwd x, y/z passes with the phase, inv x.
fse_status kinetic_full(fse_plan* P, void* f, double sign) {
  XArgs xa = x_args(P, f, nullptr);
  fse_status st;
  if ((st = xpass(P, XP_FWD, xa)) != FSE_OK) return st;
  if ((st = kinetic_yz(P, f, sign, P->p.dt)) != FSE_OK) return st;
  return xpass(P, XP_INV, xa);
}

}  // namespace fse

using namespace fse;

extern "C" fse_status fse_step_adjoint(fse_plan_t P, const void* psi_n, void* g, double t_n,
                                       const double* gamma_n, double* dgamma_n) {
  if (!P || !psi_n || !g) return FSE_ERR_INVALID;
  if (!P->ws || !P->precomputed) return fail(P, FSE_ERR_INVALID, "fse_kernel_precompute has not run");
  if (P->p.renormalize) return fail(P, FSE_ERR_UNSUPPORTED, "adjoint of a renormalised plan");
  if (P->p.order != 2) return fail(P, FSE_ERR_UNSUPPORTED, "adjoint of the fourth-order composition");
  if (reinterpret_cast<uintptr_t>(g) % P->csize != 0 || reinterpret_cast<uintptr_t>(psi_n) % P->csize != 0)
    return fail(P, FSE_ERR_INVALID, "misaligned buffer");
  const double dt = P->p.dt, ta = t_n, tb = t_n + dt;
  void* u1 = P->ws_ptr(P->off_tmp);
  void* spec = P->ws_ptr(P->off_spec);
  double* red = reinterpret_cast<double*>(P->ws_ptr(P->off_red));
  const bool nl = has_nonlocal(P);
  fse_status st;
  cudaError_t e;

  // u1 = K psi_n and (with a nonlocal term) the x-half-spectrum of rho = |u1|^2
  if ((e = cudaMemcpyAsync(u1, psi_n, P->psi_bytes, cudaMemcpyDeviceToDevice, P->stream)) != cudaSuccess)
    return cuda_fail(P, e, "adjoint copy");
  XArgs xu = x_args(P, u1, nl ? spec : nullptr);
  if ((st = xpass(P, XP_FWD, xu)) != FSE_OK) return st;
  if ((st = kinetic_yz(P, u1, 1.0, dt)) != FSE_OK) return st;
  if (nl) {
    if ((st = xpass(P, XP_E, xu)) != FSE_OK) return st;
    if ((st = nonlocal_yz(P, spec, ta, tb, true, nullptr, 1.0)) != FSE_OK) return st;
  } else {
    if ((st = xpass(P, XP_INV, xu)) != FSE_OK) return st;
  }
  // g_u2 = K^H g
  if ((st = kinetic_full(P, g, -1.0)) != FSE_OK) return st;

  // pass 1: h, r (and its spectrum), trap-gradient partials
  double pc[4];
  trap_coefficients(P, ta, tb, gamma_n, pc);
  XArgs x1 = x_args(P, g, nl ? spec : nullptr);
  x1.aux = u1;
  x1.beta_dt = P->p.beta * dt;
  x1.lam = P->p.lambda;
  x1.pa = pc[0];
  x1.pb = pc[1];
  x1.pc = pc[2];
  x1.pe = pc[3];
  lattice_nodes(P, ta, tb, x1);
  x1.part = dgamma_n ? red + kAdjBase : nullptr;
  x1.part_stride = kAdjStride;
  {
    // dP/dgamma_v = gamma_v * int (A x~)_v^2 dtau: unit-frequency trap integrals times 2 gamma_v
    for (int v = 0; v < 3; ++v) {
      double one[3] = {0.0, 0.0, 0.0};
      one[v] = 1.0;
      double c[4] = {0, 0, 0, 0};
      if (v < P->dim) trap_coefficients(P, ta, tb, one, c);  // 1/2 int (A x~)_v^2 dtau
      const double gv = v < P->dim ? (gamma_n ? gamma_n[v] : P->p.gamma[v]) : 0.0;
      for (int k = 0; k < 4; ++k) x1.dp[4 * v + k] = 2.0 * gv * c[k];
    }
  }
  const int ncx = P->prec == FSE_F32 ? xpass_ncol<float>(P->nx) : xpass_ncol<double>(P->nx);
  const int xblocks = (x1.nlines + ncx - 1) / ncx;
  if (dgamma_n && xblocks > kAdjStride) return fail(P, FSE_ERR_UNSUPPORTED, "adjoint: grid too large");
  if ((st = xpass(P, XP_ADJ1, x1)) != FSE_OK) return st;
  // Kc r, then pass 2: g_u1 = h + 2 q u1
  if (nl && (st = nonlocal_yz(P, spec, ta, tb, true, nullptr, 1.0)) != FSE_OK) return st;
  XArgs x2 = x1;
  x2.part = nullptr;
  if ((st = xpass(P, XP_ADJ2, x2)) != FSE_OK) return st;
  // g_n = K^H g_u1
  if ((st = kinetic_full(P, g, -1.0)) != FSE_OK) return st;

  if (dgamma_n) {
    double* out = red + kAdjOut;
    k_sum3<<<3, 256, 0, P->stream>>>(red + kAdjBase, xblocks, kAdjStride, out);
    if ((st = launched(P, cudaGetLastError(), "adjoint gradient sum")) != FSE_OK) return st;
    double h3[3];
    if ((e = cudaMemcpyAsync(h3, out, sizeof(h3), cudaMemcpyDeviceToHost, P->stream)) != cudaSuccess)
      return cuda_fail(P, e, "adjoint read");
    if ((e = cudaStreamSynchronize(P->stream)) != cudaSuccess) return cuda_fail(P, e, "adjoint sync");
    for (int v = 0; v < P->dim; ++v) dgamma_n[v] = h3[v];
  }
  return FSE_OK;
}

// fse_precompute.cu -- once-per-plan float64 tables (twiddles, Gaussian-sum kernel transform).
//
// Kernel transform of the cube-truncated Coulomb kernel (Section 2):
//   C^(k) = sum_q w_q prod_j g_q(k_j) + I0 - I2 |k|^2 / (2d)          (Eqs. tensor, taylor)
//   g_q(k) = int_{-W}^{W} exp(-tau_q^2 y^2) cos(k y) dy               (Eq. tensor)
// with the zero-padded period 2W per axis (W the box width), k = pi p / W,
// p = 0..n. Wide Gaussians (tau W < 6) are integrated by composite
// Gauss-Legendre quadrature on [0, W]; for narrow ones the truncation at W
// changes the integral by less than erfc(6) ~ 2e-17 relative, so the
// full-line value sqrt(pi)/tau exp(-k^2/(4 tau^2)) is used.
#include <cuda_runtime.h>

#include "fse_fft.cuh"

namespace fse {

// tw[2m] = exp(-2 pi i m / L), m = 0..L-1, from float64 sincospi, and
// tw[2m+1] the rounded remainder (exact minus tw[2m]). For float tables the
// pair (c, s) is chosen among the float neighbours of the float64 values as
// the one with |c + i s| closest to 1.
__device__ __forceinline__ void round_pair(double c, double s, float2* out) {
  const float c0 = (float)c, s0 = (float)s;
  const float cc[2] = {c0, (double)c0 > c ? nextafterf(c0, -2.f) : nextafterf(c0, 2.f)};
  const float ss[2] = {s0, (double)s0 > s ? nextafterf(s0, -2.f) : nextafterf(s0, 2.f)};
  double best = 1e300;
  float2 r = make_float2(c0, s0);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const double n = (double)cc[i] * cc[i] + (double)ss[j] * ss[j] - 1.0;
      if (fabs(n) < best) {
        best = fabs(n);
        r = make_float2(cc[i], ss[j]);
      }
    }
  *out = r;
}
__device__ __forceinline__ void round_pair(double c, double s, double2* out) { *out = make_double2(c, s); }

// For float tables the broadcast copy for the packed column passes follows at
// tw + 2L: twb[2m] = (c, c, s, s) of tw[2m] and twb[2m+1] the same of tw[2m+1].
template <typename Real>
__global__ void k_twiddles(typename Cplx<Real>::T* tw, int L) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  double s, c;
  sincospi(-2.0 * (double)m / (double)L, &s, &c);
  round_pair(c, s, &tw[2 * m]);
  // rounded remainder of the exact twiddle (second term of the exact products)
  tw[2 * m + 1] = mk(Real(c - (double)tw[2 * m].x), Real(s - (double)tw[2 * m].y));
  if constexpr (sizeof(Real) == 4) {
    float4* twb = reinterpret_cast<float4*>(tw + 2 * L);
    const float2 w = tw[2 * m], l = tw[2 * m + 1];
    twb[2 * m] = make_float4(w.x, w.x, w.y, w.y);
    twb[2 * m + 1] = make_float4(l.x, l.x, l.y, l.y);
  }
}

// Kinetic multipliers exp(-i theta_k) (half step, theta = dt/4 (|k|^2+m^2)^s)
// and exp(-2 i theta_k) (two merged half steps) on the octant of mode
// magnitudes |p_j| = 0..n_j/2, layout [nz/2+1][ny/2+1][nx/2+1]: theta depends
// on |k| only, so every sign combination shares one entry (17 MB at 256^3,
// resident in L2). float64 arithmetic, rounded to the plan's precision with the
// norm-closest float pair (see round_pair).
template <typename Real>
__global__ void k_kin_table(typename Cplx<Real>::T* half, typename Cplx<Real>::T* full, int nx, int ny, int nz,
                            double dkx, double dky, double dkz, double s, double m2, double dt) {
  const int hx = nx / 2 + 1, hy = ny / 2 + 1, hz = nz > 1 ? nz / 2 + 1 : 1;
  const long long N = (long long)hx * hy * hz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(i % hx);
    const long long r = i / hx;
    const int iy = (int)(r % hy), iz = (int)(r / hy);
    const double kx = dkx * ix, ky = dky * iy, kz = dkz * iz;
    const double k2 = kx * kx + ky * ky + kz * kz + m2;
    const double th = 0.25 * dt * (k2 > 0.0 ? pow(k2, s) : 0.0);
    double sn, cs;
    sincos(th, &sn, &cs);
    round_pair(cs, -sn, &half[i]);
    sincos(2.0 * th, &sn, &cs);
    round_pair(cs, -sn, &full[i]);
  }
}

template <typename Real>
cudaError_t launch_kin_table(void* half, void* full, int nx, int ny, int nz, double dkx, double dky, double dkz,
                             double s, double m2, double dt, cudaStream_t st) {
  k_kin_table<Real><<<1024, 256, 0, st>>>(reinterpret_cast<typename Cplx<Real>::T*>(half),
                                          reinterpret_cast<typename Cplx<Real>::T*>(full), nx, ny, nz, dkx, dky,
                                          dkz, s, m2, dt);
  return cudaGetLastError();
}
template cudaError_t launch_kin_table<float>(void*, void*, int, int, int, double, double, double, double, double,
                                             double, cudaStream_t);
template cudaError_t launch_kin_table<double>(void*, void*, int, int, int, double, double, double, double, double,
                                              double, cudaStream_t);

// Quadrature nodes on [0, W]: npan panels of ngl Gauss-Legendre points.
// cs[y * (n+1) + p] = cos(k_p y_y); e[qw * ny + y] = w_y exp(-tau_q^2 y_y^2) for the wide q.
__global__ void k_gs_cos(double* cs, const double* glx, const double* glw, int ngl, int npan,
                         double W, int n, double* ynode, double* ywt) {
  const int ny = ngl * npan;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ny * (n + 1)) return;
  const int y = idx / (n + 1), p = idx % (n + 1);
  const int pan = y / ngl, g = y % ngl;
  const double hw = 0.5 * W / npan;
  const double yy = hw * (2 * pan + 1) + hw * glx[g];
  // k_p y = (pi p / W) y
  cs[idx] = cospi((double)p * yy / W);
  if (p == 0) {
    ynode[y] = yy;
    ywt[y] = hw * glw[g];
  }
}

__global__ void k_gs_table(double* g, const double* cs, const double* ynode, const double* ywt,
                           const double* tau, int Q, int n, int ny, double W) {
  const int q = blockIdx.x;
  const double t = tau[q];
  extern __shared__ double ew[];
  const bool wide = t * W < 6.0;
  if (wide) {
    for (int y = threadIdx.x; y < ny; y += blockDim.x) ew[y] = ywt[y] * exp(-(t * ynode[y]) * (t * ynode[y]));
    __syncthreads();
  }
  for (int p = threadIdx.x; p <= n; p += blockDim.x) {
    double v;
    if (wide) {
      double acc = 0.0;
      for (int y = 0; y < ny; ++y) acc = fma(ew[y], cs[(long long)y * (n + 1) + p], acc);
      v = 2.0 * acc;
    } else {
      const double k = 3.14159265358979323846 * (double)p / W;
      v = 1.7724538509055160273 / t * exp(-k * k / (4.0 * t * t));
    }
    g[(long long)q * (n + 1) + p] = v;
  }
}

// C^ on the octant [nz+1][ny+1][cx] (dim 3) or [ny+1][cx] (dim 2): x bins
// 0..nx, then zeros up to the row stride cx (a multiple of 4, so that every
// row starts 16-byte aligned).
template <typename Real>
__global__ void k_chat(Real* out, const double* w, const double* gx, const double* gy,
                       const double* gz, int Q, int nx, int ny, int nz, int cx, int dim, double dkx,
                       double dky, double dkz, double I0, double I2) {
  const int px = blockIdx.x * blockDim.x + threadIdx.x;
  const int py = blockIdx.y;
  const int pz = blockIdx.z;
  extern __shared__ double wyz[];   // w_q g_y[q][py] g_z[q][pz]
  for (int q = threadIdx.x; q < Q; q += blockDim.x) {
    double v = w[q] * gy[(long long)q * (ny + 1) + py];
    if (dim == 3) v *= gz[(long long)q * (nz + 1) + pz];
    wyz[q] = v;
  }
  __syncthreads();
  if (px >= cx) return;
  if (px > nx) {
    out[((long long)pz * (ny + 1) + py) * cx + px] = Real(0);
    return;
  }
  double acc = 0.0;
  for (int q = 0; q < Q; ++q) acc = fma(wyz[q], gx[(long long)q * (nx + 1) + px], acc);
  const double kx = dkx * px, ky = dky * py, kz = dim == 3 ? dkz * pz : 0.0;
  acc += I0 - I2 * (kx * kx + ky * ky + kz * kz) / (2.0 * dim);
  out[((long long)pz * (ny + 1) + py) * cx + px] = Real(acc);
}

template <typename Real>
cudaError_t launch_twiddles(void* tw, int L, cudaStream_t st) {
  k_twiddles<Real><<<(L + 127) / 128, 128, 0, st>>>(reinterpret_cast<typename Cplx<Real>::T*>(tw), L);
  return cudaGetLastError();
}

cudaError_t launch_gs_axis(double* g, double* cs, double* ynode, double* ywt, const double* tau,
                           int Q, const double* glx, const double* glw, int ngl, int npan, double W,
                           int n, cudaStream_t st) {
  const int ny = ngl * npan;
  const int tot = ny * (n + 1);
  k_gs_cos<<<(tot + 255) / 256, 256, 0, st>>>(cs, glx, glw, ngl, npan, W, n, ynode, ywt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(double) * (size_t)ny;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_gs_table, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_gs_table<<<Q, 128, smem, st>>>(g, cs, ynode, ywt, tau, Q, n, ny, W);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_chat(void* out, const double* w, const double* gx, const double* gy,
                        const double* gz, int Q, int nx, int ny, int nz, int cx, int dim, double dkx,
                        double dky, double dkz, double I0, double I2, cudaStream_t st) {
  dim3 grid((cx + 127) / 128, ny + 1, dim == 3 ? nz + 1 : 1);
  const size_t smem = sizeof(double) * (size_t)Q;
  k_chat<Real><<<grid, 128, smem, st>>>(reinterpret_cast<Real*>(out), w, gx, gy, gz, Q, nx, ny, nz,
                                        cx, dim, dkx, dky, dkz, I0, I2);
  return cudaGetLastError();
}

template cudaError_t launch_twiddles<float>(void*, int, cudaStream_t);
template cudaError_t launch_twiddles<double>(void*, int, cudaStream_t);
template cudaError_t launch_chat<float>(void*, const double*, const double*, const double*,
                                        const double*, int, int, int, int, int, int, double, double,
                                        double, double, double, cudaStream_t);
template cudaError_t launch_chat<double>(void*, const double*, const double*, const double*,
                                         const double*, int, int, int, int, int, int, double, double,
                                         double, double, double, cudaStream_t);

}  // namespace fse

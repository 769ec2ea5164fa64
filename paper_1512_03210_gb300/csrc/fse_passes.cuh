// fse_passes.cuh -- the fused passes of one TS2-GauSum step (Section 4.2, Eqs. tssp1-tssp3).
//
// Data layout in HBM (x fastest, interleaved complex):
//   psi  [nz][ny][nx]            the wave function phi(x~) or its partial spectra
//   S    [nz][2ny][sx] (3D)      x-half-spectrum of the zero-padded density,
//        [ny][sx]      (2D)      sx >= nx+1 (row stride, a multiple of 16)
//   Chat [nz+1][ny+1][nx+1]      kernel transform C^ on |p_j| = 0..n_j (Real)
//
// Passes (3D; 2D drops the z passes and fuses the y passes):
//   X0  fwd-x of psi                                   (start of a call)
//   B   fwd-y of psi                 D  inv-y of psi
//   C   z: fwd . exp(-i f theta_k)/N . inv             (kinetic, Eq. tssp1/tssp3)
//   E   inv-x of psi -> u1 (stored) -> rho=|u1|^2 -> zero-padded R2C along x into S
//   F   y of S: load ny rows, zero-pad to 2ny, fwd
//   G   z of S: load nz rows, zero-pad to 2nz, fwd . K^_n/Npad . inv, keep nz rows
//   H   y of S: inv, keep ny rows
//   A   C2R inv-x of S (crop) -> varphi -> u2 = u1 exp(-i Theta) -> fwd-x of psi
//   XI  inv-x of psi                                   (end of a call)
// Theta = dt beta |u1|^2 + lambda varphi + P_n(x~) (Eqs. solu_step2, int_poten).
#pragma once

#include "fse_fft.cuh"

namespace fse {

enum { MUL_NONE = 0, MUL_KIN = 1, MUL_COULOMB = 2, MUL_DDI = 3 };
enum { XP_FWD = 0, XP_INV = 1, XP_E = 2, XP_A = 3, XP_R = 4, XP_ADJ1 = 5, XP_ADJ2 = 6 };

// Lines per tile: 128-byte rows for the column passes, at most 64 KB of tile.
__host__ __device__ constexpr int ncol_for(int N, int csize) {
  int n = 128 / csize;
  while (n > 2 && n * N * csize > 65536) n /= 2;
  return n;
}
// Threads per tile: about 16 elements per thread, so that a Stockham pass holds
// at most two radix-8 butterflies in registers per thread.
__host__ __device__ constexpr int nt_for(int N, int ncol) {
  return N * ncol >= 4096 ? 512 : (N * ncol >= 2048 ? 256 : 128);
}
// Resident tiles per SM the register budget is sized for: 64 registers per
// thread for float (1024 threads per SM), 128 for double (512 threads).
__host__ __device__ constexpr int minb_for(int nt, int csize) {
  return (csize == 8 ? 1024 : 512) / nt > 0 ? (csize == 8 ? 1024 : 512) / nt : 1;
}

struct ColArgs {
  void* data;
  long long plane_stride;  // elements between planes
  long long line_stride;   // elements between consecutive points of a line
  int nplanes, ncols;      // planes; columns (lines) per plane, contiguous
  int n_load, n_store;     // rows loaded (rest zero) and rows stored
  int tiles_per_plane;
};

struct MulArgs {
  int mode;
  int lx;            // signed-wrap length of the column (x) index; 0 = R2C bin (non-negative)
  int lp;            // signed-wrap length of the plane index (0 = no plane axis)
  int lr;            // signed-wrap length of the row index
  double dkx, dkp, dkr;
  double c0, s, m2;  // kinetic: theta = c0 (k^2 + m2)^s
  double scale;      // 1/N of the transform
  double a0;         // Coulomb: dt*scale; DDI: -dt*scale
  double q[6];       // DDI: 3*scale*(Mxx, Myy, Mrr..): see host code (x, plane, row)
  const void* chat;
  long long chat_sp, chat_sr;
  const void* kin;   // kinetic: table of exp(-i f theta_k) in the field's layout
  int conj;          // kinetic: multiply by the conjugate of the table (adjoint)
};

struct XArgs {
  void* psi;
  void* spec;
  int nlines, ny, srow_mul;
  int use_spec;           // pass A: 0 = no nonlocal term (varphi = 0)
  long long sx;
  double beta_dt, lam;
  double pa, pb, pc, pe;  // P = pa x^2 + pb y^2 + pc x y + pe z^2
  double lo0, lo1, lo2, h0, h1, h2;
  double* part;           // pass R: partial of sum varphi |psi|^2; passes E / XI: partial of sum |u1|^2
  const double* scale;    // pass A: optional renormalisation factor (device scalar)
  const void* aux;        // adjoint passes: u1 (output of the first kinetic half step)
  long long part_stride;  // adjoint pass 1: distance between the three gradient slots
  double dp[12];          // adjoint pass 1: dP/dgamma_v = dp[4v] x^2 + dp[4v+1] y^2 + dp[4v+2] x y + dp[4v+3] z^2
};

// Deterministic float64 block sum (blockDim.x a multiple of 32, <= 1024); result in lane 0 of warp 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

__device__ __forceinline__ int wrap_index(int i, int L) { return i < (L >> 1) ? i : i - L; }

// ---------------------------------------------------------------------------
// Column pass: transforms along a strided axis, tiles of NCOL adjacent columns.
// MODE 0: one transform of direction DIR; MODE 1: fwd . kinetic phase . inv;
// MODE 2: fwd . kernel transform . inv (Coulomb or 3D DDI, chosen in MulArgs).
// ---------------------------------------------------------------------------
template <typename Real, int N, int MODE, int DIR>
__global__ void __launch_bounds__(nt_for(N, ncol_for(N, 2 * sizeof(Real))),
                                  minb_for(nt_for(N, ncol_for(N, 2 * sizeof(Real))), 2 * sizeof(Real)))
k_colpass(ColArgs a, MulArgs m, const typename Cplx<Real>::T* __restrict__ tw) {
  typedef typename Cplx<Real>::T C;
  constexpr int NCOL = ncol_for(N, sizeof(C));
  constexpr int NT = nt_for(N, NCOL);
  constexpr int LDS = NCOL + 1;
  constexpr int TOT = N * NCOL;
  constexpr int PER = (TOT + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int tid = threadIdx.x;
  const int plane = blockIdx.x / a.tiles_per_plane;
  const int c0 = (blockIdx.x - plane * a.tiles_per_plane) * NCOL;
  C* base = reinterpret_cast<C*>(a.data) + (long long)plane * a.plane_stride + c0;
  const int ncv = min(NCOL, a.ncols - c0);

#pragma unroll 8
  for (int it = 0; it < PER; ++it) {
    const int idx = tid + it * NT;
    if ((TOT % NT) == 0 || idx < TOT) {
      const int j = idx / NCOL, c = idx % NCOL;
      C v = mk(Real(0), Real(0));
      if (j < a.n_load && c < ncv) v = base[(long long)j * a.line_stride + c];
      buf[j * LDS + c] = v;
    }
  }
  __syncthreads();
  if constexpr (MODE == 0) {
    fft_tile<C, N, NCOL, NT, DIR>(buf, tw);
  } else {
    fft_tile<C, N, NCOL, NT, -1>(buf, tw);
#pragma unroll 4
    for (int it = 0; it < PER; ++it) {
      const int idx = tid + it * NT;
      if ((TOT % NT) == 0 || idx < TOT) {
        const int j = idx / NCOL, c = idx % NCOL;
        const int ix = c0 + c;
        C v = buf[j * LDS + c];
        const int pr = wrap_index(j, m.lr);
        if constexpr (MODE == 1) {
          // kinetic phase exp(-i f theta_k) from the plan's table (same layout as the field)
          const C* tab = reinterpret_cast<const C*>(m.kin);
          const C t = c < ncv ? __ldg(&tab[(long long)plane * a.plane_stride + c0 + c + (long long)j * a.line_stride])
                              : mk(Real(0), Real(0));
          const Real sc = Real(m.scale);
          v = m.conj ? cmulc(v, t) : cmul(v, t);
          v = mk(sc * v.x, sc * v.y);
        } else {
          // kernel transform on the padded grid; x index is an R2C bin 0..nx
          const int px = ix;                                   // non-negative
          const int ap = m.lp ? abs(wrap_index(plane, m.lp)) : 0;
          const int ar = abs(pr);
          const Real* ch = reinterpret_cast<const Real*>(m.chat);
          const Real cv = (ix <= (m.lx >> 1)) ? __ldg(&ch[ar * m.chat_sr + ap * m.chat_sp + px]) : Real(0);
          Real f;
          if (m.mode == MUL_COULOMB) {
            f = Real(m.a0) * cv;
          } else {
            // odd factors vanish at the Nyquist index (Hermitian symmetry)
            const Real kx = Real(m.dkx) * Real(px);
            const Real kp = m.lp ? Real(m.dkp) * Real(wrap_index(plane, m.lp)) : Real(0);
            const Real kr = Real(m.dkr) * Real(pr);
            const Real kxo = (2 * px == m.lx) ? Real(0) : kx;
            const Real kpo = (m.lp && 2 * plane == m.lp) ? Real(0) : kp;
            const Real kro = (2 * j == m.lr) ? Real(0) : kr;
            const Real qf = Real(m.q[0]) * kx * kx + Real(m.q[1]) * kp * kp + Real(m.q[2]) * kr * kr +
                            Real(m.q[3]) * kxo * kpo + Real(m.q[4]) * kxo * kro + Real(m.q[5]) * kpo * kro;
            f = Real(m.a0) + qf * cv;
          }
          v = mk(f * v.x, f * v.y);
        }
        buf[j * LDS + c] = v;
      }
    }
    __syncthreads();
    fft_tile<C, N, NCOL, NT, +1>(buf, tw);
  }
#pragma unroll 8
  for (int it = 0; it < PER; ++it) {
    const int idx = tid + it * NT;
    if ((TOT % NT) == 0 || idx < TOT) {
      const int j = idx / NCOL, c = idx % NCOL;
      if (j < a.n_store && c < ncv) base[(long long)j * a.line_stride + c] = buf[j * LDS + c];
    }
  }
}

// ---------------------------------------------------------------------------
// x passes over tiles of NCOL consecutive lines (rows of psi).
// ---------------------------------------------------------------------------
template <typename Real, int NX>
struct XCfg {
  typedef typename Cplx<Real>::T C;
  static constexpr int NCOL = ncol_for(2 * NX, sizeof(C)) < 2 ? 2 : ncol_for(2 * NX, sizeof(C));
  static constexpr int NT = 256;
  static constexpr int LDS = NCOL + 1;
  static constexpr int LDS2 = NCOL / 2 + 1;
  static constexpr int TOT = NCOL * NX;
  static constexpr int PER = (TOT + NT - 1) / NT;
  static constexpr size_t smem_bytes() {
    return sizeof(C) * (size_t)((NX * LDS) > (2 * NX * LDS2) ? (NX * LDS) : (2 * NX * LDS2));
  }
};

__device__ __forceinline__ long long srow(int l, int ny, int mul) {
  return (long long)(l / ny) * (mul * ny) + (l % ny);
}

// Real values of the NCOL lines of a tile (one per (line, x) item of the
// thread, PER items) -> x-half-spectra of the zero-padded lines in S. Two real
// lines form one complex line; one FFT of length 2 NX; the two spectra are
// separated with A_k = (Z_k + conj Z_-k)/2, B_k = (Z_k - conj Z_-k)/(2i).
// The caller has synchronised (buf free); ends without a barrier.
template <typename Real, int NX>
__device__ __forceinline__ void r2c_rows(const XArgs& a, typename Cplx<Real>::T* buf, int l0,
                                         const typename Cplx<Real>::T* __restrict__ tw2n,
                                         const Real (&val)[XCfg<Real, NX>::PER]) {
  typedef XCfg<Real, NX> K;
  typedef typename K::C C;
  constexpr int NCOL = K::NCOL, NT = K::NT, LDS2 = K::LDS2, TOT = K::TOT, PER = K::PER;
  const int tid = threadIdx.x;
  C* S = reinterpret_cast<C*>(a.spec);
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int idx = tid + it * NT;
    if ((TOT % NT) == 0 || idx < TOT) {
      const int l = idx / NX, x = idx % NX;
      reinterpret_cast<Real*>(&buf[x * LDS2 + (l >> 1)])[l & 1] = val[it];
    }
  }
  for (int idx = tid; idx < (NCOL / 2) * NX; idx += NT) {
    const int q = idx / NX, x = NX + idx % NX;
    buf[x * LDS2 + q] = mk(Real(0), Real(0));
  }
  __syncthreads();
  fft_tile<C, 2 * NX, NCOL / 2, NT, -1>(buf, tw2n);
  for (int idx = tid; idx < (NCOL / 2) * (NX + 1); idx += NT) {
    const int q = idx / (NX + 1), k = idx % (NX + 1);
    const C zk = buf[k * LDS2 + q];
    const C zm = buf[((2 * NX - k) % (2 * NX)) * LDS2 + q];
    const int la = l0 + 2 * q;
    const C A = mk(Real(0.5) * (zk.x + zm.x), Real(0.5) * (zk.y - zm.y));
    const C B = mk(Real(0.5) * (zk.y + zm.y), Real(0.5) * (zm.x - zk.x));
    if (la < a.nlines) S[srow(la, a.ny, a.srow_mul) * a.sx + k] = A;
    if (la + 1 < a.nlines) S[srow(la + 1, a.ny, a.srow_mul) * a.sx + k] = B;
  }
}

// x-half-spectra in S of the tile's lines -> real values (cropped C2R of length
// 2 NX, two lines per complex line via the Hermitian extension Z = A + i B).
// The caller has synchronised (buf free); ends after the values are read
// (the caller synchronises before reusing buf).
template <typename Real, int NX>
__device__ __forceinline__ void c2r_rows(const XArgs& a, typename Cplx<Real>::T* buf, int l0,
                                         const typename Cplx<Real>::T* __restrict__ tw2n,
                                         Real (&val)[XCfg<Real, NX>::PER]) {
  typedef XCfg<Real, NX> K;
  typedef typename K::C C;
  constexpr int NCOL = K::NCOL, NT = K::NT, LDS2 = K::LDS2, TOT = K::TOT, PER = K::PER;
  const int tid = threadIdx.x;
  const C* S = reinterpret_cast<const C*>(a.spec);
  for (int idx = tid; idx < (NCOL / 2) * (NX + 1); idx += NT) {
    const int q = idx / (NX + 1), k = idx % (NX + 1);
    const int la = l0 + 2 * q;
    C A = mk(Real(0), Real(0)), B = A;
    if (la < a.nlines) A = S[srow(la, a.ny, a.srow_mul) * a.sx + k];
    if (la + 1 < a.nlines) B = S[srow(la + 1, a.ny, a.srow_mul) * a.sx + k];
    buf[k * LDS2 + q] = mk(A.x - B.y, A.y + B.x);
    if (k > 0 && k < NX) buf[(2 * NX - k) * LDS2 + q] = mk(A.x + B.y, B.x - A.y);
  }
  __syncthreads();
  fft_tile<C, 2 * NX, NCOL / 2, NT, +1>(buf, tw2n);
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int idx = tid + it * NT;
    val[it] = Real(0);
    if ((TOT % NT) == 0 || idx < TOT) {
      const int l = idx / NX, x = idx % NX;
      const C z = buf[x * LDS2 + (l >> 1)];
      val[it] = (l & 1) ? z.y : z.x;
    }
  }
}

template <typename Real>
__device__ __forceinline__ Real trap_phase(const XArgs& a, int x, int lg) {
  const Real X = Real(a.lo0) + Real(a.h0) * Real(x);
  const Real Y = Real(a.lo1) + Real(a.h1) * Real(lg % a.ny);
  const Real Z = Real(a.lo2) + Real(a.h2) * Real(lg / a.ny);
  return Real(a.pa) * X * X + Real(a.pb) * Y * Y + Real(a.pc) * X * Y + Real(a.pe) * Z * Z;
}

template <typename Real, int NX, int KIND>
__global__ void __launch_bounds__(256, sizeof(Real) == 4 ? 4 : 2)
k_xpass(XArgs a, const typename Cplx<Real>::T* __restrict__ twn,
        const typename Cplx<Real>::T* __restrict__ tw2n) {
  typedef XCfg<Real, NX> K;
  typedef typename K::C C;
  constexpr int NCOL = K::NCOL, NT = K::NT, LDS = K::LDS, TOT = K::TOT, PER = K::PER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int tid = threadIdx.x;
  const int l0 = blockIdx.x * NCOL;
  C* psi = reinterpret_cast<C*>(a.psi);

  if constexpr (KIND == XP_FWD || KIND == XP_INV || KIND == XP_E) {
#pragma unroll 8
    for (int it = 0; it < PER; ++it) {
      const int idx = tid + it * NT;
      if ((TOT % NT) == 0 || idx < TOT) {
        const int l = idx / NX, x = idx % NX;
        C v = mk(Real(0), Real(0));
        if (l0 + l < a.nlines) v = psi[(long long)(l0 + l) * NX + x];
        buf[x * LDS + l] = v;
      }
    }
    __syncthreads();
    fft_tile<C, NX, NCOL, NT, (KIND == XP_FWD ? -1 : +1)>(buf, twn);
    Real rho[PER];
#pragma unroll
    for (int it = 0; it < PER; ++it) {
      const int idx = tid + it * NT;
      rho[it] = Real(0);
      if ((TOT % NT) == 0 || idx < TOT) {
        const int l = idx / NX, x = idx % NX;
        const C v = buf[x * LDS + l];
        if (l0 + l < a.nlines) psi[(long long)(l0 + l) * NX + x] = v;
        rho[it] = v.x * v.x + v.y * v.y;
      }
    }
    if constexpr (KIND == XP_E || KIND == XP_INV) {
      if (a.part) {  // float64 mass partial of this tile (renormalisation)
        double acc = 0.0;
#pragma unroll
        for (int it = 0; it < PER; ++it) acc += (double)rho[it];
        acc = block_sum(acc, red);
        if (tid == 0) a.part[blockIdx.x] = acc;
      }
    }
    if constexpr (KIND == XP_E) {
      __syncthreads();
      r2c_rows<Real, NX>(a, buf, l0, tw2n, rho);
    }
  } else if constexpr (KIND == XP_ADJ1) {
    // adjoint, first half: g_u2 (in psi) -> h = exp(+i Theta) g_u2 (stored in psi),
    // r = Im(conj(g_u2) u2) -> x-half-spectra of r in S, trap-gradient partials
    const C* u1p = reinterpret_cast<const C*>(a.aux);
    Real vphi[PER];
#pragma unroll
    for (int it = 0; it < PER; ++it) vphi[it] = Real(0);
    if (a.use_spec) {
      c2r_rows<Real, NX>(a, buf, l0, tw2n, vphi);
      __syncthreads();
    }
    Real rr[PER];
    double dg0 = 0.0, dg1 = 0.0, dg2 = 0.0;
#pragma unroll
    for (int it = 0; it < PER; ++it) {
      const int idx = tid + it * NT;
      rr[it] = Real(0);
      if ((TOT % NT) == 0 || idx < TOT) {
        const int l = idx / NX, x = idx % NX;
        const int lg = l0 + l;
        if (lg < a.nlines) {
          const long long o = (long long)lg * NX + x;
          const C u = u1p[o];
          const C g = psi[o];
          const Real th = Real(a.beta_dt) * (u.x * u.x + u.y * u.y) + Real(a.lam) * vphi[it] + trap_phase<Real>(a, x, lg);
          Real sn, cs;
          sincos(th, &sn, &cs);
          const C u2 = mk(u.x * cs + u.y * sn, u.y * cs - u.x * sn);
          const Real r = g.x * u2.y - g.y * u2.x;
          rr[it] = r;
          psi[o] = mk(g.x * cs - g.y * sn, g.y * cs + g.x * sn);
          const double X = a.lo0 + a.h0 * x, Y = a.lo1 + a.h1 * (lg % a.ny), Z = a.lo2 + a.h2 * (lg / a.ny);
          dg0 += (double)r * (a.dp[0] * X * X + a.dp[1] * Y * Y + a.dp[2] * X * Y + a.dp[3] * Z * Z);
          dg1 += (double)r * (a.dp[4] * X * X + a.dp[5] * Y * Y + a.dp[6] * X * Y + a.dp[7] * Z * Z);
          dg2 += (double)r * (a.dp[8] * X * X + a.dp[9] * Y * Y + a.dp[10] * X * Y + a.dp[11] * Z * Z);
        }
      }
    }
    if (a.part) {
      dg0 = block_sum(dg0, red);
      if (tid == 0) a.part[blockIdx.x] = dg0;
      dg1 = block_sum(dg1, red);
      if (tid == 0) a.part[a.part_stride + blockIdx.x] = dg1;
      dg2 = block_sum(dg2, red);
      if (tid == 0) a.part[2 * a.part_stride + blockIdx.x] = dg2;
    }
    if (a.use_spec) {
      __syncthreads();
      r2c_rows<Real, NX>(a, buf, l0, tw2n, rr);
    }
  } else if constexpr (KIND == XP_ADJ2) {
    // adjoint, second half: g_u1 = h + 2 q u1, q = dt beta r + lambda Kc r, r = Im(conj(h) u1)
    const C* u1p = reinterpret_cast<const C*>(a.aux);
    Real kr[PER];
#pragma unroll
    for (int it = 0; it < PER; ++it) kr[it] = Real(0);
    if (a.use_spec) c2r_rows<Real, NX>(a, buf, l0, tw2n, kr);
#pragma unroll
    for (int it = 0; it < PER; ++it) {
      const int idx = tid + it * NT;
      if ((TOT % NT) == 0 || idx < TOT) {
        const int l = idx / NX, x = idx % NX;
        const int lg = l0 + l;
        if (lg < a.nlines) {
          const long long o = (long long)lg * NX + x;
          const C u = u1p[o];
          const C h = psi[o];
          const Real r = h.x * u.y - h.y * u.x;
          const Real q2 = Real(2) * (Real(a.beta_dt) * r + Real(a.lam) * kr[it]);
          psi[o] = mk(h.x + q2 * u.x, h.y + q2 * u.y);
        }
      }
    }
  } else {
    // XP_A / XP_R: varphi from the cropped C2R of S
    Real vphi[PER];
#pragma unroll
    for (int it = 0; it < PER; ++it) vphi[it] = Real(0);
    if (a.use_spec) c2r_rows<Real, NX>(a, buf, l0, tw2n, vphi);
    if constexpr (KIND == XP_R) {
      // sum over the tile of varphi * |psi|^2 (nonlocal interaction energy density)
      double acc = 0.0;
#pragma unroll
      for (int it = 0; it < PER; ++it) {
        const int idx = tid + it * NT;
        if ((TOT % NT) == 0 || idx < TOT) {
          const int l = idx / NX, x = idx % NX;
          if (l0 + l < a.nlines) {
            const C u = psi[(long long)(l0 + l) * NX + x];
            acc += (double)vphi[it] * ((double)u.x * u.x + (double)u.y * u.y);
          }
        }
      }
      acc = block_sum(acc, red);
      if (tid == 0) a.part[blockIdx.x] = acc;
      return;
    } else {
      __syncthreads();
#pragma unroll
      for (int it = 0; it < PER; ++it) {
        const int idx = tid + it * NT;
        if ((TOT % NT) == 0 || idx < TOT) {
          const int l = idx / NX, x = idx % NX;
          const int lg = l0 + l;
          C u2 = mk(Real(0), Real(0));
          if (lg < a.nlines) {
            const C u = psi[(long long)lg * NX + x];
            const Real rho = u.x * u.x + u.y * u.y;
            const Real th = Real(a.beta_dt) * rho + Real(a.lam) * vphi[it] + trap_phase<Real>(a, x, lg);
            Real sn, cs;
            sincos(th, &sn, &cs);
            u2 = mk(u.x * cs + u.y * sn, u.y * cs - u.x * sn);
            if (a.scale) {
              const Real f = Real(*a.scale);
              u2 = mk(f * u2.x, f * u2.y);
            }
          }
          buf[x * LDS + l] = u2;
        }
      }
      __syncthreads();
      fft_tile<C, NX, NCOL, NT, -1>(buf, twn);
#pragma unroll 8
      for (int it = 0; it < PER; ++it) {
        const int idx = tid + it * NT;
        if ((TOT % NT) == 0 || idx < TOT) {
          const int l = idx / NX, x = idx % NX;
          if (l0 + l < a.nlines) psi[(long long)(l0 + l) * NX + x] = buf[x * LDS + l];
        }
      }
    }
  }
}

// Host-side launchers (explicitly instantiated per precision).
template <typename Real>
cudaError_t launch_colpass(int N, int mode, int dir, const ColArgs& a, const MulArgs& m,
                           const void* tw, cudaStream_t st);
template <typename Real>
cudaError_t launch_xpass(int kind, int nx, const XArgs& a, const void* twn, const void* tw2n,
                         cudaStream_t st);
// Lines per tile of the column pass of length N and of the x passes of length nx.
template <typename Real> int colpass_ncol(int N);
template <typename Real> int xpass_ncol(int nx);

}  // namespace fse

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
#include "fse_fft_x2.cuh"

namespace fse {

enum { MUL_NONE = 0, MUL_KIN = 1, MUL_COULOMB = 2, MUL_DDI = 3 };
enum { XP_FWD = 0, XP_INV = 1, XP_E = 2, XP_A = 3, XP_R = 4, XP_ADJ1 = 5, XP_ADJ2 = 6, XP_AL = 7 };

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
  // > 0: tiles_per_plane full tiles cover the first tiles_per_plane * NCOL
  // columns of every plane, and further tiles each take NCOL consecutive
  // (plane, column) pairs of the `tail` remaining columns
  int tail;
};

// Blocks of a column pass: the full tiles and the gathered tail tiles.
__host__ __device__ inline long long col_blocks(const ColArgs& a, int ncol) {
  const long long full = (long long)a.nplanes * a.tiles_per_plane;
  return full + (a.tail > 0 ? ((long long)a.nplanes * a.tail + ncol - 1) / ncol : 0);
}

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
  int chat_cx;       // padded length of a C^ row (x bins 0..lx/2, then zeros), a multiple of 4
  const void* kin;   // kinetic: octant table of exp(-i f theta_k) on |p_j| = 0..n_j/2
  long long kin_sp, kin_sr;  // kinetic: octant strides of the plane and row axes
  int conj;          // kinetic: multiply by the conjugate of the table (adjoint)
  // float copies of the scalars above, written by fill_f32 before a launch: a
  // float kernel reads them as they are instead of converting the double
  // fields in every thread (double-to-float conversions issue on the narrow
  // FP64 pipe)
  struct {
    float dkx, dkp, dkr, scale, a0, q[6];
  } f;
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
  // optical lattice lat_amp sum_v sin^2(lat_k[v] x_v): its integral over the
  // window is sum_q lat_w[q] V_lat(x(tau_q)), x = (c x~ + s y~, -s x~ + c y~, z~)
  // with (c, s) = (lat_c[q], lat_s[q]) = (cos, sin)(Omega tau_q)
  double lat_amp;
  double lat_k[3];
  int lat_nq;
  double lat_w[16], lat_c[16], lat_s[16];
  void* out;              // pass R: optional real array receiving varphi (the nonlocal potential)
  // float copies of the scalars above (see MulArgs::f)
  struct {
    float beta_dt, lam, pa, pb, pc, pe, lo0, lo1, lo2, h0, h1, h2;
    float lat_amp, lat_k[3], lat_w[16], lat_c[16], lat_s[16];
  } f;
};

__host__ __device__ inline void fill_f32(MulArgs& m) {
  m.f.dkx = (float)m.dkx;
  m.f.dkp = (float)m.dkp;
  m.f.dkr = (float)m.dkr;
  m.f.scale = (float)m.scale;
  m.f.a0 = (float)m.a0;
  for (int i = 0; i < 6; ++i) m.f.q[i] = (float)m.q[i];
}

// the step-dependent scalars of an x pass (phase coefficients)
__host__ __device__ inline void fill_f32_phase(XArgs& a) {
  a.f.beta_dt = (float)a.beta_dt;
  a.f.lam = (float)a.lam;
  a.f.pa = (float)a.pa;
  a.f.pb = (float)a.pb;
  a.f.pc = (float)a.pc;
  a.f.pe = (float)a.pe;
}

__host__ __device__ inline void fill_f32(XArgs& a) {
  fill_f32_phase(a);
  a.f.lo0 = (float)a.lo0;
  a.f.lo1 = (float)a.lo1;
  a.f.lo2 = (float)a.lo2;
  a.f.h0 = (float)a.h0;
  a.f.h1 = (float)a.h1;
  a.f.h2 = (float)a.h2;
  a.f.lat_amp = (float)a.lat_amp;
  for (int i = 0; i < 3; ++i) a.f.lat_k[i] = (float)a.lat_k[i];
  for (int i = 0; i < 16; ++i) {
    a.f.lat_w[i] = (float)a.lat_w[i];
    a.f.lat_c[i] = (float)a.lat_c[i];
    a.f.lat_s[i] = (float)a.lat_s[i];
  }
}

// A scalar parameter in the kernel's precision: the double field, or its float copy.
template <typename Real>
__device__ __forceinline__ Real prm(double d, float f);
template <> __device__ __forceinline__ float prm<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double prm<double>(double d, float) { return d; }

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

// First statement of every step pass. The passes of a step are launched with
// programmatic dependent launch: a block first waits until the previous pass
// has completed and its writes are visible (griddepcontrol.wait; immediate
// for a launch without that dependency), then lets the next pass be launched
// (griddepcontrol.launch_dependents), so that the next pass's blocks are
// scheduled onto SMs as this pass's last blocks finish instead of after a
// launch gap. The next pass's blocks do nothing before their own wait.
__device__ __forceinline__ void pass_prologue() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// Column pass: transforms along a strided axis, tiles of NCOL adjacent columns.
// Variants (VAR):
//   COL_FWD / COL_INV  one transform of the wave function (exact twiddles)
//   COL_PADF           forward transform of rows [0, N/2) zero-padded to N (density)
//   COL_CROPI          inverse transform keeping rows [0, N/2) (density)
//   COL_KIN            fwd . kinetic phase . inv of the wave function
//   COL_KHAT           rows [0, N/2) zero-padded, fwd . kernel transform . inv,
//                      rows [0, N/2) kept (density)
// The first radix pass reads global memory, the last one writes it (or hands
// its outputs, in registers, to the multiplier). Known-zero inputs and
// unneeded outputs are constants / dead code for the compiler.
// ---------------------------------------------------------------------------
enum { COL_FWD = 0, COL_INV = 1, COL_PADF = 2, COL_CROPI = 3, COL_KIN = 4, COL_KHAT = 5 };

__host__ __device__ constexpr int col_ncol(int N, int csize) { return ncol_for(N, csize); }

// Threads per tile of a packed (pair) column pass: 256 by default, so that a
// long transform keeps two items per thread and registers for them; the
// zero-padded forward (F) and cropped inverse (H) transforms of the density,
// one transform each and no multiplier, fit 512 threads of one item without
// spilling and run faster with the extra warps.
__host__ __device__ constexpr int x2_maxt(int var) { return (var == 2 || var == 3) ? 512 : 256; }

template <typename Real, int N, int VAR = -1>
struct ColCfg {
  typedef typename Cplx<Real>::T C;
  static constexpr int NCOL = col_ncol(N, sizeof(C));
  // float path, power-of-two plans (radices up to 8): items of two adjacent
  // columns (16-byte row accesses, shared twiddles); otherwise one column
  static constexpr int CW = (sizeof(C) == 8 && plan_lcm(N) <= 8 && NCOL % 2 == 0) ? 2 : 1;
  static constexpr int NCP = NCOL / CW;
  // leading dimension of the exchange tile: a column pair is one 16-byte slot
  // and the 8 threads of a quarter warp always touch the NCOL / 2 slots of one
  // row, so pairs need no padding; single columns pad to NCOL + 1
  static constexpr int LDS = CW == 2 ? NCOL : NCOL + 1;
  static constexpr int MAXT = CW == 2 ? x2_maxt(VAR) : 512;
  static constexpr int E = reg_elems(N, NCOL, CW, MAXT);
  static constexpr int NT = reg_threads(N, NCOL, CW, MAXT);
  static constexpr int R0 = radix_plan(N).r[0];
  static constexpr int RL = radix_plan(N).r[radix_plan(N).npass - 1];
  static constexpr int MINB = (sizeof(C) == 8 && E > 16) ? (512 / NT > 0 ? 512 / NT : 1) : minb_for(NT, sizeof(C));
  // exchange tile, then (kernel-transform variant) the block's C^ values on |p| = 0..N/2
  static constexpr size_t TILE_BYTES = sizeof(C) * (size_t)N * LDS;
  __host__ __device__ static constexpr size_t tile_bytes() { return TILE_BYTES; }
  __host__ __device__ static constexpr size_t chat_bytes() { return sizeof(Real) * (size_t)(N / 2 + 1) * NCOL; }
  __host__ __device__ static constexpr size_t base_bytes(int var) { return tile_bytes() + (var == 5 ? chat_bytes() : 0); }
  __host__ __device__ static constexpr size_t smem_bytes(int var) { return base_bytes(var); }
  // pairs: first-pass inputs per thread (rows of the zero half of a padded
  // line are not read)
  __host__ __device__ static constexpr bool half_in(int var) { return var == 2 || var == 5; }
  __host__ __device__ static constexpr int rh(int var) { return half_in(var) ? R0 / 2 : R0; }
  __host__ __device__ static constexpr int first(int var) { return (E / 2 / R0) * rh(var); }
};

// One tile of a column pass: NCOL adjacent columns of one plane, or (GATHER)
// NCOL (plane, column) pairs of the tail columns. The two kinds are separate
// instantiations, so that the per-column state of the gathered tiles does not
// take registers from the full ones.
template <typename Real, int N, int VAR, bool GATHER>
__device__ __forceinline__ void colpass_tile(const ColArgs& a, const MulArgs& m,
                                             const typename Cplx<Real>::T* __restrict__ tw, int bid, int ngat) {
  typedef ColCfg<Real, N, VAR> K;
  typedef typename K::C C;
  constexpr int NCOL = K::NCOL, NCP = K::NCP, CW = K::CW, LDS = K::LDS, NT = K::NT, E = K::E;
  constexpr int R0 = K::R0, RL = K::RL;
  // forward . multiplier . inverse variants whose radix plan reads the same
  // reversed (all radix 8, e.g. N = 512) run the inverse straight on the
  // forward's outputs as they sit in registers (positions j + r N/RL); other
  // plans go through one exchange, which measured faster than reordering the
  // inverse's radices
  constexpr bool FUSED = (VAR == COL_KIN || VAR == COL_KHAT) && plan_palindrome(N);
  constexpr int RF = FUSED ? R0 : RL;
  // input r of the first pass (output r of the last) lies at rows >= N/2 for
  // every j when 2 r >= R: zero in a zero-padded input, dropped by the crop
  constexpr bool HALF_IN = (VAR == COL_PADF || VAR == COL_KHAT);
  constexpr bool HALF_OUT = (VAR == COL_CROPI || VAR == COL_KHAT);
  constexpr bool EXACT = (VAR == COL_FWD || VAR == COL_INV || VAR == COL_KIN);
  constexpr int DIR1 = (VAR == COL_INV || VAR == COL_CROPI) ? +1 : -1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int tid = threadIdx.x;
  static_assert(NT % NCP == 0, "a thread keeps one column group of the tile");
  const int cg = tid % NCP;  // this thread's columns of the tile: cg CW + q, q < CW
  constexpr bool gather = GATHER;
  const int breg = bid - ngat;
  const int tp = gather ? 0 : breg / a.tiles_per_plane;
  const int c0 = gather ? 0 : (breg - tp * a.tiles_per_plane) * NCOL;
  // kernel-transform pass over a full even set of planes: planes p and lp - p
  // (same |p|, same C^ values) run next to each other, so the octant is read
  // from HBM about once
  const int plane = (VAR == COL_KHAT && m.lp == a.nplanes && (m.lp & 1) == 0 && tp > 0)
                        ? ((tp & 1) ? (tp + 1) >> 1 : m.lp - (tp >> 1))
                        : tp;
  // column cc of the tile -> (plane, x index); false past the data
  auto col_of = [&](int cc, int& pl, int& px) -> bool {
    if (!gather) {
      pl = plane;
      px = c0 + cc;
      return px < a.ncols;
    }
    const int q = bid * NCOL + cc;
    pl = q / a.tail;
    px = a.tiles_per_plane * NCOL + q % a.tail;
    if (pl < a.nplanes) return true;
    pl = 0;
    px = 0;
    return false;
  };
  // this thread's columns: plane, x index, validity and base pointer (row r of
  // column q is colp[q][r * line_stride])
  int my_plane[CW], my_px[CW];
  bool my_ok[CW];
  C* colp[CW];
#pragma unroll
  for (int q = 0; q < CW; ++q) {
    my_ok[q] = col_of(cg * CW + q, my_plane[q], my_px[q]);
    // the columns of a full tile are adjacent in one plane
    colp[q] = (!gather && q > 0) ? colp[0] + q
                                 : reinterpret_cast<C*>(a.data) + (long long)my_plane[q] * a.plane_stride + my_px[q];
  }
  // both columns of a pair side by side in memory, 16-byte aligned: one access per row
  bool vec = false;
  if constexpr (CW == 2)
    vec = !gather && my_ok[0] && my_ok[1] && (reinterpret_cast<uintptr_t>(colp[0]) % 16 == 0) &&
          (a.line_stride % 2 == 0);
  C v[E];
  Real* sC = reinterpret_cast<Real*>(smem_raw + K::TILE_BYTES);
  if constexpr (VAR == COL_KHAT) {
    // start fetching C^ (|p_row| = 0..N/2, this tile's columns) while the forward transform runs
    const Real* ch = reinterpret_cast<const Real*>(m.chat);
    if (!gather) {
      // the tile's columns of a C^ row are contiguous and 16-byte aligned
      // (rows padded to a multiple of 4 values, c0 a multiple of NCOL): one
      // 16-byte copy per EPC values; copies past the padded row are zero-filled
      constexpr int EPC = 16 / (int)sizeof(Real), CPR = NCOL / EPC;
      static_assert(NCOL % EPC == 0, "C^ copies of 16 bytes");
      const Real* chp = ch + (m.lp ? (long long)abs(wrap_index(plane, m.lp)) * m.chat_sp : 0) + c0;
      const int left = m.chat_cx - c0;
      for (int idx = tid; idx < (N / 2 + 1) * CPR; idx += NT) {
        const int ar = idx / CPR, qd = idx - ar * CPR;
        Real* dst = &sC[ar * NCOL + qd * EPC];
        if (qd * EPC < left) {
          cp_async<16>(dst, &chp[(long long)ar * m.chat_sr + qd * EPC]);
        } else {
#pragma unroll
          for (int e = 0; e < EPC; ++e) dst[e] = Real(0);
        }
      }
    } else {
      for (int idx = tid; idx < (N / 2 + 1) * NCOL; idx += NT) {
        const int ar = idx / NCOL, cc = idx % NCOL;
        int pl, px;
        const bool ok = col_of(cc, pl, px);
        const int ap = m.lp ? abs(wrap_index(pl, m.lp)) : 0;
        if (ok && px <= (m.lx >> 1))
          cp_async<sizeof(Real)>(&sC[idx], &ch[(long long)ar * m.chat_sr + (long long)ap * m.chat_sp + px]);
        else
          sC[idx] = Real(0);
      }
    }
    cp_async_commit();
  }

  // inputs of the first pass straight from global memory
#pragma unroll
  for (int i = 0; i < E / (R0 * CW); ++i) {
    const int j = (tid + i * NT) / NCP;
#pragma unroll
    for (int r = 0; r < R0; ++r) {
      const int row = j + r * (N / R0);
      C* dst[CW];
#pragma unroll
      for (int q = 0; q < CW; ++q) dst[q] = &v[(i * CW + q) * R0 + r];
      if (HALF_IN && 2 * r >= R0) {
#pragma unroll
        for (int q = 0; q < CW; ++q) *dst[q] = mk(Real(0), Real(0));  // rows >= N/2 of a zero-padded line
      } else if constexpr (CW == 2) {
        if (row < a.n_load && vec) {
          ld_pair(&colp[0][(long long)row * a.line_stride], *dst[0], *dst[1]);
        } else {
#pragma unroll
          for (int q = 0; q < CW; ++q)
            *dst[q] = (row < a.n_load && my_ok[q]) ? colp[q][(long long)row * a.line_stride] : mk(Real(0), Real(0));
        }
      } else {
        *dst[0] = (row < a.n_load && my_ok[0]) ? colp[0][(long long)row * a.line_stride] : mk(Real(0), Real(0));
      }
    }
  }
  if constexpr (VAR == COL_FWD || VAR == COL_INV || VAR == COL_PADF || VAR == COL_CROPI) {
    regs_fft<C, N, NCP, CW, NT, E, LDS, DIR1, EXACT, 0, 1, false, HALF_IN>(v, buf, tw);
  } else {
    regs_fft<C, N, NCP, CW, NT, E, LDS, -1, EXACT, 0, 1, false, HALF_IN>(v, buf, tw);
    // spectral multiplier on the outputs (row = frequency index along the axis)
    if constexpr (VAR == COL_KIN) {
      // kinetic phase exp(-i f theta_k) from the plan's octant table, indexed by
      // |p_x| (column), |p_plane| and |p_row| (row = frequency index along the axis)
      const C* tab[CW];
      int ax[CW];
#pragma unroll
      for (int q = 0; q < CW; ++q) {
        tab[q] = reinterpret_cast<const C*>(m.kin) + (m.lp ? (long long)abs(wrap_index(my_plane[q], m.lp)) * m.kin_sp : 0);
        ax[q] = abs(wrap_index(min(my_px[q], m.lx - 1), m.lx));
      }
      const Real sc = prm<Real>(m.scale, m.f.scale);
#pragma unroll
      for (int i = 0; i < E / (RL * CW); ++i) {
        const int j = (tid + i * NT) / NCP;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int row = j + r * (N / RL);
          const long long ro = (long long)abs(wrap_index(row, m.lr)) * m.kin_sr;
          C y[CW];
#pragma unroll
          for (int q = 0; q < CW; ++q) {
            const C t = my_ok[q] ? __ldg(&tab[q][ro + ax[q]]) : mk(Real(1), Real(0));
            const C x = unit_mul(v[(i * CW + q) * RL + r], t.x, t.y, m.conj != 0);
            y[q] = mk(sc * x.x, sc * x.y);
            if constexpr (FUSED) v[(i * CW + q) * RL + r] = y[q];
          }
          // both columns of a pair in one 16-byte store (LDS even)
          if constexpr (!FUSED) {
            if constexpr (CW == 2) st_pair(&buf[row * LDS + cg * CW], y[0], y[1]);
            else buf[row * LDS + cg] = y[0];
          }
        }
      }
    } else {
      // kernel transform on the padded grid: f = a0 C^ (Coulomb) or a0 + (k^T Q k) C^ (DDI);
      // the column (x, an R2C bin 0..nx) and plane factors are fixed per thread
      cp_async_wait_all();
      __syncthreads();
      const bool ddi = m.mode == MUL_DDI;
      Real Aq[CW], Bq[CW];
#pragma unroll
      for (int q = 0; q < CW; ++q) {
        const Real kp = m.lp ? prm<Real>(m.dkp, m.f.dkp) * Real(wrap_index(my_plane[q], m.lp)) : Real(0);
        const Real kpo = (m.lp && 2 * my_plane[q] == m.lp) ? Real(0) : kp;
        const Real kx = prm<Real>(m.dkx, m.f.dkx) * Real(my_px[q]);
        const Real kxo = (2 * my_px[q] == m.lx) ? Real(0) : kx;
        // q(k) = A + B kr + q2 kr^2 (kr replaced by 0 in B at the Nyquist row)
        Aq[q] = prm<Real>(m.q[0], m.f.q[0]) * kx * kx + prm<Real>(m.q[1], m.f.q[1]) * kp * kp +
                prm<Real>(m.q[3], m.f.q[3]) * kxo * kpo;
        Bq[q] = prm<Real>(m.q[4], m.f.q[4]) * kxo + prm<Real>(m.q[5], m.f.q[5]) * kpo;
      }
#pragma unroll
      for (int i = 0; i < E / (RL * CW); ++i) {
        const int j = (tid + i * NT) / NCP;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int row = j + r * (N / RL);
          const int pr = wrap_index(row, m.lr);
          const Real kr = prm<Real>(m.dkr, m.f.dkr) * Real(pr);
          const Real kro = (2 * row == m.lr) ? Real(0) : kr;
          Real cvq[CW];
          C yq[CW];
          if constexpr (CW == 2) {
            const auto c2 = *reinterpret_cast<const typename Cplx<Real>::T*>(&sC[abs(pr) * NCOL + cg * CW]);
            cvq[0] = c2.x;
            cvq[1] = c2.y;
          } else {
            cvq[0] = sC[abs(pr) * NCOL + cg];
          }
#pragma unroll
          for (int q = 0; q < CW; ++q) {
            const Real cv = cvq[q];
            Real f;
            if (ddi) {
              const Real qf = Aq[q] + Bq[q] * kro + prm<Real>(m.q[2], m.f.q[2]) * kr * kr;
              f = prm<Real>(m.a0, m.f.a0) + qf * cv;
            } else {
              f = prm<Real>(m.a0, m.f.a0) * cv;
            }
            const C x = v[(i * CW + q) * RL + r];
            yq[q] = mk(f * x.x, f * x.y);
            if constexpr (FUSED) v[(i * CW + q) * RL + r] = yq[q];
          }
          if constexpr (!FUSED) {
            if constexpr (CW == 2) st_pair(&buf[row * LDS + cg * CW], yq[0], yq[1]);
            else buf[row * LDS + cg] = yq[0];
          }
        }
      }
    }
    if constexpr (!FUSED) {
      // (the forward's last exchange ended with a barrier, so buf was free)
      __syncthreads();
      smem_to_regs<C, N, NCP, CW, NT, E, R0, LDS>(v, buf);
      __syncthreads();
    }
    regs_fft<C, N, NCP, CW, NT, E, LDS, +1, EXACT, 0, 1, FUSED>(v, buf, tw);
  }
  // outputs of the last pass to global memory (rows >= n_store cropped)
#pragma unroll
  for (int i = 0; i < E / (RF * CW); ++i) {
    const int j = (tid + i * NT) / NCP;
#pragma unroll
    for (int r = 0; r < RF; ++r) {
      const int row = j + r * (N / RF);
      if (HALF_OUT && 2 * r >= RF) continue;  // rows >= N/2 are cropped
      if (row >= a.n_store) continue;
      if constexpr (CW == 2) {
        if (vec) {
          st_pair(&colp[0][(long long)row * a.line_stride], v[(i * 2) * RF + r], v[(i * 2 + 1) * RF + r]);
        } else {
#pragma unroll
          for (int q = 0; q < CW; ++q)
            if (my_ok[q]) colp[q][(long long)row * a.line_stride] = v[(i * CW + q) * RF + r];
        }
      } else {
        if (my_ok[0]) colp[0][(long long)row * a.line_stride] = v[i * RF + r];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Float column passes on pairs of adjacent columns (ColCfg::CW == 2) with
// packed two-lane arithmetic (fse_fft_x2.cuh): the same passes, zero halves,
// crops and multipliers as colpass_tile, each scalar operation of one column
// done for both columns of a pair in one instruction. A tile is its geometry
// (X2Geo), the first pass's row loads and the transform itself (x2_compute).
// ---------------------------------------------------------------------------

// This thread's column pair of one tile.
struct X2Geo {
  int plane, c0;
  int my_plane[2], my_px[2];
  bool my_ok[2];
  float2* colp[2];
  bool vec;  // both columns valid, adjacent and 16-byte aligned: one access per row
};

template <int N, int VAR, bool GATHER>
__device__ __forceinline__ void x2_geo(const ColArgs& a, const MulArgs& m, int bid, int ngat, X2Geo& g, int tid) {
  typedef ColCfg<float, N, VAR> K;
  constexpr int NCOL = K::NCOL, NCP = K::NCP;
  const int cg = tid % NCP;  // this thread's columns of the tile: 2 cg, 2 cg + 1
  const int breg = bid - ngat;
  const int tp = GATHER ? 0 : breg / a.tiles_per_plane;
  g.c0 = GATHER ? 0 : (breg - tp * a.tiles_per_plane) * NCOL;
  // kernel-transform pass over a full even set of planes: planes p and lp - p
  // (same |p|, same C^ values) run next to each other, so the octant is read
  // from HBM about once
  g.plane = (VAR == COL_KHAT && m.lp == a.nplanes && (m.lp & 1) == 0 && tp > 0)
                ? ((tp & 1) ? (tp + 1) >> 1 : m.lp - (tp >> 1))
                : tp;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int cc = cg * 2 + q;
    if (!GATHER) {
      g.my_plane[q] = g.plane;
      g.my_px[q] = g.c0 + cc;
      g.my_ok[q] = g.my_px[q] < a.ncols;
    } else {
      const int qq = bid * NCOL + cc;
      g.my_plane[q] = qq / a.tail;
      g.my_px[q] = a.tiles_per_plane * NCOL + qq % a.tail;
      g.my_ok[q] = g.my_plane[q] < a.nplanes;
      if (!g.my_ok[q]) g.my_plane[q] = g.my_px[q] = 0;
    }
    g.colp[q] = (!GATHER && q > 0) ? g.colp[0] + q
                                   : reinterpret_cast<float2*>(a.data) + (long long)g.my_plane[q] * a.plane_stride +
                                         g.my_px[q];
  }
  g.vec = !GATHER && g.my_ok[0] && g.my_ok[1] && (reinterpret_cast<uintptr_t>(g.colp[0]) % 16 == 0) &&
          (a.line_stride % 2 == 0);
}

__device__ __forceinline__ P2 x2_load_row(const ColArgs& a, const X2Geo& g, int row) {
  if (row >= a.n_load) return P2{bc(0.f), bc(0.f)};
  if (g.vec) return p2_from_row(*reinterpret_cast<const float4*>(&g.colp[0][(long long)row * a.line_stride]));
  const float2 z = make_float2(0.f, 0.f);
  const float2 u0 = g.my_ok[0] ? g.colp[0][(long long)row * a.line_stride] : z;
  const float2 u1 = g.my_ok[1] ? g.colp[1][(long long)row * a.line_stride] : z;
  return P2{make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
}

__device__ __forceinline__ void x2_store_row(const ColArgs& a, const X2Geo& g, int row, const P2& v) {
  if (g.vec) {
    *reinterpret_cast<float4*>(&g.colp[0][(long long)row * a.line_stride]) = p2_to_row(v);
  } else {
    if (g.my_ok[0]) g.colp[0][(long long)row * a.line_stride] = make_float2(v.re.x, v.im.x);
    if (g.my_ok[1]) g.colp[1][(long long)row * a.line_stride] = make_float2(v.re.y, v.im.y);
  }
}

// Row of the first-pass input c of this thread (items i, radix index r; the
// zero half of a padded line is never read), c < ColCfg::first(VAR).
template <int N, int VAR> __device__ __forceinline__ int x2_first_row(int c, int tid) {
  typedef ColCfg<float, N, VAR> K;
  constexpr int RH = K::rh(VAR);
  const int i = c / RH, r = c % RH;
  return (tid + i * K::NT) / K::NCP + r * (N / K::R0);
}

// The first pass's inputs into registers, straight from global memory.
template <int N, int VAR>
__device__ __forceinline__ void x2_first_loads(const ColArgs& a, const X2Geo& g, P2 (&v)[ColCfg<float, N, VAR>::E / 2],
                                               int tid) {
  typedef ColCfg<float, N, VAR> K;
  constexpr int RH = K::rh(VAR), R0 = K::R0;
#pragma unroll
  for (int c = 0; c < K::first(VAR); ++c) {
    const int i = c / RH, r = c % RH;
    v[i * R0 + r] = x2_load_row(a, g, x2_first_row<N, VAR>(c, tid));
  }
}

// Starts the cp.async copies of the tile's C^ values (|p_row| = 0..N/2) into
// shared memory (the caller commits the group).
template <int N, int VAR, bool GATHER>
__device__ __forceinline__ void x2_chat_issue(const ColArgs& a, const MulArgs& m, const X2Geo& g, int bid,
                                              float* sC, int tid) {
  typedef ColCfg<float, N, VAR> K;
  constexpr int NCOL = K::NCOL, NT = K::NT;
  const float* ch = reinterpret_cast<const float*>(m.chat);
  if (!GATHER) {
    // the tile's columns of a C^ row are contiguous and 16-byte aligned (rows
    // padded to a multiple of 4 values, c0 a multiple of NCOL): one 16-byte
    // copy per 4 values; copies past the padded row are zero-filled
    constexpr int CPR = NCOL / 4;
    const float* chp = ch + (m.lp ? (long long)abs(wrap_index(g.plane, m.lp)) * m.chat_sp : 0) + g.c0;
    const int left = m.chat_cx - g.c0;
    for (int idx = tid; idx < (N / 2 + 1) * CPR; idx += NT) {
      const int ar = idx / CPR, qd = idx - ar * CPR;
      float* dst = &sC[ar * NCOL + qd * 4];
      if (qd * 4 < left) cp_async<16>(dst, &chp[(long long)ar * m.chat_sr + qd * 4]);
      else *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  } else {
    for (int idx = tid; idx < (N / 2 + 1) * NCOL; idx += NT) {
      const int ar = idx / NCOL, cc = idx % NCOL;
      const int qq = bid * NCOL + cc;
      const int pl = qq / a.tail, px = a.tiles_per_plane * NCOL + qq % a.tail;
      const int ap = m.lp ? abs(wrap_index(pl, m.lp)) : 0;
      if (pl < a.nplanes && px <= (m.lx >> 1))
        cp_async<4>(&sC[idx], &ch[(long long)ar * m.chat_sr + (long long)ap * m.chat_sp + px]);
      else
        sC[idx] = 0.f;
    }
  }
}

// Transform, multiplier, inverse transform and stores of one tile whose
// first-pass inputs are in v. For the kernel-transform variant the tile's C^
// copies are the second most recent cp.async group of this thread.
template <int N, int VAR>
__device__ __forceinline__ void x2_compute(const ColArgs& a, const MulArgs& m, const float2* __restrict__ tw,
                                           const X2Geo& g, P2 (&v)[ColCfg<float, N, VAR>::E / 2], int tid) {
  typedef ColCfg<float, N, VAR> K;
  constexpr int NCOL = K::NCOL, NCP = K::NCP, LDS = K::LDS, NT = K::NT, W = K::E / 2;
  constexpr int R0 = K::R0, RL = K::RL;
  constexpr bool FUSED = (VAR == COL_KIN || VAR == COL_KHAT) && plan_palindrome(N);
  constexpr int RF = FUSED ? R0 : RL;
  constexpr bool HALF_IN = (VAR == COL_PADF || VAR == COL_KHAT);
  constexpr bool HALF_OUT = (VAR == COL_CROPI || VAR == COL_KHAT);
  constexpr bool EXACT = (VAR == COL_FWD || VAR == COL_INV || VAR == COL_KIN);
  constexpr int DIR1 = (VAR == COL_INV || VAR == COL_CROPI) ? +1 : -1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  const float* sC = reinterpret_cast<const float*>(smem_raw + K::TILE_BYTES);
  const float4* twb = twb_of<N>(tw);
  const int cg = tid % NCP;
  if constexpr (VAR == COL_FWD || VAR == COL_INV || VAR == COL_PADF || VAR == COL_CROPI) {
    pregs_fft<N, NCP, NT, W, LDS, DIR1, EXACT, 0, 1, false, HALF_IN>(v, buf, twb, tid);
  } else {
    pregs_fft<N, NCP, NT, W, LDS, -1, EXACT, 0, 1, false, HALF_IN>(v, buf, twb, tid);
    if constexpr (VAR == COL_KIN) {
      // kinetic phase exp(-i f theta_k) of both columns from the octant table,
      // its modulus error folded into the products (unit_mul), times 1/N
      const float2* tab[2];
      int ax[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        tab[q] = reinterpret_cast<const float2*>(m.kin) +
                 (m.lp ? (long long)abs(wrap_index(g.my_plane[q], m.lp)) * m.kin_sp : 0);
        ax[q] = abs(wrap_index(min(g.my_px[q], m.lx - 1), m.lx));
      }
      const float2 sc = bc(m.f.scale);
      const bool conj = m.conj != 0;
#pragma unroll
      for (int i = 0; i < W / RL; ++i) {
        const int j = (tid + i * NT) / NCP;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int row = j + r * (N / RL);
          const long long ro = (long long)abs(wrap_index(row, m.lr)) * m.kin_sr;
          const float2 t0 = g.my_ok[0] ? __ldg(&tab[0][ro + ax[0]]) : make_float2(1.f, 0.f);
          const float2 t1 = g.my_ok[1] ? __ldg(&tab[1][ro + ax[1]]) : make_float2(1.f, 0.f);
          // factor c + i s (conjugated for the adjoint) with its modulus remainder h (c + i s)
          const float2 c2 = make_float2(t0.x, t1.x);
          const float2 s2 = conj ? make_float2(-t0.y, -t1.y) : make_float2(t0.y, t1.y);
          const float2 h2 = make_float2(-0.5f * norm_err(t0.x, t0.y), -0.5f * norm_err(t1.x, t1.y));
          const float2 lc = mul2(h2, c2), ls = mul2(h2, s2);
          const P2 x = v[i * RL + r];
          const float2 lr = fma2(x.re, lc, mul2(x.im, neg2(ls)));
          const float2 li = fma2(x.re, ls, mul2(x.im, lc));
          const float2 yr = fma2(x.re, c2, fma2(x.im, neg2(s2), lr));
          const float2 yi = fma2(x.re, s2, fma2(x.im, c2, li));
          const P2 y{mul2(sc, yr), mul2(sc, yi)};
          if constexpr (FUSED) v[i * RL + r] = y;
          else p2_st(&buf[row * LDS + 2 * cg], y);
        }
      }
    } else {
      // kernel transform on the padded grid: f = a0 C^ (Coulomb) or a0 + (k^T Q k) C^ (DDI);
      // the column (x, an R2C bin 0..nx) and plane factors are fixed per thread
      cp_async_wait_group<1>();
      __syncthreads();
      const bool ddi = m.mode == MUL_DDI;
      float Aq[2], Bq[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float kp = m.lp ? m.f.dkp * float(wrap_index(g.my_plane[q], m.lp)) : 0.f;
        const float kpo = (m.lp && 2 * g.my_plane[q] == m.lp) ? 0.f : kp;
        const float kx = m.f.dkx * float(g.my_px[q]);
        const float kxo = (2 * g.my_px[q] == m.lx) ? 0.f : kx;
        Aq[q] = m.f.q[0] * kx * kx + m.f.q[1] * kp * kp + m.f.q[3] * kxo * kpo;
        Bq[q] = m.f.q[4] * kxo + m.f.q[5] * kpo;
      }
      const float2 A2 = make_float2(Aq[0], Aq[1]), B2 = make_float2(Bq[0], Bq[1]);
      const float2 a02 = bc(m.f.a0);
#pragma unroll
      for (int i = 0; i < W / RL; ++i) {
        const int j = (tid + i * NT) / NCP;
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int row = j + r * (N / RL);
          const int pr = wrap_index(row, m.lr);
          const float kr = m.f.dkr * float(pr);
          const float kro = (2 * row == m.lr) ? 0.f : kr;
          const float2 cv = *reinterpret_cast<const float2*>(&sC[abs(pr) * NCOL + 2 * cg]);
          // f = a0 + q(k) C^ with q(k) = A + B kr + q2 kr^2 (DDI), or a0 C^
          const float2 f = ddi ? fma2(fma2(B2, bc(kro), add2(A2, bc(m.f.q[2] * kr * kr))), cv, a02) : mul2(a02, cv);
          const P2 x = v[i * RL + r];
          const P2 y{mul2(f, x.re), mul2(f, x.im)};
          if constexpr (FUSED) v[i * RL + r] = y;
          else p2_st(&buf[row * LDS + 2 * cg], y);
        }
      }
    }
    if constexpr (!FUSED) {
      __syncthreads();
      psmem_to_regs<N, NCP, NT, W, R0, LDS>(v, buf, tid);
      __syncthreads();
    }
    pregs_fft<N, NCP, NT, W, LDS, +1, EXACT, 0, 1, FUSED>(v, buf, twb, tid);
  }
  // outputs of the last pass to global memory (rows >= n_store cropped)
#pragma unroll
  for (int i = 0; i < W / RF; ++i) {
    const int j = (tid + i * NT) / NCP;
#pragma unroll
    for (int r = 0; r < RF; ++r) {
      const int row = j + r * (N / RF);
      if (HALF_OUT && 2 * r >= RF) continue;  // rows >= N/2 are cropped
      if (row >= a.n_store) continue;
      x2_store_row(a, g, row, v[i * RF + r]);
    }
  }
}

// One tile (block bid).
template <int N, int VAR, bool GATHER>
__device__ __forceinline__ void colpass_tile_x2(const ColArgs& a, const MulArgs& m, const float2* __restrict__ tw,
                                                int bid, int ngat) {
  typedef ColCfg<float, N, VAR> K;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  X2Geo g;
  x2_geo<N, VAR, GATHER>(a, m, bid, ngat, g, tid);
  if constexpr (VAR == COL_KHAT) {
    x2_chat_issue<N, VAR, GATHER>(a, m, g, bid, reinterpret_cast<float*>(smem_raw + K::TILE_BYTES), tid);
    cp_async_commit();
  }
  cp_async_commit();  // an empty group: the C^ copies are the second most recent
  P2 v[K::E / 2];
  x2_first_loads<N, VAR>(a, g, v, tid);
  x2_compute<N, VAR>(a, m, tw, g, v, tid);
}

// One tile of a column pass (block bid): float plans take the packed
// column-pair path (colpass_tile_x2), float64 plans the one-column path
// (colpass_tile). Passes over R2C bins gather the bin n_x of all planes into
// the first tiles of the grid.
template <typename Real, int N, int VAR>
__device__ __forceinline__ void colpass_body(const ColArgs& a, const MulArgs& m,
                                             const typename Cplx<Real>::T* __restrict__ tw, int bid) {
  // only passes over R2C bins (ncols = nx + 1) have tail tiles; they come
  // first in the grid, so that they overlap the full tiles
  constexpr bool TAILS = (VAR == COL_PADF || VAR == COL_CROPI || VAR == COL_KHAT);
  constexpr bool X2 = ColCfg<Real, N, VAR>::CW == 2;  // float pairs: packed arithmetic
  constexpr int NCOL = ColCfg<Real, N, VAR>::NCOL;
  const int ngat = (TAILS && a.tail > 0) ? (a.nplanes * a.tail + NCOL - 1) / NCOL : 0;
  if constexpr (X2 && TAILS) {
    if (bid < ngat) colpass_tile_x2<N, VAR, true>(a, m, tw, bid, ngat);
    else colpass_tile_x2<N, VAR, false>(a, m, tw, bid, ngat);
  } else if constexpr (X2) {
    colpass_tile_x2<N, VAR, false>(a, m, tw, bid, 0);
  } else if constexpr (TAILS) {
    if (bid < ngat) colpass_tile<Real, N, VAR, true>(a, m, tw, bid, ngat);
    else colpass_tile<Real, N, VAR, false>(a, m, tw, bid, ngat);
  } else {
    colpass_tile<Real, N, VAR, false>(a, m, tw, bid, 0);
  }
}

template <typename Real, int N, int VAR>
__global__ void __launch_bounds__(ColCfg<Real, N, VAR>::NT, ColCfg<Real, N, VAR>::MINB)
k_colpass(ColArgs a, MulArgs m, const typename Cplx<Real>::T* __restrict__ tw) {
  pass_prologue();
  colpass_body<Real, N, VAR>(a, m, tw, blockIdx.x);
}

// ---------------------------------------------------------------------------
// x passes over tiles of NCOL consecutive lines (rows of psi). A tile is
// transposed into shared memory (column layout, LDS = NCOL + 1) so that one
// Stockham routine serves every axis; the real density is handled as two
// lines packed into one complex line.
// ---------------------------------------------------------------------------
template <typename Real, int NX>
struct XCfg {
  typedef typename Cplx<Real>::T C;
  static constexpr int NCOL = ncol_for(2 * NX, sizeof(C)) < 2 ? 2 : ncol_for(2 * NX, sizeof(C));
  static constexpr int NT = 256;
  static constexpr int LDS = NCOL + 1;
  // the R2C / C2R of two real lines per complex line works on NCOL / 2
  // lines of length 2 NX; with 8 of them it uses the swizzled tile layout
  static constexpr bool SWZ2 = (NCOL / 2 == 8);
  static constexpr int LDS2 = tile_ld<NCOL / 2, SWZ2>();
  __device__ __forceinline__ static int pk(int row, int q) { return tile_at<NCOL / 2, SWZ2>(row, q); }
  static constexpr int TOT = NCOL * NX;
  static constexpr int PER = (TOT + NT - 1) / NT;
  static constexpr int MINB = sizeof(Real) == 4 ? 4 : 2;
  __host__ __device__ static constexpr size_t smem_bytes() {
    return sizeof(C) * (size_t)((NX * LDS) > (2 * NX * LDS2) ? (NX * LDS) : (2 * NX * LDS2));
  }
};

// Line l0 + q of a tile -> its (y, z) indices, from y0 = l0 % ny and
// z0 = l0 / ny (one division per tile rather than one per element).
__device__ __forceinline__ void line_yz(int y0, int z0, int q, int ny, int& y, int& z) {
  y = y0 + q;
  z = z0;
  while (y >= ny) {
    y -= ny;
    ++z;
  }
}

// Row of S holding the x-half-spectrum of line l0 + q (S rows: mul * ny per z).
__device__ __forceinline__ long long srow(int y0, int z0, int q, int ny, int mul) {
  int y, z;
  line_yz(y0, z0, q, ny, y, z);
  return (long long)z * (mul * ny) + y;
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
  constexpr int NCOL = K::NCOL, NT = K::NT, TOT = K::TOT, PER = K::PER;
  const int tid = threadIdx.x;
  C* S = reinterpret_cast<C*>(a.spec);
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int idx = tid + it * NT;
    if ((TOT % NT) == 0 || idx < TOT) {
      const int l = idx / NX, x = idx % NX;
      reinterpret_cast<Real*>(&buf[K::pk(x, l >> 1)])[l & 1] = val[it];
    }
  }
  // Rows NX..2NX-1 are the zero padding. With an even first radix the first
  // pass reads none of them (it takes them as zero); with radix 3 it reads rows
  // 2NX/3..4NX/3-1, part of which lie there, so those are zero-filled first.
  if constexpr (radix_plan(2 * NX).r[0] % 2 != 0) {
    for (int idx = tid; idx < (NCOL / 2) * NX; idx += NT) {
      const int q = idx / NX, x = NX + idx % NX;
      buf[K::pk(x, q)] = mk(Real(0), Real(0));
    }
  }
  __syncthreads();
  fft_tile<C, 2 * NX, NCOL / 2, NT, -1, false, true, false, K::SWZ2>(buf, tw2n);
  const int z0 = l0 / a.ny, y0 = l0 - z0 * a.ny;
  constexpr int NH = (NCOL / 2) * (NX + 1), PH = (NH + NT - 1) / NT;
#pragma unroll
  for (int it = 0; it < PH; ++it) {
    const int idx = tid + it * NT;
    if (idx < NH) {
      const int q = idx / (NX + 1), k = idx % (NX + 1);
      const C zk = buf[K::pk(k, q)];
      const C zm = buf[K::pk((2 * NX - k) % (2 * NX), q)];
      const int la = l0 + 2 * q;
      const C A = mk(Real(0.5) * (zk.x + zm.x), Real(0.5) * (zk.y - zm.y));
      const C B = mk(Real(0.5) * (zk.y + zm.y), Real(0.5) * (zm.x - zk.x));
      if (la < a.nlines) S[srow(y0, z0, 2 * q, a.ny, a.srow_mul) * a.sx + k] = A;
      if (la + 1 < a.nlines) S[srow(y0, z0, 2 * q + 1, a.ny, a.srow_mul) * a.sx + k] = B;
    }
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
  constexpr int NCOL = K::NCOL, NT = K::NT, TOT = K::TOT, PER = K::PER;
  const int tid = threadIdx.x;
  const C* S = reinterpret_cast<const C*>(a.spec);
  const int z0 = l0 / a.ny, y0 = l0 - z0 * a.ny;
  constexpr int NH = (NCOL / 2) * (NX + 1), PH = (NH + NT - 1) / NT;
#pragma unroll
  for (int it = 0; it < PH; ++it) {
    const int idx = tid + it * NT;
    if (idx < NH) {
      const int q = idx / (NX + 1), k = idx % (NX + 1);
      const int la = l0 + 2 * q;
      C A = mk(Real(0), Real(0)), B = A;
      if (la < a.nlines) A = S[srow(y0, z0, 2 * q, a.ny, a.srow_mul) * a.sx + k];
      if (la + 1 < a.nlines) B = S[srow(y0, z0, 2 * q + 1, a.ny, a.srow_mul) * a.sx + k];
      buf[K::pk(k, q)] = mk(A.x - B.y, A.y + B.x);
      if (k > 0 && k < NX) buf[K::pk(2 * NX - k, q)] = mk(A.x + B.y, B.x - A.y);
    }
  }
  __syncthreads();
  // only rows 0..NX-1 survive the crop: the last pass stores no others
  fft_tile<C, 2 * NX, NCOL / 2, NT, +1, false, false, true, K::SWZ2>(buf, tw2n);
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int idx = tid + it * NT;
    val[it] = Real(0);
    if ((TOT % NT) == 0 || idx < TOT) {
      const int l = idx / NX, x = idx % NX;
      const C z = buf[K::pk(x, l >> 1)];
      val[it] = (l & 1) ? z.y : z.x;
    }
  }
}

// sin and cos of a potential phase. For |th| <= 1/2 the Taylor series to
// th^9 / th^8 (truncation below 3e-10) in Horner form; sincos otherwise.
__device__ __forceinline__ void phase_sincos(float th, float* sn, float* cs) {
  if (fabsf(th) <= 0.5f) {
    const float t2 = th * th;
    const float ps = fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 1.0f / 362880.0f, -1.0f / 5040.0f), 1.0f / 120.0f), -1.0f / 6.0f), 0.0f);
    const float pc = fmaf(t2, fmaf(t2, fmaf(t2, fmaf(t2, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f), -0.5f), 0.0f);
    *sn = fmaf(th, ps, th);
    *cs = 1.0f + pc;
  } else {
    sincosf(th, sn, cs);
  }
}
__device__ __forceinline__ void phase_sincos(double th, double* sn, double* cs) { sincos(th, sn, cs); }

template <typename Real>
__device__ __forceinline__ Real sin_sq(Real v);
template <> __device__ __forceinline__ float sin_sq(float v) {
  const float s = sinf(v);
  return s * s;
}
template <> __device__ __forceinline__ double sin_sq(double v) {
  const double s = sin(v);
  return s * s;
}

// Window integral of the optical lattice at the point (X, Y, Z) of the rotating
// frame (Gauss-Legendre nodes of the window in a.lat_*).
template <typename Real>
__device__ __noinline__ Real lattice_integral(const XArgs& a, Real X, Real Y, Real Z) {
  const Real kx = prm<Real>(a.lat_k[0], a.f.lat_k[0]), ky = prm<Real>(a.lat_k[1], a.f.lat_k[1]);
  const Real kz = prm<Real>(a.lat_k[2], a.f.lat_k[2]);
  const Real zt = kz != Real(0) ? sin_sq(kz * Z) : Real(0);
  Real acc = Real(0);
  for (int q = 0; q < a.lat_nq; ++q) {
    const Real c = prm<Real>(a.lat_c[q], a.f.lat_c[q]), s = prm<Real>(a.lat_s[q], a.f.lat_s[q]);
    const Real xr = c * X + s * Y, yr = -s * X + c * Y;
    acc += prm<Real>(a.lat_w[q], a.f.lat_w[q]) * (sin_sq(kx * xr) + sin_sq(ky * yr) + zt);
  }
  return prm<Real>(a.lat_amp, a.f.lat_amp) * acc;
}

// Rounded products and fused multiply-adds that the compiler does not
// re-associate or contract, so that every kernel that inlines an expression
// built from them (the single-run and the batched passes) computes the same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// P at grid point (x, y, z): the harmonic quadratic form plus, with LAT = 1,
// the optical lattice (LAT = 2: when lat_amp != 0, decided at run time). The
// evaluation order is fixed: X = lo + h x, P = ((pa X X + pb Y Y) + pc X Y) + pe Z Z.
template <typename Real, int LAT>
__device__ __forceinline__ Real trap_phase(const XArgs& a, int x, int y, int z) {
  const Real X = fma_rn(prm<Real>(a.h0, a.f.h0), Real(x), prm<Real>(a.lo0, a.f.lo0));
  const Real Y = fma_rn(prm<Real>(a.h1, a.f.h1), Real(y), prm<Real>(a.lo1, a.f.lo1));
  const Real Z = fma_rn(prm<Real>(a.h2, a.f.h2), Real(z), prm<Real>(a.lo2, a.f.lo2));
  Real P = mul_rn(mul_rn(prm<Real>(a.pa, a.f.pa), X), X);
  P = fma_rn(mul_rn(prm<Real>(a.pb, a.f.pb), Y), Y, P);
  P = fma_rn(mul_rn(prm<Real>(a.pc, a.f.pc), X), Y, P);
  P = fma_rn(mul_rn(prm<Real>(a.pe, a.f.pe), Z), Z, P);
  if (LAT == 1 || (LAT == 2 && prm<Real>(a.lat_amp, a.f.lat_amp) != Real(0)))
    return add_rn(P, lattice_integral<Real>(a, X, Y, Z));
  return P;
}

template <typename Real, int NX, int KIND>
__device__ __forceinline__ void xpass_body(const XArgs& a, const typename Cplx<Real>::T* __restrict__ twn,
                                           const typename Cplx<Real>::T* __restrict__ tw2n, int bid) {
  typedef XCfg<Real, NX> K;
  typedef typename K::C C;
  constexpr int NCOL = K::NCOL, NT = K::NT, LDS = K::LDS, TOT = K::TOT, PER = K::PER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int tid = threadIdx.x;
  const int l0 = bid * NCOL;
  const int z0 = l0 / a.ny, y0 = l0 - z0 * a.ny;  // (y, z) of the tile's first line
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
    fft_tile<C, NX, NCOL, NT, (KIND == XP_FWD ? -1 : +1), true>(buf, twn);
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
        if (tid == 0) a.part[bid] = acc;
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
          int yl, zl;
          line_yz(y0, z0, l, a.ny, yl, zl);
          const long long o = (long long)lg * NX + x;
          const C u = u1p[o];
          const C g = psi[o];
          const Real th = prm<Real>(a.beta_dt, a.f.beta_dt) * (u.x * u.x + u.y * u.y) + prm<Real>(a.lam, a.f.lam) * vphi[it] +
                           trap_phase<Real, 2>(a, x, yl, zl);
          Real sn, cs;
          sincos(th, &sn, &cs);
          const C u2 = mk(u.x * cs + u.y * sn, u.y * cs - u.x * sn);
          const Real r = g.x * u2.y - g.y * u2.x;
          rr[it] = r;
          psi[o] = mk(g.x * cs - g.y * sn, g.y * cs + g.x * sn);
          const double X = a.lo0 + a.h0 * x, Y = a.lo1 + a.h1 * yl, Z = a.lo2 + a.h2 * zl;
          dg0 += (double)r * (a.dp[0] * X * X + a.dp[1] * Y * Y + a.dp[2] * X * Y + a.dp[3] * Z * Z);
          dg1 += (double)r * (a.dp[4] * X * X + a.dp[5] * Y * Y + a.dp[6] * X * Y + a.dp[7] * Z * Z);
          dg2 += (double)r * (a.dp[8] * X * X + a.dp[9] * Y * Y + a.dp[10] * X * Y + a.dp[11] * Z * Z);
        }
      }
    }
    if (a.part) {
      dg0 = block_sum(dg0, red);
      if (tid == 0) a.part[bid] = dg0;
      dg1 = block_sum(dg1, red);
      if (tid == 0) a.part[a.part_stride + bid] = dg1;
      dg2 = block_sum(dg2, red);
      if (tid == 0) a.part[2 * a.part_stride + bid] = dg2;
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
          const Real q2 = Real(2) * (prm<Real>(a.beta_dt, a.f.beta_dt) * r + prm<Real>(a.lam, a.f.lam) * kr[it]);
          psi[o] = mk(h.x + q2 * u.x, h.y + q2 * u.y);
        }
      }
    }
  } else {
    // XP_A / XP_R: varphi from the cropped C2R of S
    if ((KIND == XP_A || KIND == XP_AL) && tid == 0 && l0 < a.nlines &&
        (reinterpret_cast<uintptr_t>(psi) & 15) == 0) {
      // the tile's rows of psi (contiguous) move to L2 while the C2R runs (the
      // bulk prefetch needs a 16-byte aligned start; psi may be only
      // element-aligned, and every line then starts 16-byte aligned too)
      const int nl = min(NCOL, a.nlines - l0);
      prefetch_l2_bulk(psi + (long long)l0 * NX, (unsigned)(nl * NX * sizeof(C)));
    }
    Real vphi[PER];
#pragma unroll
    for (int it = 0; it < PER; ++it) vphi[it] = Real(0);
    if (a.use_spec) c2r_rows<Real, NX>(a, buf, l0, tw2n, vphi);
    if constexpr (KIND == XP_R) {
      if (a.out) {
        // varphi itself, as a real field in the layout of psi
        Real* phi = reinterpret_cast<Real*>(a.out);
#pragma unroll
        for (int it = 0; it < PER; ++it) {
          const int idx = tid + it * NT;
          if ((TOT % NT) == 0 || idx < TOT) {
            const int l = idx / NX, x = idx % NX;
            if (l0 + l < a.nlines) phi[(long long)(l0 + l) * NX + x] = vphi[it];
          }
        }
      }
      if (!a.part) return;
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
      if (tid == 0) a.part[bid] = acc;
      return;
    } else {
      // optional renormalisation factor, read and converted once per thread: a
      // conversion from double inside the element loop issues on the narrow
      // FP64 pipe for every element, even where the branch is predicated off
      const bool rescale = a.scale != nullptr;
      const Real fsc = rescale ? Real(*a.scale) : Real(1);
      __syncthreads();
#pragma unroll
      for (int it = 0; it < PER; ++it) {
        const int idx = tid + it * NT;
        if ((TOT % NT) == 0 || idx < TOT) {
          const int l = idx / NX, x = idx % NX;
          const int lg = l0 + l;
          C u2 = mk(Real(0), Real(0));
          if (lg < a.nlines) {
            int yl, zl;
            line_yz(y0, z0, l, a.ny, yl, zl);
            const C u = psi[(long long)lg * NX + x];
            const Real rho = u.x * u.x + u.y * u.y;
            const Real th = prm<Real>(a.beta_dt, a.f.beta_dt) * rho + prm<Real>(a.lam, a.f.lam) * vphi[it] +
                             trap_phase<Real, KIND == XP_AL ? 1 : 0>(a, x, yl, zl);
            Real sn, cs;
            phase_sincos(th, &sn, &cs);
            u2 = unit_mul(u, cs, -sn, false);
            if (rescale) u2 = mk(fsc * u2.x, fsc * u2.y);
          }
          buf[x * LDS + l] = u2;
        }
      }
      __syncthreads();
      fft_tile<C, NX, NCOL, NT, -1, true>(buf, twn);
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

}  // namespace fse

#include "fse_xpass_x2.cuh"

namespace fse {

// Whether an x pass takes the packed two-line code (fse_xpass_x2.cuh), and
// the launch shape of either code: lines per tile, threads, resident tiles
// per SM the registers are sized for, dynamic shared memory.
template <typename Real, int NX, int KIND>
struct XLaunch {
  static constexpr bool X2 = sizeof(Real) == 4 && xpass_x2_ok<NX>() &&
                             (KIND == XP_FWD || KIND == XP_INV || KIND == XP_E || KIND == XP_A);
  static constexpr int NCOL = X2 ? XCfg2<(X2 ? NX : 256)>::NCOL : XCfg<Real, NX>::NCOL;
  static constexpr int NT = X2 ? XCfg2<(X2 ? NX : 256)>::NT : XCfg<Real, NX>::NT;
  static constexpr int MINB = X2 ? XCfg2<(X2 ? NX : 256)>::MINB : XCfg<Real, NX>::MINB;
  __host__ __device__ static constexpr size_t smem_bytes() {
    return X2 && XCfg2<(X2 ? NX : 256)>::SMEM > XCfg<Real, NX>::smem_bytes() ? XCfg2<(X2 ? NX : 256)>::SMEM
                                                                              : XCfg<Real, NX>::smem_bytes();
  }
};

// An x pass: the packed two-line code where it applies, the one-line code
// otherwise.
template <typename Real, int NX, int KIND>
__device__ __forceinline__ void xpass_any(const XArgs& a, const typename Cplx<Real>::T* __restrict__ twn,
                                          const typename Cplx<Real>::T* __restrict__ tw2n, int bid) {
  if constexpr (XLaunch<Real, NX, KIND>::X2)
    xpass_body_x2<NX, KIND>(a, twn, tw2n, bid);
  else
    xpass_body<Real, NX, KIND>(a, twn, tw2n, bid);
}

template <typename Real, int NX, int KIND>
__global__ void __launch_bounds__(XLaunch<Real, NX, KIND>::NT, XLaunch<Real, NX, KIND>::MINB)
k_xpass(XArgs a, const typename Cplx<Real>::T* __restrict__ twn, const typename Cplx<Real>::T* __restrict__ tw2n) {
  pass_prologue();
  xpass_any<Real, NX, KIND>(a, twn, tw2n, blockIdx.x);
}

// Host-side launchers (explicitly instantiated per precision).
template <typename Real>
cudaError_t launch_colpass(int N, int var, const ColArgs& a, const MulArgs& m, const void* tw, cudaStream_t st);
template <typename Real>
cudaError_t launch_xpass(int kind, int nx, const XArgs& a, const void* twn, const void* tw2n,
                         cudaStream_t st);
// Lines per tile of the column pass of length N and of the x passes of length
// nx (xpass_ncol: the one-line kinds; xpass_ncol_x2: the kinds X0, XI, E and
// A, which write the renormalisation partials of XI and E per tile).
template <typename Real> int colpass_ncol(int N);
template <typename Real> int xpass_ncol(int nx);
template <typename Real> int xpass_ncol_x2(int nx);

}  // namespace fse

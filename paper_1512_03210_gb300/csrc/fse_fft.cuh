// fse_fft.cuh -- shared-memory Stockham FFT used by every pass of the split step.
//
// The transform along one grid axis is done on a tile of NCOL independent
// lines held in shared memory as buf[j * LDS + c] (j = position along the
// line, c = line within the tile, LDS = NCOL + 1; or a swizzled layout
// without padding for tiles of 8 lines, see tile_at). Each radix-R pass of the
// mixed-radix Stockham autosort algorithm (radices 8, 4, 3, 2) reads R
// elements at stride N/R, applies the twiddles, does an in-register DFT of
// size R and writes the R results at stride Ns; all reads of a pass happen
// before a barrier and all writes after it, so one buffer suffices.
//
// The forward transform is unnormalised, X_k = sum_j x_j exp(-2 pi i jk/N);
// the inverse uses the conjugate twiddles and is also unnormalised (the
// scale 1/N is applied by the pass that owns the spectral multiplier).
// Twiddles come from a table holding at tw[2m] the rounded pair w of
// exp(-2 pi i m/N) (built in float64) and at tw[2m+1] the rounded remainder
// exp(-2 pi i m/N) - w. Transforms of the wave function (EXACT) multiply by
// both terms inside one fma chain, so each product is rounded once from a
// nearly exact twiddle. A rounded pair alone has |w| = 1 + O(1e-8), the same
// for every element that meets the entry in every step; those fixed gains
// add up to a steady drift of the norm (about 5e-8 per step in float32).
// Transforms of the density spectrum (which only sets a phase) use w alone.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fse {

template <typename R> struct Cplx;
template <> struct Cplx<float> { typedef float2 T; };
template <> struct Cplx<double> { typedef double2 T; };

__device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
// multiply by -i (DIR < 0) or +i (DIR > 0)
template <int DIR, typename C> __device__ __forceinline__ C mul_i(C a) {
  return DIR < 0 ? mk(a.y, -a.x) : mk(-a.y, a.x);
}

// Asynchronous 4/8/16-byte global -> shared copy (cp.async, completes in the
// background) and the wait for all of a thread's outstanding copies.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async size");
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (BYTES == 16)  // 16-byte copies bypass L1 (.cg): the data is streamed once
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N committed groups of this thread are still in flight
template <int N> __device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
// Bulk prefetch of a contiguous global range into L2 (address and size
// multiples of 16 bytes); no completion to wait for.
__device__ __forceinline__ void prefetch_l2_bulk(const void* gmem, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(gmem), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------
// Radix plans: N = 2^a 3^b (b <= 1) split into passes of radix 3, 8, 4, 2.
// ---------------------------------------------------------------------------
struct RadixPlan {
  int npass;
  int r[8];
};

__host__ __device__ constexpr RadixPlan radix_plan(int N) {
  RadixPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0}};
  int m = N, a = 0;
  while (m % 2 == 0) { m /= 2; ++a; }
  if (m == 3) p.r[p.npass++] = 3;
  int q = a / 3, rem = a % 3;
  if (rem == 0) {
    for (int i = 0; i < q; ++i) p.r[p.npass++] = 8;
  } else if (rem == 1) {
    if (q >= 1) {
      for (int i = 0; i < q - 1; ++i) p.r[p.npass++] = 8;
      p.r[p.npass++] = 4;
      p.r[p.npass++] = 4;
    } else {
      p.r[p.npass++] = 2;
    }
  } else {
    for (int i = 0; i < q; ++i) p.r[p.npass++] = 8;
    p.r[p.npass++] = 4;
  }
  return p;
}

__host__ __device__ constexpr bool fft_size_ok(int N) {
  int m = N;
  while (m % 2 == 0) m /= 2;
  return N >= 4 && (m == 1 || m == 3);
}

// ---------------------------------------------------------------------------
// In-register DFTs of size R. DIR = -1 forward, +1 inverse.
// ---------------------------------------------------------------------------
// ZH (dft2, dft4, dft8, and dft3 below): the inputs of the second half are
// zero and are not read.
template <int DIR, bool ZH = false, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  if constexpr (ZH) {
    b = a;
  } else {
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
  }
}

template <int DIR, bool ZH = false, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  C s02, d02, s13, d13;
  if constexpr (ZH) {
    s02 = a0;
    d02 = a0;
    s13 = a1;
    d13 = mul_i<DIR>(a1);
  } else {
    s02 = cadd(a0, a2);
    d02 = csub(a0, a2);
    s13 = cadd(a1, a3);
    d13 = mul_i<DIR>(csub(a1, a3));
  }
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

// Irrational butterfly constants as a head + tail pair, so that a product
// x * c is rounded once from its exact value (fma(x, head, x * tail)). With a
// single rounded float constant every radix-8 (or radix-3) pass would scale
// half of its outputs by the same |1 + eps| and the norm of the field would
// drift by ~1e-8 per pass, always in the same direction.
template <typename R> struct Kc;
template <> struct Kc<float> {
  static constexpr double kH = 0.70710678118654752440084436210484904;  // sqrt(1/2)
  static constexpr double kS = 0.86602540378443864676372317075293618;  // sqrt(3)/2
  static constexpr float h1 = (float)kH;
  static constexpr float h2 = (float)(kH - (double)(float)kH);
  static constexpr float s1 = (float)kS;
  static constexpr float s2 = (float)(kS - (double)(float)kS);
};
template <> struct Kc<double> {
  static constexpr double h1 = 0.70710678118654752440084436210484904, h2 = 0.0;
  static constexpr double s1 = 0.86602540378443864676372317075293618, s2 = 0.0;
};
__device__ __forceinline__ float mulk(float x, float k1, float k2) { return fmaf(x, k1, x * k2); }
__device__ __forceinline__ double mulk(double x, double k1, double) { return x * k1; }

// Product by a butterfly constant: two-term (EXACT) or the rounded head alone.
template <bool EXACT, typename R> __device__ __forceinline__ R kmul(R x, R k1, R k2) {
  if constexpr (EXACT) return mulk(x, k1, k2);
  else return x * k1;
}

// ZH: a2 is zero and not read (half of a zero-padded line). The zero inputs of
// the ZH forms are left out rather than added: x + 0 is not folded by the
// compiler (it would change the sign of a zero), so the sums would be issued.
template <int DIR, bool EXACT, bool ZH = false, typename C>
__device__ __forceinline__ void dft3(C& a0, C& a1, C& a2) {
  typedef decltype(a0.x) R;
  const R c = R(-0.5);
  C t, d;
  if constexpr (ZH) {
    t = a1;
    d = a1;
  } else {
    t = cadd(a1, a2);
    d = csub(a1, a2);
  }
  C m = mk(a0.x + c * t.x, a0.y + c * t.y);
  // i * DIR * sin(2 pi/3) * (a1 - a2): exp(DIR 2 pi i/3) = c + i DIR sin(2 pi/3)
  const R sy = kmul<EXACT>(d.y, Kc<R>::s1, Kc<R>::s2), sx = kmul<EXACT>(d.x, Kc<R>::s1, Kc<R>::s2);
  C e = DIR < 0 ? mk(sy, -sx) : mk(-sy, sx);
  a0 = cadd(a0, t);
  a1 = cadd(m, e);
  a2 = csub(m, e);
}

template <int DIR, bool EXACT, bool ZH = false, typename C> __device__ __forceinline__ void dft8(C* v) {
  typedef decltype(v[0].x) R;
  // even / odd halves (with ZH, v[4..7] = 0 is the second half of each)
  dft4<DIR, ZH>(v[0], v[2], v[4], v[6]);
  dft4<DIR, ZH>(v[1], v[3], v[5], v[7]);
  // twiddle odd half by w8^k, w8 = exp(DIR i pi/4):
  // w8^1 = h (1 + DIR i); w8^2 = DIR i; w8^3 = h (-1 + DIR i), h = sqrt(1/2)
  C o1 = v[3], o2 = v[5], o3 = v[7];
  const R a1 = o1.x - R(DIR) * o1.y, b1 = o1.y + R(DIR) * o1.x;
  const R a3 = -o3.x - R(DIR) * o3.y, b3 = -o3.y + R(DIR) * o3.x;
  C t1 = mk(kmul<EXACT>(a1, Kc<R>::h1, Kc<R>::h2), kmul<EXACT>(b1, Kc<R>::h1, Kc<R>::h2));
  C t2 = mul_i<DIR>(o2);
  C t3 = mk(kmul<EXACT>(a3, Kc<R>::h1, Kc<R>::h2), kmul<EXACT>(b3, Kc<R>::h1, Kc<R>::h2));
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1);
  v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2);
  v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3);
  v[7] = csub(e3, t3);
}

// EXACT = false drops the tails of the irrational constants (transforms of the
// density and potential, where a fixed 1e-8 scale error is harmless).
// ZH: inputs r with 2 r >= R are zero and are not read.
template <int R, int DIR, bool EXACT = true, bool ZH = false, typename C> __device__ __forceinline__ void dft(C* v) {
  if constexpr (R == 2) {
    dft2<DIR, ZH>(v[0], v[1]);
  } else if constexpr (R == 3) {
    dft3<DIR, EXACT, ZH>(v[0], v[1], v[2]);
  } else if constexpr (R == 4) {
    dft4<DIR, ZH>(v[0], v[1], v[2], v[3]);
  } else {
    static_assert(R == 8, "radix");
    dft8<DIR, EXACT, ZH>(v);
  }
}

// Error of the modulus of a float pair, c^2 + s^2 - 1, computed exactly enough
// to correct it: the two squares are split into rounded product plus fma
// remainder, and the larger square minus one is exact (Sterbenz).
__device__ __forceinline__ float norm_err(float c, float s) {
  const bool big = fabsf(c) >= fabsf(s);
  const float a = big ? c : s, b = big ? s : c;
  const float pa = a * a, ea = fmaf(a, a, -pa);
  const float pb = b * b, eb = fmaf(b, b, -pb);
  return ((pa - 1.0f) + pb) + (ea + eb);
}

// Twiddle m of the table: rounded pair w and its remainder l (EXACT float path;
// otherwise l = w unused). The transforms multiply with twiddle_apply,
// conjugated for the inverse transform.
template <bool EXACT, typename C>
__device__ __forceinline__ void twiddle_load(const C* __restrict__ tw, int m, C& w, C& l) {
  w = __ldg(&tw[2 * m]);
  if constexpr (EXACT && sizeof(C) == 8) l = __ldg(&tw[2 * m + 1]);
  else l = w;
}
template <int DIR, bool EXACT, typename C>
__device__ __forceinline__ C twiddle_apply(C v, C w, C l) {
  if constexpr (EXACT && sizeof(C) == 8) {
    if constexpr (DIR < 0) {
      const float lr = v.x * l.x - v.y * l.y, li = v.x * l.y + v.y * l.x;
      return mk(fmaf(v.x, w.x, fmaf(-v.y, w.y, lr)), fmaf(v.x, w.y, fmaf(v.y, w.x, li)));
    } else {
      const float lr = v.x * l.x + v.y * l.y, li = v.y * l.x - v.x * l.y;
      return mk(fmaf(v.x, w.x, fmaf(v.y, w.y, lr)), fmaf(-v.x, w.y, fmaf(v.y, w.x, li)));
    }
  } else {
    return DIR < 0 ? cmul(v, w) : cmulc(v, w);
  }
}

// v times twiddle m of the table (conjugated for the inverse transform).
template <int DIR, bool EXACT, typename C>
__device__ __forceinline__ C twiddle_mul(C v, const C* __restrict__ tw, int m) {
  C w, l;
  twiddle_load<EXACT>(tw, m, w, l);
  return twiddle_apply<DIR, EXACT>(v, w, l);
}

// v times the float pair (c, s) of a unit-modulus factor, with the pair's
// modulus error folded into the products before their final rounding (the
// factor's remainder is taken as -(|w|^2 - 1)/2 w from norm_err).
__device__ __forceinline__ float2 unit_mul(float2 v, float c, float s, bool conj_w) {
  const float h = -0.5f * norm_err(c, s);
  const float lc = h * c, ls = conj_w ? -h * s : h * s;
  const float sc = conj_w ? -s : s;
  const float lr = v.x * lc - v.y * ls, li = v.x * ls + v.y * lc;
  return make_float2(fmaf(v.x, c, fmaf(-v.y, sc, lr)), fmaf(v.x, sc, fmaf(v.y, c, li)));
}
__device__ __forceinline__ double2 unit_mul(double2 v, double c, double s, bool conj_w) {
  const double sc = conj_w ? -s : s;
  return make_double2(v.x * c - v.y * sc, v.x * sc + v.y * c);
}

// Element (row, c) of a shared-memory tile of NCOL lines. The plain layout
// pads rows to NCOL + 1 elements. The swizzled one (SWZ, for NCOL = 8) keeps
// rows of NCOL elements and stores column c at c ^ ((row >> 1) & 7): the four
// consecutive rows that a warp's 32 items touch in a Stockham pass then cover
// every bank twice, where the padded layout of 9 put up to three accesses on
// one bank.
template <int NCOL, bool SWZ>
__host__ __device__ constexpr int tile_ld() {
  return SWZ ? NCOL : NCOL + 1;
}
template <int NCOL, bool SWZ>
__device__ __forceinline__ int tile_at(int row, int c) {
  static_assert(!SWZ || NCOL == 8, "the swizzled layout is for tiles of 8 lines");
  if constexpr (SWZ) return row * NCOL + (c ^ ((row >> 1) & 7));
  else return row * (NCOL + 1) + c;
}

// One Stockham pass of radix R over NCOL lines of length N in shared memory.
// ZIN (first pass): rows >= N/2 of the input are zero and are not read.
// ZOUT (last pass): rows >= N/2 of the output are not needed and not stored.
template <typename C, int N, int NCOL, int NT, int DIR, bool EXACT, int R, int NS, bool ZIN = false,
          bool ZOUT = false, bool SWZ = false>
__device__ __forceinline__ void stockham_pass(C* buf, const C* __restrict__ tw) {
  constexpr int ITEMS = NCOL * (N / R);
  constexpr int PER = (ITEMS + NT - 1) / NT;
  const int tid = threadIdx.x;
  C v[PER][R];
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int w = tid + it * NT;
    if ((ITEMS % NT) == 0 || w < ITEMS) {
      const int c = w % NCOL, j = w / NCOL;
#pragma unroll
      for (int r = 0; r < R; ++r)
        v[it][r] = (ZIN && 2 * r >= R) ? mk(decltype(v[0][0].x)(0), decltype(v[0][0].x)(0))
                                        : buf[tile_at<NCOL, SWZ>(j + r * (N / R), c)];
      if constexpr (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) v[it][r] = twiddle_mul<DIR, EXACT>(v[it][r], tw, (k * r) * (N / (NS * R)));
      }
      dft<R, DIR, EXACT, ZIN>(v[it]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int w = tid + it * NT;
    if ((ITEMS % NT) == 0 || w < ITEMS) {
      const int c = w % NCOL, j = w / NCOL;
      const int k = j % NS;
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (!(ZOUT && 2 * r >= R)) buf[tile_at<NCOL, SWZ>(base + r * NS, c)] = v[it][r];
    }
  }
  __syncthreads();
}

template <typename C, int N, int NCOL, int NT, int DIR, bool EXACT, int PASS, int NS, bool ZIN, bool ZOUT, bool SWZ>
__device__ __forceinline__ void stockham_rec(C* buf, const C* __restrict__ tw) {
  constexpr RadixPlan P = radix_plan(N);
  if constexpr (PASS < P.npass) {
    constexpr int R = P.r[PASS];
    stockham_pass<C, N, NCOL, NT, DIR, EXACT, R, NS, ZIN && PASS == 0, ZOUT && PASS + 1 == P.npass, SWZ>(buf, tw);
    stockham_rec<C, N, NCOL, NT, DIR, EXACT, PASS + 1, NS * R, ZIN, ZOUT, SWZ>(buf, tw);
  }
}

// Full transform of NCOL lines of length N held in buf (caller synchronised
// before the call; the call ends with a barrier). ZIN: the input's rows >= N/2
// are zero (inputs r of the first pass with 2 r >= R lie there for every j and
// are not read); ZOUT: only output rows < N/2 are needed (outputs r of the last
// pass with 2 r >= R are not stored). SWZ: the tile uses the swizzled layout
// (tile_at).
template <typename C, int N, int NCOL, int NT, int DIR, bool EXACT, bool ZIN = false, bool ZOUT = false,
          bool SWZ = false>
__device__ __forceinline__ void fft_tile(C* buf, const C* __restrict__ tw) {
  static_assert(fft_size_ok(N), "FFT length must be 2^a or 3*2^a");
  stockham_rec<C, N, NCOL, NT, DIR, EXACT, 0, 1, ZIN, ZOUT, SWZ>(buf, tw);
}

// ---------------------------------------------------------------------------
// Register-staged Stockham for column tiles. A tile holds NCP groups of CW
// adjacent columns (CW = 2 on the float path: one 16-byte access moves a row of
// both columns, and the two share every twiddle). Each thread owns E elements
// in registers; pass p works on items (g, j), j < N/R_p, item i of thread t
// being w = t + i NT, g = w % NCP, j = w / NCP, and element (item i, column q,
// radix index r) is v[(i CW + q) R_p + r]. An item's inputs are at positions
// j + r N/R_p and its outputs at (j / Ns) Ns R_p + j % Ns + r Ns. The first
// pass's inputs come from global memory and the last pass's outputs
// (positions j + r N/R_last) stay in registers, so a transform of P passes
// makes P - 1 exchanges through the shared tile (leading dimension LDS).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int plan_lcm(int N) {
  RadixPlan p = radix_plan(N);
  int two = 1;
  bool three = false;
  for (int i = 0; i < p.npass; ++i) {
    if (p.r[i] == 3) three = true;
    else if (p.r[i] > two) two = p.r[i];
  }
  return two * (three ? 3 : 1);
}
// elements per thread and threads per tile of NCOL lines of length N, CW columns per item
// (at most maxt threads per tile)
__host__ __device__ constexpr int reg_elems(int N, int ncol, int cw = 1, int maxt = 512) {
  int e = plan_lcm(N) * cw;
  while (N * ncol / e > maxt) e *= 2;
  return e;
}
__host__ __device__ constexpr int reg_threads(int N, int ncol, int cw = 1, int maxt = 512) {
  return N * ncol / reg_elems(N, ncol, cw, maxt);
}

__device__ __forceinline__ void st_pair(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  a = make_float2(t.x, t.y);
  b = make_float2(t.z, t.w);
}

// ZIN (a first pass, NS = 1): inputs r with 2 r >= R are zero and are not read.
template <typename C, int N, int NCP, int CW, int NT, int E, int DIR, bool EXACT, int R, int NS, bool ZIN = false>
__device__ __forceinline__ void regs_pass(C (&v)[E], const C* __restrict__ tw) {
  static_assert(!ZIN || NS == 1, "zero inputs only in a first pass");
  constexpr int I = E / (R * CW);
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < I; ++i) {
    const int j = (tid + i * NT) / NCP;
    if constexpr (NS > 1) {
      const int k = j % NS;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w, l;
        twiddle_load<EXACT>(tw, (k * r) * (N / (NS * R)), w, l);
#pragma unroll
        for (int q = 0; q < CW; ++q) v[(i * CW + q) * R + r] = twiddle_apply<DIR, EXACT>(v[(i * CW + q) * R + r], w, l);
      }
    }
#pragma unroll
    for (int q = 0; q < CW; ++q) dft<R, DIR, EXACT, ZIN>(&v[(i * CW + q) * R]);
  }
}

template <typename C, int N, int NCP, int CW, int NT, int E, int R, int NS, int LDS>
__device__ __forceinline__ void regs_to_smem(const C (&v)[E], C* buf) {
  constexpr int I = E / (R * CW);
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < I; ++i) {
    const int w = tid + i * NT, g = w % NCP, j = w / NCP;
    const int base = (j / NS) * NS * R + j % NS;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      C* p = &buf[(base + r * NS) * LDS + g * CW];
      if constexpr (CW == 2) st_pair(p, v[(i * 2) * R + r], v[(i * 2 + 1) * R + r]);
      else *p = v[i * R + r];
    }
  }
}

template <typename C, int N, int NCP, int CW, int NT, int E, int R, int LDS>
__device__ __forceinline__ void smem_to_regs(C (&v)[E], const C* buf) {
  constexpr int I = E / (R * CW);
  const int tid = threadIdx.x;
#pragma unroll
  for (int i = 0; i < I; ++i) {
    const int w = tid + i * NT, g = w % NCP, j = w / NCP;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const C* p = &buf[(j + r * (N / R)) * LDS + g * CW];
      if constexpr (CW == 2) ld_pair(p, v[(i * 2) * R + r], v[(i * 2 + 1) * R + r]);
      else v[i * R + r] = *p;
    }
  }
}

// True when the plan for N lists the same radices in reverse order.
__host__ __device__ constexpr bool plan_palindrome(int N) {
  const RadixPlan p = radix_plan(N);
  for (int i = 0; i < p.npass; ++i)
    if (p.r[i] != p.r[p.npass - 1 - i]) return false;
  return true;
}

// Radix of pass p of the plan for N, taken in reverse order when REV is set.
template <int N, bool REV>
__host__ __device__ constexpr int plan_radix(int p) {
  return REV ? radix_plan(N).r[radix_plan(N).npass - 1 - p] : radix_plan(N).r[p];
}

// Runs passes PASS..last on v (holding the inputs of pass PASS). On return v
// holds the outputs of the last pass at positions j + r N/R_last. With REV the
// radices are taken in reverse order: a transform whose inputs are the outputs
// of a forward-order transform (positions j + r N/R_last) then starts without an
// exchange, since its first radix is that transform's last one. ZIN: the
// inputs at rows >= N/2 are zero (a zero-padded line) and pass 0 does not read them.
template <typename C, int N, int NCP, int CW, int NT, int E, int LDS, int DIR, bool EXACT, int PASS, int NS,
          bool REV = false, bool ZIN = false>
__device__ __forceinline__ void regs_fft(C (&v)[E], C* buf, const C* __restrict__ tw) {
  constexpr int NP = radix_plan(N).npass;
  constexpr int R = plan_radix<N, REV>(PASS);
  regs_pass<C, N, NCP, CW, NT, E, DIR, EXACT, R, NS, ZIN && PASS == 0>(v, tw);
  if constexpr (PASS + 1 < NP) {
    constexpr int R2 = plan_radix<N, REV>(PASS + 1);
    regs_to_smem<C, N, NCP, CW, NT, E, R, NS, LDS>(v, buf);
    __syncthreads();
    smem_to_regs<C, N, NCP, CW, NT, E, R2, LDS>(v, buf);
    __syncthreads();
    regs_fft<C, N, NCP, CW, NT, E, LDS, DIR, EXACT, PASS + 1, NS * R, REV>(v, buf, tw);
  }
}

}  // namespace fse

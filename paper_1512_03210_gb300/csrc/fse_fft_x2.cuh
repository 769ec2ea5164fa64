// fse_fft_x2.cuh -- register-staged Stockham passes on pairs of columns with
// packed two-lane float32 arithmetic (sm_100 family: add/mul/fma on float2
// register pairs, one instruction for both lanes).
//
// The column passes of the float path work on items of two adjacent columns
// that see exactly the same operations (same rows, same twiddles). Keeping an
// element of the pair as P2 = {re = (re_0, re_1), im = (im_0, im_1)} -- the
// real parts of both columns in one register pair, the imaginary parts in
// another -- turns every scalar operation of a one-column butterfly into one
// packed instruction for the two columns. Multiplying by +-i only renames re
// and im (the sign goes into the following add or subtract), so no lane ever
// has to be swapped, and a twiddle shared by the pair is applied with four
// packed instructions from a table holding each twiddle as (c, c, s, s).
//
// Layouts: in registers w[i R + r] is element r of item i (both columns); in
// the shared exchange tile an element of the pair is one 16-byte slot
// (re_0, re_1, im_0, im_1); in global memory a row of the pair is
// (re_0, im_0, re_1, im_1).
//
// Rounding is that of the one-column code: each packed lane rounds like the
// scalar operation it replaces (round to nearest, products of an fma rounded
// once), and the exact twiddles and butterfly constants keep their head +
// tail products (see fse_fft.cuh).
#pragma once

#include "fse_fft.cuh"

namespace fse {

struct P2 {
  float2 re, im;
};

__device__ __forceinline__ float2 bc(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b (the sign is an operand modifier of the packed add, not an instruction)
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ P2 padd(const P2& a, const P2& b) { return {add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ P2 psub(const P2& a, const P2& b) { return {sub2(a.re, b.re), sub2(a.im, b.im)}; }
// a + (DIR i) t and a - (DIR i) t: multiplying by -i maps (re, im) to (im, -re),
// by +i to (-im, re)
template <int DIR> __device__ __forceinline__ P2 padd_i(const P2& a, const P2& t) {
  return DIR < 0 ? P2{add2(a.re, t.im), sub2(a.im, t.re)} : P2{sub2(a.re, t.im), add2(a.im, t.re)};
}
template <int DIR> __device__ __forceinline__ P2 psub_i(const P2& a, const P2& t) {
  return DIR < 0 ? P2{sub2(a.re, t.im), add2(a.im, t.re)} : P2{add2(a.re, t.im), sub2(a.im, t.re)};
}

// x times a butterfly constant given as head k1 + tail k2 (EXACT) or head alone
template <bool EXACT> __device__ __forceinline__ float2 kmul2(float2 x, float k1, float k2) {
  if constexpr (EXACT) return fma2(x, bc(k1), mul2(x, bc(k2)));
  else return mul2(x, bc(k1));
}

template <int DIR, bool ZH> __device__ __forceinline__ void pdft2(P2& a, P2& b) {
  if constexpr (ZH) {
    b = a;
  } else {
    const P2 t = a;
    a = padd(t, b);
    b = psub(t, b);
  }
}

template <int DIR, bool ZH> __device__ __forceinline__ void pdft4(P2& a0, P2& a1, P2& a2, P2& a3) {
  if constexpr (ZH) {
    // a2 = a3 = 0
    const P2 x0 = a0, x1 = a1;
    a0 = padd(x0, x1);
    a2 = psub(x0, x1);
    a1 = padd_i<DIR>(x0, x1);
    a3 = psub_i<DIR>(x0, x1);
  } else {
    const P2 s02 = padd(a0, a2), d02 = psub(a0, a2), s13 = padd(a1, a3), t13 = psub(a1, a3);
    a0 = padd(s02, s13);
    a2 = psub(s02, s13);
    a1 = padd_i<DIR>(d02, t13);
    a3 = psub_i<DIR>(d02, t13);
  }
}

// Radix 8 as two radix-4 butterflies on the even and odd halves and the
// twiddles w8^k = exp(DIR i pi k / 4) on the odd half: w8 = h (1 + DIR i),
// w8^2 = DIR i, w8^3 = h (-1 + DIR i), h = sqrt(1/2).
template <int DIR, bool EXACT, bool ZH> __device__ __forceinline__ void pdft8(P2* v) {
  pdft4<DIR, ZH>(v[0], v[2], v[4], v[6]);
  pdft4<DIR, ZH>(v[1], v[3], v[5], v[7]);
  const P2 o1 = v[3], o2 = v[5], o3 = v[7];
  const float h1 = Kc<float>::h1, h2 = Kc<float>::h2;
  // w8 o1 = h ((re - DIR im) + i (im + DIR re)); w8^3 o3 = -h ((re + DIR im) + i (im - DIR re))
  const P2 t1 = DIR < 0 ? P2{kmul2<EXACT>(add2(o1.re, o1.im), h1, h2), kmul2<EXACT>(sub2(o1.im, o1.re), h1, h2)}
                        : P2{kmul2<EXACT>(sub2(o1.re, o1.im), h1, h2), kmul2<EXACT>(add2(o1.im, o1.re), h1, h2)};
  const P2 t3 = DIR < 0 ? P2{kmul2<EXACT>(sub2(o3.re, o3.im), -h1, -h2), kmul2<EXACT>(add2(o3.im, o3.re), -h1, -h2)}
                        : P2{kmul2<EXACT>(add2(o3.re, o3.im), -h1, -h2), kmul2<EXACT>(sub2(o3.im, o3.re), -h1, -h2)};
  const P2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
  v[0] = padd(e0, o0);
  v[4] = psub(e0, o0);
  v[1] = padd(e1, t1);
  v[5] = psub(e1, t1);
  v[2] = padd_i<DIR>(e2, o2);
  v[6] = psub_i<DIR>(e2, o2);
  v[3] = padd(e3, t3);
  v[7] = psub(e3, t3);
}

template <int R, int DIR, bool EXACT, bool ZH> __device__ __forceinline__ void pdft(P2* v) {
  if constexpr (R == 2) {
    pdft2<DIR, ZH>(v[0], v[1]);
  } else if constexpr (R == 4) {
    pdft4<DIR, ZH>(v[0], v[1], v[2], v[3]);
  } else {
    static_assert(R == 8, "packed radix");
    pdft8<DIR, EXACT, ZH>(v);
  }
}

// The broadcast twiddle table of length L sits right after the float2 table
// (2 L entries): twb[2m] = (c, c, s, s) of the rounded twiddle m, twb[2m+1] the
// same of its remainder.
template <int L> __device__ __forceinline__ const float4* twb_of(const float2* tw) {
  return reinterpret_cast<const float4*>(tw + 2 * L);
}

// v times twiddle (c + i s), conjugated for the inverse transform; EXACT adds
// the remainder's products inside the same fma chain (see twiddle_apply).
template <int DIR, bool EXACT>
__device__ __forceinline__ P2 ptwiddle(const P2& v, const float4* __restrict__ twb, int m) {
  const float4 w = __ldg(&twb[2 * m]);
  const float2 wc = make_float2(w.x, w.y), ws = make_float2(w.z, w.w);
  if constexpr (EXACT) {
    const float4 l = __ldg(&twb[2 * m + 1]);
    const float2 lc = make_float2(l.x, l.y), ls = make_float2(l.z, l.w);
    if constexpr (DIR < 0) {
      const float2 lr = fma2(v.re, lc, mul2(v.im, neg2(ls)));
      const float2 li = fma2(v.re, ls, mul2(v.im, lc));
      return {fma2(v.re, wc, fma2(v.im, neg2(ws), lr)), fma2(v.re, ws, fma2(v.im, wc, li))};
    } else {
      const float2 lr = fma2(v.re, lc, mul2(v.im, ls));
      const float2 li = fma2(v.im, lc, mul2(v.re, neg2(ls)));
      return {fma2(v.re, wc, fma2(v.im, ws, lr)), fma2(v.re, neg2(ws), fma2(v.im, wc, li))};
    }
  } else {
    if constexpr (DIR < 0)
      return {fma2(v.im, neg2(ws), mul2(v.re, wc)), fma2(v.im, wc, mul2(v.re, ws))};
    else
      return {fma2(v.im, ws, mul2(v.re, wc)), fma2(v.re, neg2(ws), mul2(v.im, wc))};
  }
}

// Global row of a column pair (re_0, im_0, re_1, im_1) <-> P2.
__device__ __forceinline__ P2 p2_from_row(const float4 t) { return {make_float2(t.x, t.z), make_float2(t.y, t.w)}; }
__device__ __forceinline__ float4 p2_to_row(const P2& v) { return make_float4(v.re.x, v.im.x, v.re.y, v.im.y); }
// Shared exchange slot (re_0, re_1, im_0, im_1) <-> P2.
__device__ __forceinline__ void p2_st(float2* p, const P2& v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
}
__device__ __forceinline__ P2 p2_ld(const float2* p) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  return {make_float2(t.x, t.y), make_float2(t.z, t.w)};
}

// One radix-R pass on the registers (items i of this thread, I = W / R of them).
// ZIN (a first pass, NS = 1): inputs r with 2 r >= R are zero and are not read.
template <int N, int NCP, int NT, int W, int DIR, bool EXACT, int R, int NS, bool ZIN = false>
__device__ __forceinline__ void pregs_pass(P2 (&v)[W], const float4* __restrict__ twb, int tid) {
  static_assert(!ZIN || NS == 1, "zero inputs only in a first pass");
  constexpr int I = W / R;
#pragma unroll
  for (int i = 0; i < I; ++i) {
    if constexpr (NS > 1) {
      const int j = (tid + i * NT) / NCP;
      const int k = j % NS;
      if constexpr (EXACT) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[i * R + r] = ptwiddle<DIR, EXACT>(v[i * R + r], twb, (k * r) * (N / (NS * R)));
      } else {
        // transforms of the density: twiddle r as the r-th power of twiddle 1
        // (one table load instead of R - 1; the powers drift by ~r ulp, far
        // below what a density spectrum that only sets a phase notices), so
        // that only two twiddles are ever live in registers
        const float4 w = __ldg(&twb[2 * (k * (N / (NS * R)))]);
        const float2 c1 = make_float2(w.x, w.y), s1 = make_float2(w.z, w.w);
        float2 c = c1, sn = s1;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          if (r > 1) {
            const float2 cn = fma2(c, c1, mul2(sn, neg2(s1)));
            sn = fma2(c, s1, mul2(sn, c1));
            c = cn;
          }
          const P2 x = v[i * R + r];
          v[i * R + r] = DIR < 0 ? P2{fma2(x.im, neg2(sn), mul2(x.re, c)), fma2(x.im, c, mul2(x.re, sn))}
                                 : P2{fma2(x.im, sn, mul2(x.re, c)), fma2(x.re, neg2(sn), mul2(x.im, c))};
        }
      }
    }
    pdft<R, DIR, EXACT, ZIN>(&v[i * R]);
  }
}

template <int N, int NCP, int NT, int W, int R, int NS, int LDS>
__device__ __forceinline__ void pregs_to_smem(const P2 (&v)[W], float2* buf, int tid) {
  constexpr int I = W / R;
#pragma unroll
  for (int i = 0; i < I; ++i) {
    const int w = tid + i * NT, g = w % NCP, j = w / NCP;
    const int base = (j / NS) * NS * R + j % NS;
#pragma unroll
    for (int r = 0; r < R; ++r) p2_st(&buf[(base + r * NS) * LDS + 2 * g], v[i * R + r]);
  }
}

template <int N, int NCP, int NT, int W, int R, int LDS>
__device__ __forceinline__ void psmem_to_regs(P2 (&v)[W], const float2* buf, int tid) {
  constexpr int I = W / R;
#pragma unroll
  for (int i = 0; i < I; ++i) {
    const int w = tid + i * NT, g = w % NCP, j = w / NCP;
#pragma unroll
    for (int r = 0; r < R; ++r) v[i * R + r] = p2_ld(&buf[(j + r * (N / R)) * LDS + 2 * g]);
  }
}

// Passes PASS..last of the transform of length N on v (as regs_fft, for
// pairs); tid is the thread's index in the tile.
template <int N, int NCP, int NT, int W, int LDS, int DIR, bool EXACT, int PASS, int NS, bool REV = false,
          bool ZIN = false>
__device__ __forceinline__ void pregs_fft(P2 (&v)[W], float2* buf, const float4* __restrict__ twb, int tid) {
  constexpr int NP = radix_plan(N).npass;
  constexpr int R = plan_radix<N, REV>(PASS);
  pregs_pass<N, NCP, NT, W, DIR, EXACT, R, NS, ZIN && PASS == 0>(v, twb, tid);
  if constexpr (PASS + 1 < NP) {
    constexpr int R2 = plan_radix<N, REV>(PASS + 1);
    pregs_to_smem<N, NCP, NT, W, R, NS, LDS>(v, buf, tid);
    __syncthreads();
    psmem_to_regs<N, NCP, NT, W, R2, LDS>(v, buf, tid);
    __syncthreads();
    pregs_fft<N, NCP, NT, W, LDS, DIR, EXACT, PASS + 1, NS * R, REV>(v, buf, twb, tid);
  }
}

}  // namespace fse

// fse_xpass_x2.cuh -- the float x passes on pairs of lines with packed
// two-lane arithmetic (the line counterpart of the column passes of
// fse_fft_x2.cuh).
//
// A tile of 16 consecutive lines (rows of psi) is held in shared memory as
// 16-byte slots, slot (position j, pair p) = (re of line 2p, re of line
// 2p + 1, im of line 2p, im of line 2p + 1): every Stockham pass moves whole
// slots and does the butterfly of both lines of a pair (which share position
// and twiddle) in one packed instruction per scalar operation. The zero-padded
// transforms of the density (length 2 n_x, two real lines per complex line)
// use the same slots for pairs of complex lines, 4 slots per row.
//
// Bank layout: a row of 8 slots is 128 bytes, and slot p of row j sits at
// column p ^ ((j ^ (j >> 3)) & 7), so that the Stockham passes (a quarter warp
// reads the 8 slots of one row), the transposing accesses (one slot in each
// of 8 consecutive rows) and the first pass's writes (one slot in each of rows
// 8j + r for 8 consecutive j) are all conflict-free. A
// row of 4 slots is 64 bytes: rows are permuted (row j stored at
// j ^ ((j >> 3) & 1), so that the two rows a quarter warp writes in a first
// radix-8 pass fall on different bank halves) and slot p sits at column
// p ^ ((j >> 1) & 3).
//
// The transforms of the lines (plan 8, 8, 4 or 8, 8, 8) load their first pass from
// global memory and keep their last pass in registers, stored straight back,
// so that the tile is exchanged through shared memory once; pass E's densities
// enter the first pass of the zero-padded R2C in registers too. The potential
// phase of pass A is computed with one position x per thread (all 8 pairs),
// the layout the C2R leaves in shared memory. Used for the float passes X0
// (forward x), XI (inverse x), E (inverse x, density, zero-padded R2C) and A
// (cropped C2R, potential phase, forward x) at n_x = 256 and 512 with 16-line
// tiles of n_x threads; other passes and sizes run the one-line code
// (xpass_body). At n_x = 512 the densities reach the R2C through the tile.
#pragma once

#include "fse_fft_x2.cuh"

namespace fse {

template <int NX> __host__ __device__ constexpr bool xpass_x2_ok() { return NX == 256 || NX == 512; }

// A tile is 16 lines and NX threads (one position per thread in pass A's
// phase): at n_x = 256 four tiles of 32 KB per SM, at n_x = 512 two of 64 KB.
template <int NX>
struct XCfg2 {
  static_assert(xpass_x2_ok<NX>(), "packed x passes: n_x = 256 or 512");
  static constexpr int NCOL = 16, NP = 8, NP2 = 4, NT = NX;
  static constexpr int MINB = 1024 / NT;     // 64 registers per thread
  static constexpr int PERP = NP;            // pairs per thread (all pairs at position x)
  static constexpr int NB = NX / 2 + 1;      // bin pairs (2b, 2b + 1) of a half spectrum (bins 0..NX)
  static constexpr int NHB = NP2 * NB;       // (complex-line pair, bin pair) items
  static constexpr int PHB = (NHB + NT - 1) / NT;
  // the 8-slot tile of the lines (NX rows) and the 4-slot tile of the
  // zero-padded densities (2 NX rows) share the buffer
  static constexpr size_t SMEM = 16 * (size_t)NX * NP;
};

// slot of (row, pair) in a tile of NP = 8 or NP = 4 slots per row (see above)
template <int NP> __device__ __forceinline__ int pslot(int row, int p) {
  static_assert(NP == 8 || NP == 4, "slot layouts");
  if constexpr (NP == 8) return row * 8 + (p ^ ((row ^ (row >> 3)) & 7));
  else return (row ^ ((row >> 3) & 1)) * 4 + (p ^ ((row >> 1) & 3));
}

__device__ __forceinline__ P2 p2_lds(const float4* buf, int s) {
  const float4 t = buf[s];
  return {make_float2(t.x, t.y), make_float2(t.z, t.w)};
}
__device__ __forceinline__ void p2_sts(float4* buf, int s, const P2& v) {
  buf[s] = make_float4(v.re.x, v.re.y, v.im.x, v.im.y);
}

// One radix-R Stockham pass over NP pair-slots per row of a length-N tile in
// shared memory (reads before a barrier, writes after it). ZIN: rows >= N/2
// of the input are zero and not read; ZOUT: rows >= N/2 of the output are not stored.
template <int N, int NP, int NT, int DIR, bool EXACT, int R, int NS, bool ZIN, bool ZOUT>
__device__ __forceinline__ void pstockham_pass(float4* buf, const float4* __restrict__ twb) {
  constexpr int ITEMS = NP * (N / R);
  constexpr int PER = (ITEMS + NT - 1) / NT;
  const int tid = threadIdx.x;
  P2 v[PER][R];
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int w = tid + it * NT;
    if ((ITEMS % NT) == 0 || w < ITEMS) {
      const int g = w % NP, j = w / NP;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (!(ZIN && 2 * r >= R)) v[it][r] = p2_lds(buf, pslot<NP>(j + r * (N / R), g));
      if constexpr (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) v[it][r] = ptwiddle<DIR, EXACT>(v[it][r], twb, (k * r) * (N / (NS * R)));
      }
      pdft<R, DIR, EXACT, ZIN>(v[it]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < PER; ++it) {
    const int w = tid + it * NT;
    if ((ITEMS % NT) == 0 || w < ITEMS) {
      const int g = w % NP, j = w / NP;
      const int base = (j / NS) * NS * R + j % NS;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (!(ZOUT && 2 * r >= R)) p2_sts(buf, pslot<NP>(base + r * NS, g), v[it][r]);
    }
  }
  __syncthreads();
}

template <int N, int NP, int NT, int DIR, bool EXACT, int PASS, int NS, bool ZIN, bool ZOUT>
__device__ __forceinline__ void pstockham_rec(float4* buf, const float4* __restrict__ twb) {
  constexpr RadixPlan P = radix_plan(N);
  if constexpr (PASS < P.npass) {
    constexpr int R = P.r[PASS];
    pstockham_pass<N, NP, NT, DIR, EXACT, R, NS, ZIN && PASS == 0, ZOUT && PASS + 1 == P.npass>(buf, twb);
    pstockham_rec<N, NP, NT, DIR, EXACT, PASS + 1, NS * R, ZIN, ZOUT>(buf, twb);
  }
}

// Transform of the NP pairs of lines of length N held in buf (the caller
// synchronised before; the call ends with a barrier). The 4-slot layout's row
// permutation keeps a first radix-8 pass conflict-free.
template <int N, int NP, int NT, int DIR, bool EXACT, bool ZIN = false, bool ZOUT = false>
__device__ __forceinline__ void pfft_tile(float4* buf, const float4* __restrict__ twb) {
  static_assert((N & (N - 1)) == 0 && N >= 32 && radix_plan(N).r[0] == 8, "packed x transforms: radix-8 first pass");
  pstockham_rec<N, NP, NT, DIR, EXACT, 0, 1, ZIN, ZOUT>(buf, twb);
}

// The transforms of the lines with their first pass on registers and their
// last pass into registers, so that the tile is read from and written to
// global memory directly. Length 256 (plan 8, 8, 4): thread t works on pair
// g = t / 32 and positions j + 32 r (first pass, j = t % 32), and on pairs
// 2 (t / 64) and 2 (t / 64) + 1 at positions j + 64 r (last pass, j = t % 64).
// Length 512 (plan 8, 8, 8): pair t / 64 and positions t % 64 + 64 r in both.
// Both coalesced along the lines.
static_assert(radix_plan(256).npass == 3 && radix_plan(256).r[0] == 8 && radix_plan(256).r[1] == 8 &&
                  radix_plan(256).r[2] == 4 && radix_plan(512).npass == 3 && radix_plan(512).r[0] == 8 &&
                  radix_plan(512).r[1] == 8 && radix_plan(512).r[2] == 8,
              "register first and last passes: plans 8, 8, 4 and 8, 8, 8");

// First pass (radix 8, no twiddles) of the values v[r] at positions
// j + (NX / 8) r of pair g, written to the tile (the caller synchronises after).
template <int DIR, bool EXACT>
__device__ __forceinline__ void pfirst_pass(float4* buf, P2 (&v)[8], int g, int j) {
  pdft<8, DIR, EXACT, false>(v);
#pragma unroll
  for (int r = 0; r < 8; ++r) p2_sts(buf, pslot<8>(j * 8 + r, g), v[r]);
}

// Last pass (radix 4, twiddles j r) from the tile into registers: out[it][r]
// holds position j + 64 r of pair g_it = 2 p + it, with p = t / 64, j = t % 64
// (SLOT false: a warp stores 256 contiguous bytes of a line), or p = t % 4,
// j = t / 4 (SLOT true: the two pairs of a thread are slot p of the
// zero-padded density tile at the rows its first radix-8 pass reads).
template <int DIR, bool EXACT, bool SLOT = false>
__device__ __forceinline__ void plast_pass(const float4* buf, const float4* __restrict__ twb, P2 (&out)[2][4], int tid) {
  const int j = SLOT ? tid >> 2 : tid & 63;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int g = 2 * (SLOT ? tid & 3 : tid >> 6) + it;
#pragma unroll
    for (int r = 0; r < 4; ++r) out[it][r] = p2_lds(buf, pslot<8>(j + 64 * r, g));
#pragma unroll
    for (int r = 1; r < 4; ++r) out[it][r] = ptwiddle<DIR, EXACT>(out[it][r], twb, j * r);
    pdft<4, DIR, EXACT, false>(out[it]);
  }
}

// Last pass (radix R, stride N / R) of pair g of the 8-slot tile, item j,
// into registers: v[r] = output position j + (N / R) r.
template <int N, int R, int DIR, bool EXACT>
__device__ __forceinline__ void preg_last(const float4* buf, const float4* __restrict__ twb, P2 (&v)[R], int g, int j) {
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = p2_lds(buf, pslot<8>(j + (N / R) * r, g));
#pragma unroll
  for (int r = 1; r < R; ++r) v[r] = ptwiddle<DIR, EXACT>(v[r], twb, j * r);
  pdft<R, DIR, EXACT, false>(v);
}

// The transformed densities in the packed tile (Z_k of complex line 2q + c in
// lane c of slot q, row k; the caller's last pass ended with a barrier) ->
// x-half-spectra of the tile's lines in S. Ends without a barrier.
template <int NX>
__device__ __forceinline__ void r2c_separate(const XArgs& a, const float4* buf, int l0) {
  typedef XCfg2<NX> K;
  constexpr int NP2 = K::NP2, NT = K::NT;
  const int tid = threadIdx.x;
  float2* S = reinterpret_cast<float2*>(a.spec);
  const int z0 = l0 / a.ny, y0 = l0 - z0 * a.ny;
  const float2 half = bc(0.5f);
  // bins in pairs (2b, 2b + 1), one 16-byte store per line (rows of S are
  // 16-byte aligned); the last pair is bin NX alone
#pragma unroll
  for (int it = 0; it < K::PHB; ++it) {
    const int idx = tid + it * NT;
    if (idx < K::NHB) {
      const int q = idx / K::NB, k0 = 2 * (idx % K::NB);
      float2 vals[2][4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = min(k0 + h, NX);
        const P2 zk = p2_lds(buf, pslot<NP2>(k, q));
        const P2 zm = p2_lds(buf, pslot<NP2>((2 * NX - k) % (2 * NX), q));
        const float2 ar = mul2(half, add2(zk.re, zm.re)), ai = mul2(half, sub2(zk.im, zm.im));
        const float2 br = mul2(half, add2(zk.im, zm.im)), bi = mul2(half, sub2(zm.re, zk.re));
        // complex line 2q + c carries real lines 4q + 2c (A) and 4q + 2c + 1 (B)
        vals[h][0] = make_float2(ar.x, ai.x);
        vals[h][1] = make_float2(br.x, bi.x);
        vals[h][2] = make_float2(ar.y, ai.y);
        vals[h][3] = make_float2(br.y, bi.y);
      }
      const int lb = 4 * q;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (l0 + lb + u >= a.nlines) continue;
        float2* row = &S[srow(y0, z0, lb + u, a.ny, a.srow_mul) * a.sx + k0];
        if (k0 < NX)
          *reinterpret_cast<float4*>(row) = make_float4(vals[0][u].x, vals[0][u].y, vals[1][u].x, vals[1][u].y);
        else
          *row = vals[0][u];
      }
    }
  }
}

// Densities of the tile's lines -> x-half-spectra of the zero-padded lines in
// S. Two real lines form one complex line (line 2p real part, 2p + 1 imaginary
// part), two complex lines one slot; one packed FFT of length 2 NX; the
// spectra are separated with A_k = (Z_k + conj Z_-k)/2, B_k = (Z_k - conj
// Z_-k)/(2i). Ends without a barrier.
// Thread t holds the densities rho[it][r] of pair 2 (t % 4) + it at positions
// t / 4 + 64 r (plast_pass with SLOT): the lines of slot q = t % 4 at the rows
// item t / 4 of the first radix-8 pass reads (rows NX..2NX-1 are the zero
// padding and are not read), so that pass runs on registers. The caller has
// synchronised (buf free).
template <int NX>
__device__ __forceinline__ void r2c_rows_x2(const XArgs& a, float4* buf, int l0, const float4* __restrict__ twb2,
                                            const float2 (&rho)[2][4]) {
  typedef XCfg2<NX> K;
  constexpr int NP2 = K::NP2, NT = K::NT;
  static_assert(2 * NX == 512 && radix_plan(2 * NX).npass == 3 && radix_plan(2 * NX).r[0] == 8,
                "R2C with its first pass on registers: length 512, plan 8, 8, 8");
  const int tid = threadIdx.x;
  {
    const int q = tid & 3, j = tid >> 2;
    P2 v[8];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      v[r] = P2{make_float2(rho[0][r].x, rho[1][r].x), make_float2(rho[0][r].y, rho[1][r].y)};
      v[r + 4] = P2{bc(0.f), bc(0.f)};
    }
    pdft<8, -1, false, true>(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) p2_sts(buf, pslot<NP2>(8 * j + r, q), v[r]);
  }
  __syncthreads();
  pstockham_pass<2 * NX, NP2, NT, -1, false, 8, 8, false, false>(buf, twb2);
  pstockham_pass<2 * NX, NP2, NT, -1, false, 8, 64, false, false>(buf, twb2);
  r2c_separate<NX>(a, buf, l0);
}

// The densities written into rows 0..NX-1 of the packed tile (complex line c
// in lane c & 1 of slot c >> 1; the caller has not synchronised) -> S, as
// r2c_rows_x2 with the whole transform in shared memory.
template <int NX>
__device__ __forceinline__ void r2c_rows_staged(const XArgs& a, float4* buf, int l0, const float4* __restrict__ twb2) {
  typedef XCfg2<NX> K;
  // rows NX..2NX-1 are the zero padding: the first (radix-8) pass does not read them
  __syncthreads();
  pfft_tile<2 * NX, K::NP2, K::NT, -1, false, true, false>(buf, twb2);
  r2c_separate<NX>(a, buf, l0);
}

// x-half-spectra in S of the tile's lines -> real values val[p] of lines 2p,
// 2p + 1 at this thread's position x (cropped C2R of length 2 NX, two complex
// lines per slot via the Hermitian extension Z = A + i B). The caller has
// synchronised (buf free); ends after the values are read (the caller
// synchronises before reusing buf).
template <int NX>
__device__ __forceinline__ void c2r_rows_x2(const XArgs& a, float4* buf, int l0, const float4* __restrict__ twb2,
                                            float2 (&val)[XCfg2<NX>::PERP]) {
  typedef XCfg2<NX> K;
  constexpr int NP2 = K::NP2, NT = K::NT;
  const int tid = threadIdx.x, x = tid;
  const float2* S = reinterpret_cast<const float2*>(a.spec);
  const int z0 = l0 / a.ny, y0 = l0 - z0 * a.ny;
  // bins in pairs (2b, 2b + 1), one 16-byte load per line (rows of S are
  // 16-byte aligned: sx is a multiple of 16); the last pair holds bin NX and a
  // padding bin of the row, which is not used
#pragma unroll
  for (int it = 0; it < K::PHB; ++it) {
    const int idx = tid + it * NT;
    if (idx < K::NHB) {
      const int q = idx / K::NB, k0 = 2 * (idx % K::NB);
      const int lb = 4 * q;
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        v[u] = (l0 + lb + u < a.nlines)
                   ? *reinterpret_cast<const float4*>(&S[srow(y0, z0, lb + u, a.ny, a.srow_mul) * a.sx + k0])
                   : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = k0 + h;
        if (k > NX) break;
        float2 w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = h ? make_float2(v[u].z, v[u].w) : make_float2(v[u].x, v[u].y);
        // lane c: A = w[2c], B = w[2c + 1]; Z_k = A + i B, Z_{2NX-k} = conj(A) + i conj(B)
        const P2 zk{make_float2(w[0].x - w[1].y, w[2].x - w[3].y), make_float2(w[0].y + w[1].x, w[2].y + w[3].x)};
        p2_sts(buf, pslot<NP2>(k, q), zk);
        if (k > 0 && k < NX) {
          const P2 zm{make_float2(w[0].x + w[1].y, w[2].x + w[3].y), make_float2(w[1].x - w[0].y, w[3].x - w[2].y)};
          p2_sts(buf, pslot<NP2>(2 * NX - k, q), zm);
        }
      }
    }
  }
  __syncthreads();
  // only rows 0..NX-1 survive the crop: the last pass stores no others
  pfft_tile<2 * NX, NP2, NT, +1, false, false, true>(buf, twb2);
#pragma unroll
  for (int q = 0; q < NP2; ++q) {
    const float4 t = buf[pslot<NP2>(x, q)];
    val[2 * q] = make_float2(t.x, t.z);
    val[2 * q + 1] = make_float2(t.y, t.w);
  }
}

// sin and cos of the phases of two lines: the short series of phase_sincos
// in packed form when both are within 1/2, sincosf otherwise.
__device__ __forceinline__ void phase_sincos2(float2 th, float2& sn, float2& cs) {
  if (fabsf(th.x) <= 0.5f && fabsf(th.y) <= 0.5f) {
    const float2 t2 = mul2(th, th);
    const float2 ps = mul2(t2, fma2(t2, fma2(t2, fma2(t2, bc(1.0f / 362880.0f), bc(-1.0f / 5040.0f)), bc(1.0f / 120.0f)),
                                    bc(-1.0f / 6.0f)));
    const float2 pc = mul2(t2, fma2(t2, fma2(t2, fma2(t2, bc(1.0f / 40320.0f), bc(-1.0f / 720.0f)), bc(1.0f / 24.0f)),
                                    bc(-0.5f)));
    sn = fma2(th, ps, th);
    cs = add2(bc(1.0f), pc);
  } else {
    phase_sincos(th.x, &sn.x, &cs.x);
    phase_sincos(th.y, &sn.y, &cs.y);
  }
}

template <int NX, int KIND>
__device__ __forceinline__ void xpass_body_x2(const XArgs& a, const float2* __restrict__ twn,
                                              const float2* __restrict__ tw2n, int bid) {
  typedef XCfg2<NX> K;
  constexpr int NCOL = K::NCOL, NP = K::NP, NT = K::NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  float4* buf = reinterpret_cast<float4*>(smem_raw);
  const float4* twb1 = twb_of<NX>(twn);
  const float4* twb2 = twb_of<2 * NX>(tw2n);
  const int tid = threadIdx.x, x = tid;
  const int l0 = bid * NCOL;
  float2* psi = reinterpret_cast<float2*>(a.psi) + (long long)l0 * NX + x;  // line l0 at position x
  const int nl = a.nlines - l0;  // lines of this tile that exist (may exceed NCOL)
  const float2 z = make_float2(0.f, 0.f);

  if constexpr (KIND == XP_FWD || KIND == XP_INV || KIND == XP_E) {
    constexpr int DIR = KIND == XP_FWD ? -1 : +1;
    constexpr int L = NX / 8;  // first pass: pair t / L, positions t % L + L r
    float2* line0 = reinterpret_cast<float2*>(a.psi) + (long long)l0 * NX;  // line l0 of the tile
    {
      const int g = tid / L, j = tid % L;
      P2 v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float2 u0 = 2 * g < nl ? line0[(2 * g) * NX + j + L * r] : z;
        const float2 u1 = 2 * g + 1 < nl ? line0[(2 * g + 1) * NX + j + L * r] : z;
        v[r] = P2{make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
      }
      pfirst_pass<DIR, true>(buf, v, g, j);
    }
    __syncthreads();
    pstockham_pass<NX, NP, NT, DIR, true, 8, 8, false, false>(buf, twb1);
    if constexpr (NX == 512) {
      // last pass (radix 8, stride 64): pair t / 64, positions t % 64 + 64 r
      const int g = tid >> 6, j = tid & 63;
      P2 out[8];
      preg_last<NX, 8, DIR, true>(buf, twb1, out, g, j);
      float2 rho[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const P2 u = out[r];
        if (2 * g < nl) line0[(2 * g) * NX + j + 64 * r] = make_float2(u.re.x, u.im.x);
        if (2 * g + 1 < nl) line0[(2 * g + 1) * NX + j + 64 * r] = make_float2(u.re.y, u.im.y);
        rho[r] = fma2(u.re, u.re, mul2(u.im, u.im));
      }
      if constexpr (KIND == XP_E || KIND == XP_INV) {
        if (a.part) {  // float64 mass partial of this tile (renormalisation)
          double acc = 0.0;
#pragma unroll
          for (int r = 0; r < 8; ++r) acc += (double)rho[r].x + (double)rho[r].y;
          acc = block_sum(acc, red);
          if (tid == 0) a.part[bid] = acc;
        }
      }
      if constexpr (KIND == XP_E) {
        // the densities into the zero-padded packed tile: complex line g
        // (lines 2g, 2g + 1) is lane g & 1 of slot g >> 1 (the last pass's
        // reads of the tile are finished before it is overwritten)
        __syncthreads();
        float* bf = reinterpret_cast<float*>(buf);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int sl = pslot<K::NP2>(j + 64 * r, g >> 1) * 4 + (g & 1);
          bf[sl] = rho[r].x;
          bf[sl + 2] = rho[r].y;
        }
        r2c_rows_staged<NX>(a, buf, l0, twb2);
      }
    } else {
      constexpr bool SLOT = KIND == XP_E;
      P2 out[2][4];
      plast_pass<DIR, true, SLOT>(buf, twb1, out, tid);
      const int j = SLOT ? tid >> 2 : tid & 63;
      float2 rho[2][4];
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int g = 2 * (SLOT ? tid & 3 : tid >> 6) + it;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const P2 u = out[it][r];
          if (2 * g < nl) line0[(2 * g) * NX + j + 64 * r] = make_float2(u.re.x, u.im.x);
          if (2 * g + 1 < nl) line0[(2 * g + 1) * NX + j + 64 * r] = make_float2(u.re.y, u.im.y);
          rho[it][r] = fma2(u.re, u.re, mul2(u.im, u.im));
        }
      }
      if constexpr (KIND == XP_E || KIND == XP_INV) {
        if (a.part) {  // float64 mass partial of this tile (renormalisation)
          double acc = 0.0;
#pragma unroll
          for (int it = 0; it < 2; ++it)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc += (double)rho[it][r].x + (double)rho[it][r].y;
          acc = block_sum(acc, red);
          if (tid == 0) a.part[bid] = acc;
        }
      }
      if constexpr (KIND == XP_E) {
        // the last pass's reads of the tile are finished before it is overwritten
        __syncthreads();
        r2c_rows_x2<NX>(a, buf, l0, twb2, rho);
      }
    }
  } else {
    static_assert(KIND == XP_A, "packed x passes: X0, XI, E, A");
    if (tid == 0 && nl > 0 && (reinterpret_cast<uintptr_t>(a.psi) & 15) == 0) {
      // the tile's rows of psi (contiguous) move to L2 while the C2R runs
      prefetch_l2_bulk(reinterpret_cast<float2*>(a.psi) + (long long)l0 * NX,
                       (unsigned)(min(NCOL, nl) * NX * sizeof(float2)));
    }
    float2 vphi[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) vphi[p] = z;
    if (a.use_spec) c2r_rows_x2<NX>(a, buf, l0, twb2, vphi);
    const bool rescale = a.scale != nullptr;
    const float fsc = rescale ? float(*a.scale) : 1.0f;
    const int z0 = l0 / a.ny, y0 = l0 - z0 * a.ny;
    __syncthreads();
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const bool ok0 = 2 * p < nl, ok1 = 2 * p + 1 < nl;
      const float2 u0 = ok0 ? psi[(2 * p) * NX] : z;
      const float2 u1 = ok1 ? psi[(2 * p + 1) * NX] : z;
      int ya, za, yb, zb;
      line_yz(y0, z0, 2 * p, a.ny, ya, za);
      line_yz(y0, z0, 2 * p + 1, a.ny, yb, zb);
      const P2 u{make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
      const float2 rho = fma2(u.re, u.re, mul2(u.im, u.im));
      const float2 P = make_float2(trap_phase<float, 0>(a, x, ya, za), trap_phase<float, 0>(a, x, yb, zb));
      const float2 th = fma2(bc(a.f.beta_dt), rho, fma2(bc(a.f.lam), vphi[p], P));
      float2 sn, cs;
      phase_sincos2(th, sn, cs);
      // u2 = u (cs - i sn), the factor's modulus error folded in (unit_mul)
      const float2 h = make_float2(-0.5f * norm_err(cs.x, sn.x), -0.5f * norm_err(cs.y, sn.y));
      const float2 s2 = neg2(sn);
      const float2 lc = mul2(h, cs), ls = mul2(h, s2);
      const float2 lr = fma2(u.re, lc, mul2(u.im, neg2(ls)));
      const float2 li = fma2(u.re, ls, mul2(u.im, lc));
      float2 yr = fma2(u.re, cs, fma2(u.im, neg2(s2), lr));
      float2 yi = fma2(u.re, s2, fma2(u.im, cs, li));
      if (rescale) {
        yr = mul2(bc(fsc), yr);
        yi = mul2(bc(fsc), yi);
      }
      if (!ok0) yr.x = yi.x = 0.f;
      if (!ok1) yr.y = yi.y = 0.f;
      p2_sts(buf, pslot<NP>(x, p), P2{yr, yi});
    }
    __syncthreads();
    pstockham_pass<NX, NP, NT, -1, true, 8, 1, false, false>(buf, twb1);
    pstockham_pass<NX, NP, NT, -1, true, 8, 8, false, false>(buf, twb1);
    float2* line0 = reinterpret_cast<float2*>(a.psi) + (long long)l0 * NX;
    if constexpr (NX == 512) {
      // last pass (radix 8, stride 64): pair t / 64, positions t % 64 + 64 r
      const int g = tid >> 6, j = tid & 63;
      P2 o[8];
      preg_last<NX, 8, -1, true>(buf, twb1, o, g, j);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        if (2 * g < nl) line0[(2 * g) * NX + j + 64 * r] = make_float2(o[r].re.x, o[r].im.x);
        if (2 * g + 1 < nl) line0[(2 * g + 1) * NX + j + 64 * r] = make_float2(o[r].re.y, o[r].im.y);
      }
    } else {
      P2 out[2][4];
      plast_pass<-1, true>(buf, twb1, out, tid);
      const int j = tid & 63;
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int g = 2 * (tid >> 6) + it;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const P2 u = out[it][r];
          if (2 * g < nl) line0[(2 * g) * NX + j + 64 * r] = make_float2(u.re.x, u.im.x);
          if (2 * g + 1 < nl) line0[(2 * g + 1) * NX + j + 64 * r] = make_float2(u.re.y, u.im.y);
        }
      }
    }
  }
}

}  // namespace fse

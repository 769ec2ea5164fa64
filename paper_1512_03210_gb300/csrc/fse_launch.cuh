// fse_launch.cuh -- size dispatch of the pass kernels (included by one .cu per precision and kind).
#pragma once

#include <atomic>

#include "fse_passes.cuh"

namespace fse {

// FFT lengths of the column passes (n and 2n) and of the x passes (n).
#define FSE_COL_SIZES(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)
#define FSE_X_SIZES(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512)

// Launch of a step pass with programmatic dependent launch on the previous
// kernel in the stream (see pass_prologue).
template <typename... Params, typename... Args>
static cudaError_t launch_pass(void (*kernel)(Params...), unsigned blocks, unsigned threads, size_t smem,
                               cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// cudaFuncSetAttribute once per kernel and device when the dynamic tile comes
// near the 48 KB default (the kernels also hold up to 1 KB of static shared memory).
template <typename F>
static cudaError_t allow_smem(F* fn, size_t bytes, std::atomic<unsigned long long>& done) {
  if (bytes + 1024 <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

template <typename Real, int N, int VAR>
static cudaError_t col_launch(const ColArgs& a, const MulArgs& m, const void* tw, cudaStream_t st) {
  typedef ColCfg<Real, N, VAR> K;
  typedef typename K::C C;
  const size_t smem = K::smem_bytes(VAR);
  static std::atomic<unsigned long long> done{0};
  cudaError_t e = allow_smem(k_colpass<Real, N, VAR>, smem, done);
  if (e != cudaSuccess) return e;
  const long long blocks = col_blocks(a, K::NCOL);
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  MulArgs mf = m;
  fill_f32(mf);
  return launch_pass(k_colpass<Real, N, VAR>, (unsigned)blocks, K::NT, smem, st, a, mf, reinterpret_cast<const C*>(tw));
}

template <typename Real>
cudaError_t launch_colpass(int N, int var, const ColArgs& a, const MulArgs& m, const void* tw, cudaStream_t st) {
  switch (N) {
#define FSE_CASE(n)                                                         \
  case n:                                                                   \
    switch (var) {                                                          \
      case COL_FWD: return col_launch<Real, n, COL_FWD>(a, m, tw, st);      \
      case COL_INV: return col_launch<Real, n, COL_INV>(a, m, tw, st);      \
      case COL_PADF: return col_launch<Real, n, COL_PADF>(a, m, tw, st);    \
      case COL_CROPI: return col_launch<Real, n, COL_CROPI>(a, m, tw, st);  \
      case COL_KIN: return col_launch<Real, n, COL_KIN>(a, m, tw, st);      \
      default: return col_launch<Real, n, COL_KHAT>(a, m, tw, st);          \
    }
    FSE_COL_SIZES(FSE_CASE)
#undef FSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename Real> int colpass_ncol(int N) {
  return col_ncol(N, 2 * (int)sizeof(Real));
}

template <typename Real, int NX, int KIND>
static cudaError_t x_launch(const XArgs& a, const void* twn, const void* tw2n, cudaStream_t st) {
  typedef XLaunch<Real, NX, KIND> K;
  typedef typename Cplx<Real>::T C;
  const size_t smem = K::smem_bytes();
  static std::atomic<unsigned long long> done{0};
  cudaError_t e = allow_smem(k_xpass<Real, NX, KIND>, smem, done);
  if (e != cudaSuccess) return e;
  const int blocks = (a.nlines + K::NCOL - 1) / K::NCOL;
  if (blocks <= 0) return cudaSuccess;
  XArgs af = a;
  fill_f32(af);
  return launch_pass(k_xpass<Real, NX, KIND>, (unsigned)blocks, K::NT, smem, st, af, reinterpret_cast<const C*>(twn),
                     reinterpret_cast<const C*>(tw2n));
}

template <typename Real>
cudaError_t launch_xpass(int kind, int nx, const XArgs& a, const void* twn, const void* tw2n,
                         cudaStream_t st) {
  switch (nx) {
#define FSE_CASE(n)                                                   \
  case n:                                                             \
    switch (kind) {                                                   \
      case XP_FWD: return x_launch<Real, n, XP_FWD>(a, twn, tw2n, st); \
      case XP_INV: return x_launch<Real, n, XP_INV>(a, twn, tw2n, st); \
      case XP_E: return x_launch<Real, n, XP_E>(a, twn, tw2n, st);     \
      case XP_R: return x_launch<Real, n, XP_R>(a, twn, tw2n, st);     \
      case XP_ADJ1: return x_launch<Real, n, XP_ADJ1>(a, twn, tw2n, st); \
      case XP_ADJ2: return x_launch<Real, n, XP_ADJ2>(a, twn, tw2n, st); \
      case XP_AL: return x_launch<Real, n, XP_AL>(a, twn, tw2n, st);   \
      default: return x_launch<Real, n, XP_A>(a, twn, tw2n, st);       \
    }
    FSE_X_SIZES(FSE_CASE)
#undef FSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename Real> int xpass_ncol(int nx) {
  switch (nx) {
#define FSE_CASE(n) \
  case n:           \
    return XCfg<Real, n>::NCOL;
    FSE_X_SIZES(FSE_CASE)
#undef FSE_CASE
    default:
      return 0;
  }
}

template <typename Real> int xpass_ncol_x2(int nx) {
  switch (nx) {
#define FSE_CASE(n) \
  case n:           \
    return XLaunch<Real, n, XP_E>::NCOL;
    FSE_X_SIZES(FSE_CASE)
#undef FSE_CASE
    default:
      return 0;
  }
}

}  // namespace fse

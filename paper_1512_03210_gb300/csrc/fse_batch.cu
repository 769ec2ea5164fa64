// fse_batch.cu -- many independent 2D TS2-GauSum runs advanced together.
//
// Runs with the same grid size form a group. Every pass of the split step
// (Section 4.2, Eqs. tssp1-tssp3) is one launch per group: blockIdx.x walks
// the tiles of one run, blockIdx.y selects the run, whose buffers and
// parameters (s through its kinetic tables, Omega, beta, lambda, dt, gamma)
// come from a device descriptor table. The pass bodies are the single-run
// ones, so a run advanced in a batch is bit-identical to the same run
// advanced alone. Runs never wait on one another. The launches of a call of
// nsteps steps are captured once as a CUDA graph (per step count) and replayed
// by later calls; the call's data (wave-function pointers, start time) reach
// the kernels through device tables uploaded ahead of each replay.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fse.h"
#include "fse_internal.h"
#include "fse_launch.cuh"

namespace fse {

struct BatchRun {
  void* psi;
  void* spec;
  const void* kin_half;
  const void* kin_full;
  double beta, lam, dt, omega, gx2, gy2;
};

__device__ __forceinline__ double sin_over_dev(double a, double d) {
  const double z = a * d;
  return fabs(z) < 1e-6 ? d * (1.0 - z * z / 6.0) : sin(z) / a;
}

template <typename Real, int N, int VAR>
__global__ void __launch_bounds__(ColCfg<Real, N, VAR>::NT, ColCfg<Real, N, VAR>::MINB)
k_colpass_batch(ColArgs a, MulArgs m, const typename Cplx<Real>::T* __restrict__ tw, const BatchRun* runs,
                int on_spec, int kin_full, int conj) {
  const BatchRun r = runs[blockIdx.y];
  a.data = on_spec ? r.spec : r.psi;
  if constexpr (VAR == COL_KIN) {
    m.kin = kin_full ? r.kin_full : r.kin_half;
    m.conj = conj;
  } else {
    m.a0 = r.dt * m.scale;
    m.f.a0 = (float)m.a0;
  }
  colpass_body<Real, N, VAR>(a, m, tw, blockIdx.x);
}

template <typename Real, int NX, int KIND>
__global__ void __launch_bounds__(XLaunch<Real, NX, KIND>::NT, XLaunch<Real, NX, KIND>::MINB)
k_xpass_batch(XArgs a, const typename Cplx<Real>::T* __restrict__ twn, const typename Cplx<Real>::T* __restrict__ tw2n,
              const BatchRun* runs, const double* t0p, int step) {
  const BatchRun r = runs[blockIdx.y];
  a.psi = r.psi;
  a.spec = a.use_spec ? r.spec : nullptr;
  if constexpr (KIND == XP_A) {
    // exact time integral of the rotating harmonic trap over the run's step
    // (Eq. int_poten); the call's start time t0 is a device scalar, so that a
    // captured graph of the step sequence serves every call. One thread
    // evaluates the float64 sines and cosines (GB300's float64 pipe is
    // narrow) and the block reads the coefficients from shared memory.
    __shared__ double trap[3];
    if (threadIdx.x == 0) {
      const double ta = *t0p + step * r.dt, d = r.dt, mid = 2.0 * ta + d;
      const double C2 = cos(r.omega * mid) * sin_over_dev(r.omega, d);
      const double S2 = sin(r.omega * mid) * sin_over_dev(r.omega, d);
      trap[0] = 0.25 * (r.gx2 * (d + C2) + r.gy2 * (d - C2));
      trap[1] = 0.25 * (r.gx2 * (d - C2) + r.gy2 * (d + C2));
      trap[2] = 0.5 * (r.gx2 - r.gy2) * S2;
    }
    __syncthreads();
    a.pa = trap[0];
    a.pb = trap[1];
    a.pc = trap[2];
    a.pe = 0.0;
    a.beta_dt = r.beta * r.dt;
    a.lam = r.lam;
    fill_f32_phase(a);
  }
  xpass_any<Real, NX, KIND>(a, twn, tw2n, blockIdx.x);
}

template <int N, int VAR>
static cudaError_t colb(const ColArgs& a, const MulArgs& m, const void* tw, const BatchRun* runs, int nr,
                        int on_spec, int kin_full, int conj, cudaStream_t st) {
  typedef ColCfg<float, N, VAR> K;
  const size_t smem = K::smem_bytes(VAR);
  static std::atomic<unsigned long long> done{0};
  cudaError_t e = allow_smem(k_colpass_batch<float, N, VAR>, smem, done);
  if (e != cudaSuccess) return e;
  dim3 grid(a.nplanes * a.tiles_per_plane, nr);
  MulArgs mf = m;
  fill_f32(mf);
  k_colpass_batch<float, N, VAR><<<grid, K::NT, smem, st>>>(a, mf, reinterpret_cast<const float2*>(tw), runs, on_spec,
                                                             kin_full, conj);
  return cudaGetLastError();
}

static cudaError_t launch_colb(int N, int mode, const ColArgs& a, const MulArgs& m, const void* tw,
                               const BatchRun* runs, int nr, int on_spec, int kin_full, int conj, cudaStream_t st) {
  switch (N) {
#define FSE_CASE(n)                                                                          \
  case n:                                                                                    \
    return mode == 1 ? colb<n, COL_KIN>(a, m, tw, runs, nr, on_spec, kin_full, conj, st)      \
                     : colb<n, COL_KHAT>(a, m, tw, runs, nr, on_spec, kin_full, conj, st);
    FSE_COL_SIZES(FSE_CASE)
#undef FSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <int NX, int KIND>
static cudaError_t xb(const XArgs& a, const void* twn, const void* tw2n, const BatchRun* runs, int nr,
                      const double* t0, int step, cudaStream_t st) {
  typedef XLaunch<float, NX, KIND> K;
  const size_t smem = K::smem_bytes();
  static std::atomic<unsigned long long> done{0};
  cudaError_t e = allow_smem(k_xpass_batch<float, NX, KIND>, smem, done);
  if (e != cudaSuccess) return e;
  dim3 grid((a.nlines + K::NCOL - 1) / K::NCOL, nr);
  XArgs af = a;
  fill_f32(af);
  k_xpass_batch<float, NX, KIND><<<grid, K::NT, smem, st>>>(af, reinterpret_cast<const float2*>(twn),
                                                            reinterpret_cast<const float2*>(tw2n), runs, t0, step);
  return cudaGetLastError();
}

static cudaError_t launch_xb(int kind, int nx, const XArgs& a, const void* twn, const void* tw2n,
                             const BatchRun* runs, int nr, const double* t0, int step, cudaStream_t st) {
  switch (nx) {
#define FSE_CASE(n)                                                    \
  case n:                                                              \
    switch (kind) {                                                    \
      case XP_FWD: return xb<n, XP_FWD>(a, twn, tw2n, runs, nr, t0, step, st); \
      case XP_INV: return xb<n, XP_INV>(a, twn, tw2n, runs, nr, t0, step, st); \
      case XP_E: return xb<n, XP_E>(a, twn, tw2n, runs, nr, t0, step, st);     \
      default: return xb<n, XP_A>(a, twn, tw2n, runs, nr, t0, step, st);       \
    }
    FSE_X_SIZES(FSE_CASE)
#undef FSE_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

const void* twiddle(const fse_plan* P, int L);
template <typename Real>
cudaError_t launch_kin_table(void* half, void* full, int nx, int ny, int nz, double dkx, double dky, double dkz,
                             double s, double m2, double dt, cudaStream_t st);

}  // namespace fse

using namespace fse;

struct fse_batch {
  struct Group {
    int nx = 0, ny = 0;
    std::vector<int> runs;
    fse_plan* plan = nullptr;  // twiddles and kernel transform of the group (shared by its runs)
    size_t off_plan = 0, off_desc = 0;
  };
  std::vector<fse_params> runs;
  std::vector<Group> groups;
  std::vector<size_t> off_kh, off_kf, off_spec;
  cudaStream_t stream = nullptr;
  size_t ws_bytes = 0;
  void* ws = nullptr;
  bool precomputed = false;
  long long launches = 0;
  std::string err;
  std::vector<BatchRun> desc;  // host staging of the descriptor tables
  // groups are independent: each runs on its own stream, forked from and
  // joined back into `stream` with events (created at the first step)
  std::vector<cudaStream_t> gstream;
  std::vector<cudaEvent_t> gdone;
  cudaEvent_t fork = nullptr;
  // the step sequence of a call of nsteps steps, captured once as a CUDA graph
  // and replayed on `cap` (a stream of the batch's own: the caller's stream may
  // be the legacy default stream, which cannot be captured)
  struct Graph {
    int nsteps;
    cudaGraphExec_t exec;
    long long launches;
  };
  std::vector<Graph> graphs;
  cudaStream_t cap = nullptr;
  cudaEvent_t cap_in = nullptr, cap_out = nullptr;
  size_t off_t0 = 0;  // device scalar: the call's start time
  char* ptr(size_t off) const { return static_cast<char*>(ws) + off; }
};

namespace {
size_t al(size_t v) { return (v + 255) & ~(size_t)255; }
fse_status bfail(fse_batch* B, fse_status st, const std::string& m) {
  B->err = m;
  return st;
}
}  // namespace

extern "C" {

fse_status fse_batch_create(const fse_params* runs, int nruns, void* stream, fse_batch_t* out,
                            size_t* workspace_bytes) {
  if (!runs || nruns <= 0 || !out || !workspace_bytes) return FSE_ERR_INVALID;
  *out = nullptr;
  *workspace_bytes = 0;
  const fse_params e0 = effective_params(runs[0]);
  for (int r = 0; r < nruns; ++r) {
    const fse_params& p = runs[r];
    // every run gets the checks of fse_plan_create (only the first run of a
    // size group builds a plan)
    const fse_status vst = validate_params(p);
    if (vst != FSE_OK) return vst;
    // the group's kernel transform is built from its first run: the exponent
    // and the Gaussian-sum fit must be the same for every run
    const fse_params e = effective_params(p);
    if (e.mu != e0.mu || e.gs_delta != e0.gs_delta || e.gs_h != e0.gs_h || e.gs_tmin != e0.gs_tmin)
      return FSE_ERR_UNSUPPORTED;
    if (p.dim != 2 || p.prec != FSE_F32 || p.renormalize != 0 || (p.order != 0 && p.order != 2) ||
        p.lat_amp != 0.0)
      return FSE_ERR_UNSUPPORTED;
    if (p.kernel == FSE_KERNEL_DDI3D || p.kernel == FSE_KERNEL_DDI2D) return FSE_ERR_INVALID;
    if (p.lo[0] != runs[0].lo[0] || p.lo[1] != runs[0].lo[1] || p.hi[0] != runs[0].hi[0] ||
        p.hi[1] != runs[0].hi[1] || p.kernel != runs[0].kernel)
      return FSE_ERR_UNSUPPORTED;  // one box and one kernel per batch
  }
  fse_batch* B = new (std::nothrow) fse_batch();
  if (!B) return FSE_ERR_NOMEM;
  B->runs.assign(runs, runs + nruns);
  B->stream = reinterpret_cast<cudaStream_t>(stream);
  for (int r = 0; r < nruns; ++r) {
    int g = -1;
    for (size_t k = 0; k < B->groups.size(); ++k)
      if (B->groups[k].nx == runs[r].n[0] && B->groups[k].ny == runs[r].n[1]) g = (int)k;
    if (g < 0) {
      B->groups.emplace_back();
      g = (int)B->groups.size() - 1;
      B->groups[g].nx = runs[r].n[0];
      B->groups[g].ny = runs[r].n[1];
    }
    B->groups[g].runs.push_back(r);
  }
  size_t off = 0;
  B->off_kh.assign(nruns, 0);
  B->off_kf.assign(nruns, 0);
  B->off_spec.assign(nruns, 0);
  for (auto& G : B->groups) {
    size_t nb = 0;
    fse_status st = fse_plan_create(&runs[G.runs[0]], stream, &G.plan, &nb);
    if (st != FSE_OK) {
      fse_batch_destroy(B);
      return st;
    }
    G.off_plan = off;
    off = al(off + nb);
    G.off_desc = off;
    off = al(off + sizeof(BatchRun) * G.runs.size());
    const size_t kin_bytes = (size_t)(G.nx / 2 + 1) * (G.ny / 2 + 1) * 8;
    const size_t spec_bytes = (size_t)G.ny * G.plan->sx * 8;
    for (size_t k = 1; k < G.runs.size(); ++k) {
      const int r = G.runs[k];
      B->off_kh[r] = off;
      off = al(off + kin_bytes);
      B->off_kf[r] = off;
      off = al(off + kin_bytes);
      B->off_spec[r] = off;
      off = al(off + spec_bytes);
    }
  }
  B->off_t0 = off;
  off = al(off + sizeof(double));
  B->ws_bytes = off;
  *workspace_bytes = off;
  *out = B;
  return FSE_OK;
}

fse_status fse_batch_set_workspace(fse_batch_t B, void* ptr, size_t bytes) {
  if (!B || !ptr) return FSE_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(ptr) % 256 != 0) return bfail(B, FSE_ERR_INVALID, "workspace not 256-byte aligned");
  if (bytes < B->ws_bytes) return bfail(B, FSE_ERR_NOMEM, "workspace smaller than fse_batch_create reported");
  B->ws = ptr;
  B->precomputed = false;
  for (auto& G : B->groups) {
    fse_status st = fse_plan_set_workspace(G.plan, B->ptr(G.off_plan), G.plan->ws_bytes);
    if (st != FSE_OK) return bfail(B, st, G.plan->err);
  }
  return FSE_OK;
}

fse_status fse_batch_precompute(fse_batch_t B) {
  if (!B) return FSE_ERR_INVALID;
  if (!B->ws) return bfail(B, FSE_ERR_INVALID, "no workspace attached");
  for (auto& G : B->groups) {
    fse_status st = fse_kernel_precompute(G.plan);
    if (st != FSE_OK) return bfail(B, st, G.plan->err);
    B->launches += G.plan->launches;
    G.plan->launches = 0;
    for (size_t k = 1; k < G.runs.size(); ++k) {
      const fse_params& p = B->runs[G.runs[k]];
      const double dkx = 2 * kPi / (p.hi[0] - p.lo[0]), dky = 2 * kPi / (p.hi[1] - p.lo[1]);
      cudaError_t e = launch_kin_table<float>(B->ptr(B->off_kh[G.runs[k]]), B->ptr(B->off_kf[G.runs[k]]), G.nx, G.ny,
                                              1, dkx, dky, 0.0, p.s, p.m * p.m, p.dt, B->stream);
      if (e != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string("kinetic tables: ") + cudaGetErrorString(e));
      ++B->launches;
    }
  }
  B->precomputed = true;
  return FSE_OK;
}

}  // extern "C"

namespace {

// The launches of nsteps steps of every group, each group on its own stream
// (forked from and joined back into `st`); the descriptor tables and the start
// time are read from the workspace when the kernels run. Returns the number
// of launches in *count.
fse_status batch_sequence(fse_batch* B, int nsteps, cudaStream_t st0, long long* count) {
  const bool multi = B->groups.size() > 1;
  long long nl = 0;
  if (multi) {
    cudaError_t e = cudaEventRecord(B->fork, st0);
    for (size_t g = 0; g < B->groups.size() && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(B->gstream[g], B->fork, 0);
    if (e != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string("group fork: ") + cudaGetErrorString(e));
  }
  const double* t0 = reinterpret_cast<const double*>(B->ptr(B->off_t0));
  for (size_t gi = 0; gi < B->groups.size(); ++gi) {
    auto& G = B->groups[gi];
    const cudaStream_t st = multi ? B->gstream[gi] : st0;
    fse_plan* P = G.plan;
    const int nr = (int)G.runs.size();
    const BatchRun* ddesc = reinterpret_cast<const BatchRun*>(B->ptr(G.off_desc));
    const bool nl_on = B->runs[G.runs[0]].kernel != FSE_KERNEL_NONE;
    XArgs xa = x_args(P, nullptr, nl_on ? reinterpret_cast<void*>(1) : nullptr);  // pointers come from the table
    xa.use_spec = nl_on ? 1 : 0;
    const void* twn = twiddle(P, P->nx);
    const void* tw2n = twiddle(P, 2 * P->nx);
    MulArgs mk1;
    std::memset(&mk1, 0, sizeof(mk1));
    mk1.mode = MUL_KIN;
    mk1.lx = P->nx;
    mk1.lr = P->ny;
    mk1.kin_sr = P->nx / 2 + 1;
    mk1.scale = 1.0 / ((double)P->nx * P->ny);
    ColArgs ck{nullptr, 0, P->nx, 1, P->nx, P->ny, P->ny, tiles(P, P->ny, P->nx)};
    MulArgs mk2;
    std::memset(&mk2, 0, sizeof(mk2));
    mk2.mode = MUL_COULOMB;
    mk2.lx = 2 * P->nx;
    mk2.lr = 2 * P->ny;
    mk2.chat = P->ws_ptr(P->off_chat);
    mk2.chat_cx = P->chat_cx;
    mk2.chat_sr = P->chat_cx;
    mk2.scale = 1.0 / (4.0 * P->nx * P->ny);
    ColArgs cg{nullptr, 0, P->sx, 1, P->nx + 1, P->ny, P->ny, tiles(P, 2 * P->ny, P->nx + 1)};
    auto chk = [&](cudaError_t ee, const char* w) -> fse_status {
      if (ee != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string(w) + ": " + cudaGetErrorString(ee));
      ++nl;
      return FSE_OK;
    };
    fse_status s;
    if ((s = chk(launch_xb(XP_FWD, P->nx, xa, twn, tw2n, ddesc, nr, t0, 0, st), "batch x")) != FSE_OK) return s;
    for (int n = 0; n < nsteps; ++n) {
      if ((s = chk(launch_colb(P->ny, 1, ck, mk1, twiddle(P, P->ny), ddesc, nr, 0, n > 0, 0, st), "batch kinetic")) != FSE_OK)
        return s;
      if (nl_on) {
        if ((s = chk(launch_xb(XP_E, P->nx, xa, twn, tw2n, ddesc, nr, t0, n, st), "batch density")) != FSE_OK) return s;
        if ((s = chk(launch_colb(2 * P->ny, 2, cg, mk2, twiddle(P, 2 * P->ny), ddesc, nr, 1, 0, 0, st), "batch kernel")) != FSE_OK)
          return s;
      } else {
        if ((s = chk(launch_xb(XP_INV, P->nx, xa, twn, tw2n, ddesc, nr, t0, n, st), "batch x")) != FSE_OK) return s;
      }
      if ((s = chk(launch_xb(XP_A, P->nx, xa, twn, tw2n, ddesc, nr, t0, n, st), "batch phase")) != FSE_OK) return s;
    }
    if ((s = chk(launch_colb(P->ny, 1, ck, mk1, twiddle(P, P->ny), ddesc, nr, 0, 0, 0, st), "batch kinetic")) != FSE_OK)
      return s;
    if ((s = chk(launch_xb(XP_INV, P->nx, xa, twn, tw2n, ddesc, nr, t0, nsteps, st), "batch x")) != FSE_OK) return s;
    if (multi) {
      cudaError_t e = cudaEventRecord(B->gdone[gi], st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st0, B->gdone[gi], 0);
      if (e != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string("group join: ") + cudaGetErrorString(e));
    }
  }
  *count = nl;
  return FSE_OK;
}

}  // namespace

extern "C" {

fse_status fse_batch_step(fse_batch_t B, void* const* psi, double t0, int nsteps) {
  if (!B || !psi || nsteps < 0) return FSE_ERR_INVALID;
  if (!B->ws || !B->precomputed) return bfail(B, FSE_ERR_INVALID, "fse_batch_precompute has not run");
  for (size_t r = 0; r < B->runs.size(); ++r)
    if (!psi[r] || reinterpret_cast<uintptr_t>(psi[r]) % 8 != 0) return bfail(B, FSE_ERR_INVALID, "bad psi pointer");
  if (nsteps == 0) return FSE_OK;
  cudaError_t e = cudaSuccess;
  if (B->gstream.empty()) {
    // the batch's own streams (one per group, one to replay graphs on) and events
    e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->cap_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->cap_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    for (size_t g = 0; g < B->groups.size() && e == cudaSuccess; ++g) {
      cudaStream_t s = nullptr;
      cudaEvent_t d = nullptr;
      e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      if (e == cudaSuccess) B->gstream.push_back(s);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d, cudaEventDisableTiming);
      if (e == cudaSuccess) B->gdone.push_back(d);
    }
    if (e != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string("batch streams: ") + cudaGetErrorString(e));
  }
  // this call's descriptor tables (wave-function pointers and run parameters)
  // and start time, stream-ordered on the caller's stream ahead of the kernels
  for (auto& G : B->groups) {
    fse_plan* P = G.plan;
    const int nr = (int)G.runs.size();
    B->desc.resize(nr);
    for (int k = 0; k < nr; ++k) {
      const int r = G.runs[k];
      const fse_params& p = B->runs[r];
      BatchRun d;
      d.psi = psi[r];
      d.spec = k == 0 ? P->ws_ptr(P->off_spec) : B->ptr(B->off_spec[r]);
      d.kin_half = k == 0 ? P->ws_ptr(P->off_kin_half) : B->ptr(B->off_kh[r]);
      d.kin_full = k == 0 ? P->ws_ptr(P->off_kin_full) : B->ptr(B->off_kf[r]);
      d.beta = p.beta;
      d.lam = p.lambda;
      d.dt = p.dt;
      d.omega = p.omega;
      d.gx2 = p.gamma[0] * p.gamma[0];
      d.gy2 = p.gamma[1] * p.gamma[1];
      B->desc[k] = d;
    }
    // pageable source: the copy is staged before the call returns
    e = cudaMemcpyAsync(B->ptr(G.off_desc), B->desc.data(), sizeof(BatchRun) * nr, cudaMemcpyHostToDevice, B->stream);
    if (e != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string("descriptor upload: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(B->ptr(B->off_t0), &t0, sizeof(double), cudaMemcpyHostToDevice, B->stream);
  if (e != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string("start time upload: ") + cudaGetErrorString(e));
  // the captured step sequence for nsteps (captured at the first call with this count)
  fse_batch::Graph* gr = nullptr;
  for (auto& g : B->graphs)
    if (g.nsteps == nsteps) gr = &g;
  if (!gr) {
    e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    long long nl = 0;
    const fse_status sq = batch_sequence(B, nsteps, B->cap, &nl);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(B->cap, &graph);
    if (sq != FSE_OK) {
      if (graph) cudaGraphDestroy(graph);
      return sq;
    }
    if (e != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    B->graphs.push_back({nsteps, exec, nl});
    gr = &B->graphs.back();
  }
  e = cudaEventRecord(B->cap_in, B->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(B->cap, B->cap_in, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(gr->exec, B->cap);
  if (e == cudaSuccess) e = cudaEventRecord(B->cap_out, B->cap);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(B->stream, B->cap_out, 0);
  if (e != cudaSuccess) return bfail(B, FSE_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  B->launches += gr->launches;
  return FSE_OK;
}

fse_status fse_batch_destroy(fse_batch_t B) {
  if (!B) return FSE_OK;
  for (auto& g : B->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& G : B->groups) fse_plan_destroy(G.plan);
  for (cudaStream_t s : B->gstream) cudaStreamDestroy(s);
  for (cudaEvent_t e : B->gdone) cudaEventDestroy(e);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->cap_in) cudaEventDestroy(B->cap_in);
  if (B->cap_out) cudaEventDestroy(B->cap_out);
  if (B->cap) cudaStreamDestroy(B->cap);
  delete B;
  return FSE_OK;
}

const char* fse_batch_error(fse_batch_t B) { return B ? B->err.c_str() : ""; }

long long fse_batch_launch_count(fse_batch_t B) { return B ? B->launches : 0; }

}  // extern "C"

// fse_internal.h -- the plan object behind fse_plan_t (host metadata only).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "fse.h"

struct fse_plan {
  fse_params p;
  cudaStream_t stream = nullptr;
  int device = 0;
  int dim = 2, nx = 0, ny = 0, nz = 1;
  int prec = FSE_F32;
  size_t rsize = 4, csize = 8;
  double h[3] = {0, 0, 0};
  long long sx = 0;  // row stride of the padded density spectrum S (elements)
  int chat_cx = 0;   // row stride of the C^ octant: nx + 1 rounded up to a multiple of 4 (16-byte rows)

  // Gaussian-sum fit (Eq. GS-Gene) and near-field integrals (Eq. taylor), float64 on the host
  std::vector<double> gs_w, gs_tau, gl_x, gl_w;
  double I0 = 0, I2 = 0;

  // workspace layout (byte offsets)
  std::vector<int> tw_len;
  std::vector<size_t> tw_off;
  size_t off_chat = 0, off_spec = 0, off_stage = 0, off_tmp = 0, off_red = 0, off_kin_half = 0, off_kin_full = 0;
  // fourth-order composition: kinetic table of the (w1 + w0) dt / 2 sub-step
  // between sub-steps (and the unused full-step output of its build)
  size_t off_kin_mid = 0, off_kin_mid2 = 0;
  size_t pre_w = 0, pre_tau = 0, pre_gl = 0, pre_g[3] = {0, 0, 0}, pre_cs = 0, pre_y = 0, pre_yw = 0;
  size_t ws_bytes = 0, psi_bytes = 0;

  // per-kernel timing (fse_plan_profile)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> recs;

  // ground state: page-locked copies of the device-side Krylov scalars (two
  // slots of 16 doubles) and the events that order their reads (created at
  // the first fse_ground_state call, released by fse_plan_destroy)
  double* gs_host = nullptr;
  cudaEvent_t gs_ev[2] = {nullptr, nullptr};
  // the stream the solve runs on (its BiCGStab iteration is captured as a
  // graph, which the legacy default stream does not allow) and its fork/join events
  cudaStream_t gs_stream = nullptr;
  cudaEvent_t gs_fork = nullptr, gs_join = nullptr;

  void* ws = nullptr;
  bool precomputed = false;
  long long launches = 0;
  std::string err;

  void* ws_ptr(size_t off) const { return static_cast<char*>(ws) + off; }
};

// Helpers shared by the translation units of the library (fse_api.cu).
namespace fse {
struct ColArgs;
struct MulArgs;
struct XArgs;
const double kPi = 3.14159265358979323846;
fse_status fail(fse_plan* p, fse_status st, const std::string& msg);
fse_status cuda_fail(fse_plan* p, cudaError_t e, const char* where);
fse_status launched(fse_plan* P, cudaError_t e, const char* where);
cudaEvent_t prof_begin(fse_plan* P);
void prof_end(fse_plan* P, int kind, cudaEvent_t a);
fse_status col(fse_plan* P, int kind, int N, int var, const ColArgs& a, const MulArgs& m);
fse_status xpass(fse_plan* P, int kind, const XArgs& a);
int tiles(fse_plan* P, int N, int ncols);
XArgs x_args(fse_plan* P, void* psi, void* spec);
void lattice_nodes(fse_plan* P, double ta, double tb, XArgs& a);
fse_status kinetic_yz(fse_plan* P, void* psi, double f, double dt);
fse_status nonlocal_yz(fse_plan* P, void* spec, double ta, double tb, bool integrated, const double* mdir,
                       double extra_scale);
bool has_nonlocal(const fse_plan* P);
fse_status validate_params(const fse_params& p);
fse_params effective_params(const fse_params& p);
void trap_coefficients(const fse_plan* P, double ta, double tb, const double* gam, double out[4]);
void dipole_matrix(const fse_plan* P, double ta, double tb, double M[6]);
fse_status run_steps(fse_plan* P, void* psi, double t0, int nsteps, const double* gps);
double* renorm_part(fse_plan* P);
// full transform of a field in the plan's layout: forward (dir < 0) or inverse
// (dir > 0), both unnormalised (fse_observables.cu)
template <typename Real> fse_status fft_full(fse_plan* P, void* buf, int dir);
// nonlocal potential Phi = U * |psi|^2 of the un-integrated kernel with dipole
// axis mdir (null: the plan's axis), written as a real field to phi (fse_observables.cu)
fse_status nonlocal_field(fse_plan* P, const void* psi, const double* mdir, void* phi);
const double* renorm_scale(fse_plan* P);
fse_status renorm_begin(fse_plan* P, const void* psi);
fse_status renorm_step(fse_plan* P, int count);
}  // namespace fse

// fse_api.cu -- the C ABI of include/fse.h: plan, workspace layout, precompute and step driver.
//
// Host work is limited to float64 scalars per step (the trap integral
// coefficients of Eq. int_poten and the dipole matrix of the time-integrated
// DDI kernel, Section 4.2) and to launching the pass kernels on the plan's
// stream; every grid-sized operation runs on the GPU.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fse.h"
#include "fse_internal.h"
#include "fse_passes.cuh"

namespace fse {
template <typename Real> cudaError_t launch_twiddles(void* tw, int L, cudaStream_t st);
template <typename Real>
cudaError_t launch_kin_table(void* half, void* full, int nx, int ny, int nz, double dkx, double dky, double dkz,
                             double s, double m2, double dt, cudaStream_t st);
cudaError_t launch_gs_axis(double* g, double* cs, double* ynode, double* ywt, const double* tau,
                           int Q, const double* glx, const double* glw, int ngl, int npan,
                           double W, int n, cudaStream_t st);
template <typename Real>
cudaError_t launch_chat(void* out, const double* w, const double* gx, const double* gy,
                        const double* gz, int Q, int nx, int ny, int nz, int cx, int dim, double dkx,
                        double dky, double dkz, double I0, double I2, cudaStream_t st);
}  // namespace fse

using namespace fse;

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Weights of the fourth-order triple jump (Yoshida 1990): w1 = 1/(2 - 2^{1/3}), w0 = 1 - 2 w1.
const double kTripleW1 = 1.0 / (2.0 - std::cbrt(2.0));
const double kTripleW0 = 1.0 - 2.0 * kTripleW1;

bool size_supported(int n) {
  static const int ok[] = {8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512};
  for (int v : ok)
    if (v == n) return true;
  return false;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// int_0^delta r^j exp(-tau^2 r^2) dr for j = 1..4.
double radial_gauss_moment(int j, double tau, double delta) {
  const double x = tau * tau * delta * delta;
  if (x < 2.0) {
    // sum_k (-x)^k / (k! (2k + j + 1)) * delta^{j+1}
    double term = 1.0, sum = 0.0;
    for (int k = 0; k < 80; ++k) {
      const double add = term / (2.0 * k + j + 1.0);
      sum += add;
      if (std::fabs(add) < 1e-18 * std::fabs(sum)) break;
      term *= -x / (k + 1.0);
    }
    return sum * std::pow(delta, j + 1);
  }
  const double t2 = tau * tau, e = std::exp(-x), sp = std::sqrt(kPi);
  switch (j) {
    case 1: return (1.0 - e) / (2.0 * t2);
    case 2: return sp * std::erf(tau * delta) / (4.0 * t2 * tau) - delta * e / (2.0 * t2);
    case 3: return (1.0 - (1.0 + x) * e) / (2.0 * t2 * t2);
    default:
      return 3.0 * sp * std::erf(tau * delta) / (8.0 * t2 * t2 * tau) -
             e * (delta * delta * delta / (2.0 * t2) + 3.0 * delta / (4.0 * t2 * t2));
  }
}

// sin(a * d) / a, continuous at a = 0.
double sin_over(double a, double d) {
  const double z = a * d;
  if (std::fabs(z) < 1e-6) return d * (1.0 - z * z / 6.0);
  return std::sin(z) / a;
}

struct StepScalars {
  double C1, S1, C2, S2, dt;
};

// Time integrals of cos/sin(Omega tau) and cos/sin(2 Omega tau) over [ta, tb].
StepScalars step_scalars(double omega, double ta, double tb) {
  StepScalars s;
  const double d = tb - ta, m = ta + tb;
  s.dt = d;
  s.C2 = std::cos(omega * m) * sin_over(omega, d);
  s.S2 = std::sin(omega * m) * sin_over(omega, d);
  s.C1 = std::cos(0.5 * omega * m) * 2.0 * sin_over(omega, 0.5 * d);
  s.S1 = std::sin(0.5 * omega * m) * 2.0 * sin_over(omega, 0.5 * d);
  return s;
}

}  // namespace

// ---------------------------------------------------------------------------
// internal helpers shared with other translation units
// ---------------------------------------------------------------------------
namespace fse {

fse_status fail(fse_plan* p, fse_status st, const std::string& msg) {
  if (p) p->err = msg;
  return st;
}

fse_status cuda_fail(fse_plan* p, cudaError_t e, const char* where) {
  return fail(p, FSE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

void trap_coefficients(const fse_plan* P, double ta, double tb, const double* gam, double out[4]) {
  const StepScalars s = step_scalars(P->p.omega, ta, tb);
  const double gx = gam ? gam[0] : P->p.gamma[0];
  const double gy = gam ? gam[1] : P->p.gamma[1];
  const double gz = (P->dim == 3) ? (gam ? gam[2] : P->p.gamma[2]) : 0.0;
  const double gx2 = gx * gx, gy2 = gy * gy;
  out[0] = 0.25 * (gx2 * (s.dt + s.C2) + gy2 * (s.dt - s.C2));
  out[1] = 0.25 * (gx2 * (s.dt - s.C2) + gy2 * (s.dt + s.C2));
  out[2] = 0.5 * (gx2 - gy2) * s.S2;
  out[3] = 0.5 * gz * gz * s.dt;
}

// M = int_{ta}^{tb} m m^T dtau, m(tau) = A(tau)^T n: (Mxx, Myy, Mzz, Mxy, Mxz, Myz).
void dipole_matrix(const fse_plan* P, double ta, double tb, double M[6]) {
  const StepScalars s = step_scalars(P->p.omega, ta, tb);
  const double n1 = P->p.dip_n[0], n2 = P->p.dip_n[1], n3 = P->p.dip_n[2];
  M[0] = n1 * n1 * (s.dt + s.C2) / 2 + n2 * n2 * (s.dt - s.C2) / 2 - n1 * n2 * s.S2;
  M[1] = n1 * n1 * (s.dt - s.C2) / 2 + n2 * n2 * (s.dt + s.C2) / 2 + n1 * n2 * s.S2;
  M[2] = n3 * n3 * s.dt;
  M[3] = (n1 * n1 - n2 * n2) * s.S2 / 2 + n1 * n2 * s.C2;
  M[4] = n3 * (n1 * s.C1 - n2 * s.S1);
  M[5] = n3 * (n1 * s.S1 + n2 * s.C1);
}

const void* twiddle(const fse_plan* P, int L) {
  for (size_t i = 0; i < P->tw_len.size(); ++i)
    if (P->tw_len[i] == L) return P->ws_ptr(P->tw_off[i]);
  return nullptr;
}

fse_status launched(fse_plan* P, cudaError_t e, const char* where) {
  if (e != cudaSuccess) return cuda_fail(P, e, where);
  ++P->launches;
  return FSE_OK;
}

cudaEvent_t take_event(fse_plan* P) {
  if (!P->ev_pool.empty()) {
    cudaEvent_t e = P->ev_pool.back();
    P->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Bracket one launch with events when profiling; `kind` is an fse_pass_kind.
cudaEvent_t prof_begin(fse_plan* P) {
  if (!P->profiling) return nullptr;
  cudaEvent_t a = take_event(P);
  if (a) cudaEventRecord(a, P->stream);
  return a;
}

void prof_end(fse_plan* P, int kind, cudaEvent_t a) {
  if (!a) return;
  cudaEvent_t b = take_event(P);
  if (!b) {
    P->ev_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, P->stream);
  P->recs.push_back({kind, a, b});
}

fse_status col(fse_plan* P, int kind, int N, int var, const ColArgs& a, const MulArgs& m) {
  if (!twiddle(P, N)) return fail(P, FSE_ERR_INVALID, "no twiddle table for a column pass length");
  cudaEvent_t ev = prof_begin(P);
  cudaError_t e = P->prec == FSE_F32
                      ? launch_colpass<float>(N, var, a, m, twiddle(P, N), P->stream)
                      : launch_colpass<double>(N, var, a, m, twiddle(P, N), P->stream);
  prof_end(P, kind, ev);
  return launched(P, e, "column pass");
}

fse_status xpass(fse_plan* P, int kind, const XArgs& a) {
  if (!twiddle(P, P->nx) || !twiddle(P, 2 * P->nx)) return fail(P, FSE_ERR_INVALID, "no twiddle table for the x pass");
  static const int kinds[8] = {FSE_PASS_XFWD, FSE_PASS_XINV, FSE_PASS_E, FSE_PASS_A, FSE_PASS_OTHER,
                               FSE_PASS_OTHER, FSE_PASS_OTHER, FSE_PASS_A};
  cudaEvent_t ev = prof_begin(P);
  cudaError_t e = P->prec == FSE_F32
                      ? launch_xpass<float>(kind, P->nx, a, twiddle(P, P->nx), twiddle(P, 2 * P->nx), P->stream)
                      : launch_xpass<double>(kind, P->nx, a, twiddle(P, P->nx), twiddle(P, 2 * P->nx), P->stream);
  prof_end(P, kinds[kind], ev);
  return launched(P, e, "x pass");
}

int tiles(fse_plan* P, int N, int ncols) {
  const int nc = P->prec == FSE_F32 ? colpass_ncol<float>(N) : colpass_ncol<double>(N);
  return (ncols + nc - 1) / nc;
}

// Passes over the R2C bins 0..nx of many planes: the last, nearly empty tile
// of every plane (nx + 1 = k NCOL + 1 bins for the usual sizes) is replaced by
// tail tiles holding that column of NCOL planes each.
ColArgs with_tail(fse_plan* P, ColArgs a, int N) {
  const int nc = P->prec == FSE_F32 ? colpass_ncol<float>(N) : colpass_ncol<double>(N);
  const int rem = a.ncols % nc;
  if (a.nplanes > 1 && rem > 0 && 2 * rem <= nc) {
    a.tiles_per_plane = a.ncols / nc;
    a.tail = rem;
  }
  return a;
}

XArgs x_args(fse_plan* P, void* psi, void* spec) {
  XArgs a;
  std::memset(&a, 0, sizeof(a));
  a.psi = psi;
  a.spec = spec;
  a.nlines = P->ny * (P->dim == 3 ? P->nz : 1);
  a.ny = P->ny;
  a.srow_mul = P->dim == 3 ? 2 : 1;
  a.sx = P->sx;
  a.use_spec = spec != nullptr;
  a.lo0 = P->p.lo[0];
  a.lo1 = P->p.lo[1];
  a.lo2 = P->dim == 3 ? P->p.lo[2] : 0.0;
  a.h0 = P->h[0];
  a.h1 = P->h[1];
  a.h2 = P->dim == 3 ? P->h[2] : 0.0;
  a.lat_amp = P->p.lat_amp;
  for (int j = 0; j < 3; ++j) a.lat_k[j] = j < P->dim ? P->p.lat_k[j] : 0.0;
  return a;
}

// Gauss-Legendre nodes of the window [ta, tb] for the lattice integral (Eq.
// int_poten by quadrature): weights and (cos, sin)(Omega tau_q). Without
// rotation the integrand is constant in time and one node is exact.
void lattice_nodes(fse_plan* P, double ta, double tb, XArgs& a) {
  if (P->p.lat_amp == 0.0) return;
  const int n = P->p.omega == 0.0 ? 1 : P->p.quad_nodes;
  std::vector<double> x, w;
  gauss_legendre(n, x, w);
  a.lat_nq = n;
  for (int q = 0; q < n; ++q) {
    const double t = 0.5 * (ta + tb) + 0.5 * (tb - ta) * x[q];
    a.lat_w[q] = 0.5 * (tb - ta) * w[q];
    a.lat_c[q] = std::cos(P->p.omega * t);
    a.lat_s[q] = std::sin(P->p.omega * t);
  }
}

// Kinetic sub-step of factor f (1: dt/2 as in Eqs. tssp1/tssp3; 2: two merged halves)
// on a field already transformed along x: fwd-y, fwd-z . phase . inv-z, inv-y
// (3D) or fwd-y . phase . inv-y (2D). On exit the field is x-spectral.
// f selects the plan's kinetic table: 1 the half step (dt/2; w1 dt/2 at order
// 4), 2 two merged half steps (dt; w1 dt), 3 the middle of the fourth-order
// composition ((w1 + w0) dt / 2); -1 the conjugate half step (adjoint).
fse_status kinetic_yz(fse_plan* P, void* psi, double f, double dt) {
  (void)dt;  // the phase tables were built with the plan's dt
  MulArgs m;
  std::memset(&m, 0, sizeof(m));
  m.mode = MUL_KIN;
  if (f == 1.0 || f == -1.0) {
    m.kin = P->ws_ptr(P->off_kin_half);
  } else if (f == 2.0) {
    m.kin = P->ws_ptr(P->off_kin_full);
  } else if (f == 3.0 && P->p.order == 4) {
    m.kin = P->ws_ptr(P->off_kin_mid);
  } else {
    return fail(P, FSE_ERR_INVALID, "kinetic table selector must be 1, 2, 3 (order 4) or -1");
  }
  m.conj = f < 0.0;
  m.lx = P->nx;
  fse_status st;
  if (P->dim == 2) {
    m.lp = 0;
    m.lr = P->ny;
    m.kin_sr = P->nx / 2 + 1;
    m.scale = 1.0 / ((double)P->nx * P->ny);
    ColArgs a{psi, 0, P->nx, 1, P->nx, P->ny, P->ny, tiles(P, P->ny, P->nx)};
    return col(P, FSE_PASS_KIN, P->ny, COL_KIN, a, m);
  }
  ColArgs ay{psi, (long long)P->nx * P->ny, P->nx, P->nz, P->nx, P->ny, P->ny, tiles(P, P->ny, P->nx)};
  if ((st = col(P, FSE_PASS_COL, P->ny, COL_FWD, ay, m)) != FSE_OK) return st;
  m.lp = P->ny;
  m.lr = P->nz;
  m.kin_sp = P->nx / 2 + 1;
  m.kin_sr = (long long)(P->nx / 2 + 1) * (P->ny / 2 + 1);
  m.scale = 1.0 / ((double)P->nx * P->ny * P->nz);
  ColArgs az{psi, P->nx, (long long)P->nx * P->ny, P->ny, P->nx, P->nz, P->nz, tiles(P, P->nz, P->nx)};
  if ((st = col(P, FSE_PASS_KIN, P->nz, COL_KIN, az, m)) != FSE_OK) return st;
  return col(P, FSE_PASS_COL, P->ny, COL_INV, ay, m);
}

// Padded forward transform along y (and z), kernel multiplier, inverse and crop
// of the x-half-spectrum in S (passes F, G, H; in 2D one fused y pass).
fse_status nonlocal_yz(fse_plan* P, void* spec, double ta, double tb, bool integrated, const double* mdir,
                       double extra_scale) {
  MulArgs m;
  std::memset(&m, 0, sizeof(m));
  const double d = integrated ? (tb - ta) : 1.0;
  const bool ddi = P->p.kernel == FSE_KERNEL_DDI3D || P->p.kernel == FSE_KERNEL_DDI2D;
  m.mode = ddi ? MUL_DDI : MUL_COULOMB;
  // M = int m m^T over the window (or m m^T of the axis mdir at one time)
  double M[6] = {0, 0, 0, 0, 0, 0};
  if (ddi) {
    if (integrated) {
      dipole_matrix(P, ta, tb, M);
    } else {
      M[0] = mdir[0] * mdir[0]; M[1] = mdir[1] * mdir[1]; M[2] = mdir[2] * mdir[2];
      M[3] = mdir[0] * mdir[1]; M[4] = mdir[0] * mdir[2]; M[5] = mdir[1] * mdir[2];
    }
  }
  m.lx = 2 * P->nx;
  m.dkx = 2 * kPi / (2.0 * (P->p.hi[0] - P->p.lo[0]));
  m.chat = P->ws_ptr(P->off_chat);
  m.chat_cx = P->chat_cx;
  m.chat_sp = P->chat_cx;
  m.chat_sr = (long long)P->chat_cx * (P->ny + 1);
  fse_status st;
  if (P->dim == 2) {
    m.lp = 0;
    m.lr = 2 * P->ny;
    m.dkr = 2 * kPi / (2.0 * (P->p.hi[1] - P->p.lo[1]));
    m.chat_sp = 0;
    m.chat_sr = P->chat_cx;
    m.scale = extra_scale / (4.0 * P->nx * P->ny);
    if (m.mode == MUL_COULOMB) {
      m.a0 = d * m.scale;
    } else {
      // 2D DDI: 3/2 (k^T M_perp k - n_3^2 d |k|^2) C^ (Eq. Kernel, 2D DDI row, with the
      // rotation-invariant n_3 term kept); columns carry k_x, rows k_y
      const double n3 = P->p.dip_n[2], c = 1.5 * m.scale;
      m.a0 = 0.0;
      m.q[0] = c * (M[0] - n3 * n3 * d);
      m.q[2] = c * (M[1] - n3 * n3 * d);
      m.q[4] = 2 * c * M[3];
    }
    ColArgs a{spec, 0, P->sx, 1, P->nx + 1, P->ny, P->ny, tiles(P, 2 * P->ny, P->nx + 1)};
    return col(P, FSE_PASS_KHAT, 2 * P->ny, COL_KHAT, a, m);
  }
  ColArgs af{spec, (long long)2 * P->ny * P->sx, P->sx, P->nz, P->nx + 1, P->ny, 2 * P->ny,
             tiles(P, 2 * P->ny, P->nx + 1)};
  if ((st = col(P, FSE_PASS_PAD, 2 * P->ny, COL_PADF, with_tail(P, af, 2 * P->ny), m)) != FSE_OK) return st;
  m.lp = 2 * P->ny;
  m.dkp = 2 * kPi / (2.0 * (P->p.hi[1] - P->p.lo[1]));
  m.lr = 2 * P->nz;
  m.dkr = 2 * kPi / (2.0 * (P->p.hi[2] - P->p.lo[2]));
  m.scale = extra_scale / (8.0 * P->nx * P->ny * P->nz);
  if (m.mode == MUL_COULOMB) {
    m.a0 = d * m.scale;
  } else {
    m.a0 = -d * m.scale;
    const double c = 3.0 * m.scale;
    m.q[0] = c * M[0];
    m.q[1] = c * M[1];
    m.q[2] = c * M[2];
    m.q[3] = 2 * c * M[3];
    m.q[4] = 2 * c * M[4];
    m.q[5] = 2 * c * M[5];
  }
  ColArgs ag{spec, P->sx, (long long)2 * P->ny * P->sx, 2 * P->ny, P->nx + 1, P->nz, P->nz,
             tiles(P, 2 * P->nz, P->nx + 1)};
  if ((st = col(P, FSE_PASS_KHAT, 2 * P->nz, COL_KHAT, with_tail(P, ag, 2 * P->nz), m)) != FSE_OK) return st;
  ColArgs ah{spec, (long long)2 * P->ny * P->sx, P->sx, P->nz, P->nx + 1, 2 * P->ny, P->ny,
             tiles(P, 2 * P->ny, P->nx + 1)};
  return col(P, FSE_PASS_PAD, 2 * P->ny, COL_CROPI, with_tail(P, ah, 2 * P->ny), m);
}

// Host-side checks of one parameter set (shared by fse_plan_create and
// fse_batch_create): ranges of Eq. SFSE and Eq. Kernel, supported sizes,
// finite scalars.
fse_status validate_params(const fse_params& p) {
  if (p.dim != 2 && p.dim != 3) return FSE_ERR_INVALID;
  if (!(p.s > 0.0) || !std::isfinite(p.s) || !(p.m >= 0.0) || !std::isfinite(p.m)) return FSE_ERR_INVALID;
  if (p.dt == 0.0 || !std::isfinite(p.dt)) return FSE_ERR_INVALID;
  if (!std::isfinite(p.omega) || !std::isfinite(p.beta) || !std::isfinite(p.lambda)) return FSE_ERR_INVALID;
  if (p.kernel < FSE_KERNEL_NONE || p.kernel > FSE_KERNEL_DDI2D) return FSE_ERR_INVALID;
  if (p.kernel == FSE_KERNEL_DDI3D && p.dim != 3) return FSE_ERR_INVALID;
  if (p.kernel == FSE_KERNEL_DDI2D && (p.dim != 2 || p.mu != 1.0)) return FSE_ERR_INVALID;
  if (p.prec != FSE_F32 && p.prec != FSE_F64) return FSE_ERR_INVALID;
  for (int j = 0; j < p.dim; ++j) {
    if (!std::isfinite(p.lo[j]) || !std::isfinite(p.hi[j]) || !(p.hi[j] > p.lo[j])) return FSE_ERR_INVALID;
    if (!std::isfinite(p.gamma[j])) return FSE_ERR_INVALID;
    if (!size_supported(p.n[j])) return FSE_ERR_UNSUPPORTED;
  }
  for (int j = 0; j < 3; ++j)
    if (!std::isfinite(p.dip_n[j]) || !std::isfinite(p.lat_k[j])) return FSE_ERR_INVALID;
  if (p.kernel == FSE_KERNEL_COULOMB && !(p.mu > 0.0 && p.mu <= p.dim - 1)) return FSE_ERR_INVALID;
  if (p.kernel == FSE_KERNEL_DDI3D && p.mu != 1.0) return FSE_ERR_INVALID;
  if (!std::isfinite(p.gs_delta) || !std::isfinite(p.gs_h) || !std::isfinite(p.gs_tmin)) return FSE_ERR_INVALID;
  if (p.renormalize != 0 && p.renormalize != 1) return FSE_ERR_INVALID;
  if (p.order != 0 && p.order != 2 && p.order != 4) return FSE_ERR_INVALID;
  if (!std::isfinite(p.lat_amp) || p.quad_nodes < 0 || p.quad_nodes > 16) return FSE_ERR_INVALID;
  return FSE_OK;
}

// The parameter set with the documented defaults filled in (0 = default).
fse_params effective_params(const fse_params& in) {
  fse_params p = in;
  if (p.gs_delta <= 0) p.gs_delta = 1e-3;
  if (p.gs_h <= 0) p.gs_h = 0.125;
  if (p.kernel == FSE_KERNEL_NONE) p.mu = 1.0;
  if (p.order == 0) p.order = 2;
  if (p.quad_nodes == 0) p.quad_nodes = 8;
  // the dropped tail of the sinc quadrature is ~ e^{mu t_min} / mu
  if (p.gs_tmin == 0) p.gs_tmin = -36.0 / p.mu;
  return p;
}

bool has_nonlocal(const fse_plan* P) { return P->p.kernel != FSE_KERNEL_NONE && P->p.lambda != 0.0; }

fse_status run_steps(fse_plan* P, void* psi, double t0, int nsteps, const double* gps) {
  if (nsteps == 0) return FSE_OK;
  const double dt = P->p.dt;
  void* spec = P->ws_ptr(P->off_spec);
  const bool nl = has_nonlocal(P);
  const bool rn = P->p.renormalize != 0;
  fse_status st;
  if (rn && (st = renorm_begin(P, psi)) != FSE_OK) return st;
  XArgs xa = x_args(P, psi, nl ? spec : nullptr);
  XArgs xe = xa;  // E or XI: also writes the mass partials when renormalising
  if (rn) xe.part = renorm_part(P);
  // tiles of pass E, one mass partial each
  const int ncx = P->prec == FSE_F32 ? xpass_ncol_x2<float>(P->nx) : xpass_ncol_x2<double>(P->nx);
  const int xblocks = (xa.nlines + ncx - 1) / ncx;
  // sub-steps of one step: TS2-GauSum itself, or the fourth-order triple jump
  // w1, w0, w1; the kinetic half steps between sub-steps and between steps merge
  const int nsub = P->p.order == 4 ? 3 : 1;
  const double wsub[3] = {nsub == 3 ? kTripleW1 : 1.0, kTripleW0, kTripleW1};
  if ((st = xpass(P, XP_FWD, xa)) != FSE_OK) return st;
  for (int n = 0; n < nsteps * nsub; ++n) {
    const int step = n / nsub, sub = n % nsub;
    double ta = t0 + step * dt;
    for (int i = 0; i < sub; ++i) ta += wsub[i] * dt;
    const double tb = sub == nsub - 1 ? t0 + (step + 1) * dt : ta + wsub[sub] * dt;
    const double kf = n == 0 ? 1.0 : (sub == 0 ? 2.0 : 3.0);
    if ((st = kinetic_yz(P, psi, kf, dt)) != FSE_OK) return st;
    if (nl) {
      if ((st = xpass(P, XP_E, xe)) != FSE_OK) return st;
      if ((st = nonlocal_yz(P, spec, ta, tb, true, nullptr, 1.0)) != FSE_OK) return st;
    } else {
      if ((st = xpass(P, XP_INV, xe)) != FSE_OK) return st;
    }
    if (rn && (st = renorm_step(P, xblocks)) != FSE_OK) return st;
    double pc[4];
    trap_coefficients(P, ta, tb, gps ? gps + (size_t)step * P->dim : nullptr, pc);
    XArgs xA = xa;
    xA.beta_dt = P->p.beta * (tb - ta);
    xA.lam = P->p.lambda;
    xA.pa = pc[0];
    xA.pb = pc[1];
    xA.pc = pc[2];
    xA.pe = pc[3];
    lattice_nodes(P, ta, tb, xA);
    if (rn) xA.scale = renorm_scale(P);
    if ((st = xpass(P, P->p.lat_amp != 0.0 ? XP_AL : XP_A, xA)) != FSE_OK) return st;
  }
  if ((st = kinetic_yz(P, psi, 1.0, dt)) != FSE_OK) return st;
  return xpass(P, XP_INV, xa);
}

}  // namespace fse

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* fse_status_string(fse_status s) {
  switch (s) {
    case FSE_OK: return "ok";
    case FSE_ERR_INVALID: return "invalid argument";
    case FSE_ERR_UNSUPPORTED: return "unsupported request";
    case FSE_ERR_NOMEM: return "workspace too small";
    case FSE_ERR_CUDA: return "CUDA error";
    case FSE_ERR_TIMEOUT: return "device wait timed out";
    case FSE_ERR_NONFINITE: return "non-finite value";
  }
  return "unknown status";
}

const char* fse_plan_error(fse_plan_t plan) { return plan ? plan->err.c_str() : ""; }

long long fse_plan_launch_count(fse_plan_t plan) { return plan ? plan->launches : 0; }

fse_status fse_plan_create(const fse_params* prm, void* stream, fse_plan_t* out, size_t* ws_bytes) {
  if (!out || !prm || !ws_bytes) return FSE_ERR_INVALID;
  *out = nullptr;
  *ws_bytes = 0;
  const fse_params& p = *prm;
  const fse_status vst = validate_params(p);
  if (vst != FSE_OK) return vst;
  fse_plan* P = new (std::nothrow) fse_plan();
  if (!P) return FSE_ERR_NOMEM;
  P->p = effective_params(p);
  P->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaGetDevice(&P->device);
  P->dim = p.dim;
  P->nx = p.n[0];
  P->ny = p.n[1];
  P->nz = p.dim == 3 ? p.n[2] : 1;
  P->prec = p.prec;
  P->rsize = p.prec == FSE_F32 ? 4 : 8;
  P->csize = 2 * P->rsize;
  for (int j = 0; j < 3; ++j) P->h[j] = j < p.dim ? (p.hi[j] - p.lo[j]) / p.n[j] : 0.0;
  P->sx = ((P->nx + 1 + 15) / 16) * 16;
  P->chat_cx = ((P->nx + 1 + 3) / 4) * 4;

  // Gaussian-sum nodes (Eq. GS-Gene): sinc quadrature of
  // r^-mu = (2 / Gamma(mu/2)) int exp(mu t - r^2 e^{2t}) dt in unit-box units, scaled.
  double wmax = 0.0;
  for (int j = 0; j < p.dim; ++j) wmax = std::fmax(wmax, p.hi[j] - p.lo[j]);
  const double sc = 0.5 * wmax;
  const double tmax = std::log(7.0 / P->p.gs_delta);
  const int Q = (int)std::ceil((tmax - P->p.gs_tmin) / P->p.gs_h) + 1;
  const double pref = 1.0 / (std::pow(2.0, p.dim - 1) * kPi);
  const double mu = P->p.mu;
  P->gs_w.resize(Q);
  P->gs_tau.resize(Q);
  for (int q = 0; q < Q; ++q) {
    const double t = P->p.gs_tmin + P->p.gs_h * q;
    P->gs_w[q] = pref * (2.0 * P->p.gs_h / std::tgamma(0.5 * mu)) * std::exp(mu * t) / std::pow(sc, mu);
    P->gs_tau[q] = std::exp(t) / sc;
  }
  // Near-field integrals I0, I2 over the ball of radius delta (Eq. taylor).
  const double del = P->p.gs_delta * sc;
  double s0 = 0.0, s2 = 0.0;
  for (int q = 0; q < Q; ++q) {
    if (p.dim == 2) {
      s0 += P->gs_w[q] * radial_gauss_moment(1, P->gs_tau[q], del);
      s2 += P->gs_w[q] * radial_gauss_moment(3, P->gs_tau[q], del);
    } else {
      s0 += P->gs_w[q] * radial_gauss_moment(2, P->gs_tau[q], del);
      s2 += P->gs_w[q] * radial_gauss_moment(4, P->gs_tau[q], del);
    }
  }
  // kernel part: pref * |S^{d-1}| * int_0^delta r^{d-1-mu} (1, r^2) dr
  const double sd = p.dim == 2 ? 2.0 * kPi : 4.0 * kPi, dd = p.dim;
  P->I0 = pref * sd * std::pow(del, dd - mu) / (dd - mu) - sd * s0;
  P->I2 = pref * sd * std::pow(del, dd + 2.0 - mu) / (dd + 2.0 - mu) - sd * s2;
  gauss_legendre(16, P->gl_x, P->gl_w);

  // Workspace layout.
  size_t off = 0;
  int lens[6] = {P->nx, P->ny, P->nz, 2 * P->nx, 2 * P->ny, 2 * P->nz};
  for (int i = 0; i < 6; ++i) {
    if (p.dim == 2 && (i == 2 || i == 5)) continue;
    bool seen = false;
    for (int L : P->tw_len) seen |= (L == lens[i]);
    if (seen) continue;
    P->tw_len.push_back(lens[i]);
    P->tw_off.push_back(off);
    // (cos, sin) and remainder; float plans also hold their (c, c, s, s)
    // broadcast copy for the packed column passes
    off = align256(off + 2 * (size_t)lens[i] * P->csize + (P->prec == FSE_F32 ? 2 * (size_t)lens[i] * 16 : 0));
  }
  P->off_chat = off;
  const size_t nchat = (size_t)P->chat_cx * (P->ny + 1) * (p.dim == 3 ? P->nz + 1 : 1);
  off = align256(off + nchat * P->rsize);
  const size_t kin_elems = (size_t)(P->nx / 2 + 1) * (P->ny / 2 + 1) * (p.dim == 3 ? P->nz / 2 + 1 : 1);
  P->off_kin_half = off;
  off = align256(off + kin_elems * P->csize);
  P->off_kin_full = off;
  off = align256(off + kin_elems * P->csize);
  if (P->p.order == 4) {
    P->off_kin_mid = off;
    off = align256(off + kin_elems * P->csize);
    P->off_kin_mid2 = off;
    off = align256(off + kin_elems * P->csize);
  }
  P->off_spec = off;
  const size_t spec_rows = (size_t)(p.dim == 3 ? P->nz * 2 * P->ny : P->ny);
  const size_t spec_bytes = spec_rows * P->sx * P->csize;
  // precompute scratch (float64), aliased with S
  const int nmax = std::max(P->nx, std::max(P->ny, P->nz));
  const int npan_max = nmax / 2 + 8;
  const int nyq = 16 * npan_max;
  size_t pre = 0;
  P->pre_w = pre;      pre = align256(pre + sizeof(double) * Q);
  P->pre_tau = pre;    pre = align256(pre + sizeof(double) * Q);
  P->pre_gl = pre;     pre = align256(pre + sizeof(double) * 32);
  for (int j = 0; j < 3; ++j) {
    P->pre_g[j] = pre;
    pre = align256(pre + sizeof(double) * (size_t)Q * (nmax + 1));
  }
  P->pre_cs = pre;     pre = align256(pre + sizeof(double) * (size_t)nyq * (nmax + 1));
  P->pre_y = pre;      pre = align256(pre + sizeof(double) * nyq);
  P->pre_yw = pre;     pre = align256(pre + sizeof(double) * nyq);
  off = align256(off + std::max(spec_bytes, pre));
  const size_t psi_bytes = (size_t)P->nx * P->ny * P->nz * P->csize;
  P->off_stage = off;
  off = align256(off + psi_bytes);
  P->off_tmp = off;
  off = align256(off + psi_bytes);
  P->off_red = off;
  off = align256(off + (16 * 65536 + 64) * sizeof(double));  // reduction partials
  P->ws_bytes = off;
  P->psi_bytes = psi_bytes;
  *ws_bytes = off;
  *out = P;
  return FSE_OK;
}

fse_status fse_plan_set_workspace(fse_plan_t P, void* ptr, size_t bytes) {
  if (!P || !ptr) return FSE_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(ptr) % 256 != 0) return fail(P, FSE_ERR_INVALID, "workspace not 256-byte aligned");
  if (bytes < P->ws_bytes) return fail(P, FSE_ERR_NOMEM, "workspace smaller than fse_plan_create reported");
  P->ws = ptr;
  P->precomputed = false;
  return FSE_OK;
}

fse_status fse_plan_set_stream(fse_plan_t P, void* stream) {
  if (!P) return FSE_ERR_INVALID;
  P->stream = reinterpret_cast<cudaStream_t>(stream);
  return FSE_OK;
}

fse_status fse_kernel_precompute(fse_plan_t P) {
  if (!P) return FSE_ERR_INVALID;
  if (!P->ws) return fail(P, FSE_ERR_INVALID, "no workspace attached");
  cudaError_t e;
  for (size_t i = 0; i < P->tw_len.size(); ++i) {
    e = P->prec == FSE_F32 ? launch_twiddles<float>(P->ws_ptr(P->tw_off[i]), P->tw_len[i], P->stream)
                           : launch_twiddles<double>(P->ws_ptr(P->tw_off[i]), P->tw_len[i], P->stream);
    if (launched(P, e, "twiddles") != FSE_OK) return FSE_ERR_CUDA;
  }
  {
    const double dk[3] = {2 * kPi / (P->p.hi[0] - P->p.lo[0]), 2 * kPi / (P->p.hi[1] - P->p.lo[1]),
                          P->dim == 3 ? 2 * kPi / (P->p.hi[2] - P->p.lo[2]) : 0.0};
    // (half, full) tables of a step length L: phases L/4 and L/2 times (|k|^2+m^2)^s.
    // Order 2: L = dt. Order 4: L = w1 dt (first/last half step, merged w1 dt
    // between steps), then L = (w1 + w0) dt for the middle half steps.
    const int nt = P->p.order == 4 ? 2 : 1;
    for (int it = 0; it < nt; ++it) {
      const double L = P->p.order == 4 ? (it == 0 ? kTripleW1 : kTripleW1 + kTripleW0) * P->p.dt : P->p.dt;
      void* kh = P->ws_ptr(it == 0 ? P->off_kin_half : P->off_kin_mid);
      void* kf = P->ws_ptr(it == 0 ? P->off_kin_full : P->off_kin_mid2);
      e = P->prec == FSE_F32
              ? launch_kin_table<float>(kh, kf, P->nx, P->ny, P->nz, dk[0], dk[1], dk[2], P->p.s, P->p.m * P->p.m,
                                        L, P->stream)
              : launch_kin_table<double>(kh, kf, P->nx, P->ny, P->nz, dk[0], dk[1], dk[2], P->p.s, P->p.m * P->p.m,
                                         L, P->stream);
      if (launched(P, e, "kinetic tables") != FSE_OK) return FSE_ERR_CUDA;
    }
  }
  if (P->p.kernel != FSE_KERNEL_NONE) {
    char* base = reinterpret_cast<char*>(P->ws_ptr(P->off_spec));
    double* dw = reinterpret_cast<double*>(base + P->pre_w);
    double* dtau = reinterpret_cast<double*>(base + P->pre_tau);
    double* dgl = reinterpret_cast<double*>(base + P->pre_gl);
    const int Q = (int)P->gs_w.size();
    std::vector<double> gl(32);
    for (int i = 0; i < 16; ++i) {
      gl[i] = P->gl_x[i];
      gl[16 + i] = P->gl_w[i];
    }
    // pageable sources: the copies are staged before these calls return
    if ((e = cudaMemcpyAsync(dw, P->gs_w.data(), sizeof(double) * Q, cudaMemcpyHostToDevice, P->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dtau, P->gs_tau.data(), sizeof(double) * Q, cudaMemcpyHostToDevice, P->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dgl, gl.data(), sizeof(double) * 32, cudaMemcpyHostToDevice, P->stream)) != cudaSuccess)
      return cuda_fail(P, e, "precompute upload");
    if ((e = cudaStreamSynchronize(P->stream)) != cudaSuccess) return cuda_fail(P, e, "precompute upload");
    const int n3[3] = {P->nx, P->ny, P->nz};
    for (int j = 0; j < P->dim; ++j) {
      const double W = P->p.hi[j] - P->p.lo[j];
      const int npan = n3[j] / 2 + 8;
      e = launch_gs_axis(reinterpret_cast<double*>(base + P->pre_g[j]), reinterpret_cast<double*>(base + P->pre_cs),
                         reinterpret_cast<double*>(base + P->pre_y), reinterpret_cast<double*>(base + P->pre_yw),
                         dtau, Q, dgl, dgl + 16, 16, npan, W, n3[j], P->stream);
      if (launched(P, e, "gausum tables") != FSE_OK) return FSE_ERR_CUDA;
      ++P->launches;
    }
    const double* gz = P->dim == 3 ? reinterpret_cast<double*>(base + P->pre_g[2]) : nullptr;
    const double dk[3] = {kPi / (P->p.hi[0] - P->p.lo[0]), kPi / (P->p.hi[1] - P->p.lo[1]),
                          P->dim == 3 ? kPi / (P->p.hi[2] - P->p.lo[2]) : 0.0};
    e = P->prec == FSE_F32
            ? launch_chat<float>(P->ws_ptr(P->off_chat), dw, reinterpret_cast<double*>(base + P->pre_g[0]),
                                 reinterpret_cast<double*>(base + P->pre_g[1]), gz, Q, P->nx, P->ny, P->nz,
                                 P->chat_cx, P->dim, dk[0], dk[1], dk[2], P->I0, P->I2, P->stream)
            : launch_chat<double>(P->ws_ptr(P->off_chat), dw, reinterpret_cast<double*>(base + P->pre_g[0]),
                                  reinterpret_cast<double*>(base + P->pre_g[1]), gz, Q, P->nx, P->ny, P->nz,
                                  P->chat_cx, P->dim, dk[0], dk[1], dk[2], P->I0, P->I2, P->stream);
    if (launched(P, e, "kernel transform") != FSE_OK) return FSE_ERR_CUDA;
  }
  P->precomputed = true;
  return FSE_OK;
}

fse_status fse_step(fse_plan_t P, void* psi, double t0, int nsteps, const double* gps) {
  if (!P || !psi || nsteps < 0) return FSE_ERR_INVALID;
  if (!P->ws || !P->precomputed) return fail(P, FSE_ERR_INVALID, "fse_kernel_precompute has not run");
  if (reinterpret_cast<uintptr_t>(psi) % P->csize != 0) return fail(P, FSE_ERR_INVALID, "psi misaligned");
  return run_steps(P, psi, t0, nsteps, gps);
}

fse_status fse_step_host(fse_plan_t P, void* psi_host, double t0, int nsteps, const double* gps) {
  if (!P || !psi_host || nsteps < 0) return FSE_ERR_INVALID;
  if (!P->ws || !P->precomputed) return fail(P, FSE_ERR_INVALID, "fse_kernel_precompute has not run");
  void* d = P->ws_ptr(P->off_stage);
  cudaError_t e = cudaMemcpyAsync(d, psi_host, P->psi_bytes, cudaMemcpyHostToDevice, P->stream);
  if (e != cudaSuccess) return cuda_fail(P, e, "host-to-device copy");
  fse_status st = run_steps(P, d, t0, nsteps, gps);
  if (st != FSE_OK) return st;
  e = cudaMemcpyAsync(psi_host, d, P->psi_bytes, cudaMemcpyDeviceToHost, P->stream);
  if (e != cudaSuccess) return cuda_fail(P, e, "device-to-host copy");
  e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return cuda_fail(P, e, "stream synchronize");
  return FSE_OK;
}

fse_status fse_plan_profile(fse_plan_t P, int enable) {
  if (!P) return FSE_ERR_INVALID;
  P->profiling = enable != 0;
  return FSE_OK;
}

fse_status fse_plan_profile_read(fse_plan_t P, double* ms, long long* count) {
  if (!P || !ms || !count) return FSE_ERR_INVALID;
  for (int k = 0; k < FSE_NPASS; ++k) {
    ms[k] = 0.0;
    count[k] = 0;
  }
  fse_status st = FSE_OK;
  for (auto& r : P->recs) {
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && st == FSE_OK) st = cuda_fail(P, e, "profile read");
    if (r.kind >= 0 && r.kind < FSE_NPASS) {
      ms[r.kind] += t;
      count[r.kind] += 1;
    }
    P->ev_pool.push_back(r.a);
    P->ev_pool.push_back(r.b);
  }
  P->recs.clear();
  return st;
}

fse_status fse_plan_destroy(fse_plan_t P) {
  if (!P) return FSE_OK;
  for (auto& r : P->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : P->ev_pool) cudaEventDestroy(e);
  for (auto e : P->gs_ev)
    if (e) cudaEventDestroy(e);
  if (P->gs_host) cudaFreeHost(P->gs_host);
  if (P->gs_fork) cudaEventDestroy(P->gs_fork);
  if (P->gs_join) cudaEventDestroy(P->gs_join);
  if (P->gs_stream) cudaStreamDestroy(P->gs_stream);
  delete P;
  return FSE_OK;
}

}  // extern "C"

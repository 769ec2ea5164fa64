/*
 * fse.h -- C ABI of the GB300 TS2-GauSum split-step library.
 *
 * The library advances the space-fractional nonlinear Schroedinger /
 * Gross-Pitaevskii equation with rotation and nonlocal (Coulomb or dipolar)
 * interaction (Antoine, Tang & Zhang, arXiv 1512.03210, Eqs. SFSE and
 * NonLocalPot) by the second-order time-splitting Fourier pseudo-spectral
 * scheme TS2-GauSum (Section 4.2, Eqs. tssp1-tssp3), written in the rotating
 * Lagrangian coordinates x~ = A(t)^T x (Eqs. Amatrix, transform, FSE1_Rot),
 * with the nonlocal term evaluated by the Gaussian-sum method (Section 2,
 * Eqs. key_form00, GS-Gene, FourSeriB3, tensor, taylor).
 *
 * Conventions shared by every call
 * - The unknown is phi(x~, t) = psi(A(t) x~, t) on the box B = prod [lo_j, hi_j)
 *   (Eq. transform79), sampled at x~_l = lo + l h, l = 0..n-1, h = (hi-lo)/n.
 * - Layout: row-major [nz][ny][nx] (3D) or [ny][nx] (2D), x fastest,
 *   interleaved complex: float2 for FSE_F32 plans, double2 for FSE_F64 plans.
 * - Device pointers are CUDA device memory on the plan's device; the caller
 *   owns every buffer (wave function, cotangent, workspace). The library
 *   allocates no device memory: all scratch lives in the caller's workspace.
 * - Calls are asynchronous on the plan's stream unless stated otherwise; a
 *   CUDA launch or copy error is reported as FSE_ERR_CUDA by the call that
 *   observes it. No call throws across the ABI.
 * - Supported grid sizes per axis: n in {8,12,16,24,32,48,64,96,128,192,256,
 *   384,512}; padded lengths 2n are handled internally.
 * - A plan is not thread-safe: one host thread at a time per plan.
 */
#ifndef FSE_H_
#define FSE_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fse_plan* fse_plan_t;

typedef enum {
  FSE_OK = 0,
  FSE_ERR_INVALID = 1,      /* a null pointer, a bad parameter or call order */
  FSE_ERR_UNSUPPORTED = 2,  /* a valid request the library does not implement */
  FSE_ERR_NOMEM = 3,        /* the workspace given is smaller than required */
  FSE_ERR_CUDA = 4,         /* a CUDA runtime call failed (message in fse_plan_error) */
  FSE_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
  FSE_ERR_NONFINITE = 6     /* a reduction met NaN or Inf */
} fse_status;

typedef enum { FSE_KERNEL_NONE = 0, FSE_KERNEL_COULOMB = 1, FSE_KERNEL_DDI3D = 2, FSE_KERNEL_DDI2D = 3 } fse_kernel;
typedef enum { FSE_F32 = 0, FSE_F64 = 1 } fse_prec;

/*
 * Problem parameters (Eq. SFSE; Eq. Kernel; Eq. harm_poten; Section 4.2).
 *   dim        2 or 3
 *   n[j], lo[j], hi[j]   grid of axis j (x, y, z); n[2] ignored for dim 2
 *   s, m       fractional order s > 0 and mass m >= 0 of (-Lap + m^2)^s / 2
 *   omega      rotation speed Omega of the -Omega L_z term (Eq. Amatrix)
 *   beta       local cubic interaction strength
 *   lambda     nonlocal interaction strength
 *   dt         time step (may be negative: the scheme is time-reversible)
 *   kernel     fse_kernel: none, Coulomb-type 1/(2^{d-1} pi |x|^mu), 3D DDI
 *              (-1 + 3 (n.k)^2/|k|^2) or 2D DDI (3 [(n_perp.k)^2 - n3^2 |k|^2] /
 *              (2|k|)), Eq. Kernel
 *   mu         exponent of the Coulomb-type kernel, 0 < mu <= dim - 1 (Eq.
 *              Kernel); the DDI kernels are built on mu = 1
 *   dip_n[3]   dipole axis n (unit vector) for FSE_KERNEL_DDI3D and
 *              FSE_KERNEL_DDI2D (2D: n_perp = (n1, n2) in the plane, n3 normal)
 *   gamma[3]   harmonic trap frequencies (Eq. harm_poten)
 *   gs_delta, gs_h, gs_tmin  Gaussian-sum fit (Eq. GS-Gene): near-field
 *              radius in unit-box units, sinc-quadrature step and lower
 *              end; 0 selects 1e-3, 0.125, -36/mu
 *   prec       fse_prec: arithmetic of the split step
 *   renormalize  0: the paper's scheme; 1: after each step rescale psi so that
 *              its float64 mass equals the mass at the start of the fse_step
 *              call (holds the float32 mass drift; not part of the paper)
 *   order      time-splitting order: 0 or 2 = TS2-GauSum (Strang, Eqs.
 *              tssp1-tssp3); 4 = symmetric composition of three TS2-GauSum
 *              sub-steps of lengths w1 dt, w0 dt, w1 dt with w1 = 1/(2 - 2^{1/3})
 *              and w0 = 1 - 2 w1 (the higher-order extension of Section 4.2;
 *              not available to fse_step_adjoint and the batch calls)
 *   lat_amp, lat_k[3]  optical lattice added to the harmonic trap,
 *              V += lat_amp sum_v sin^2(lat_k[v] x_v) in the lab frame (the
 *              harmonic-plus-lattice potential of Section 3.3); 0 = none. Its
 *              time integral over each step (Eq. int_poten) is taken by
 *              Gauss-Legendre quadrature, as Section 4.2 prescribes for a
 *              general V; not available to the batch calls
 *   quad_nodes  Gauss-Legendre nodes of that quadrature, 1..16; 0 selects 8
 */
typedef struct {
  int dim;
  int n[3];
  double lo[3], hi[3];
  double s, m, omega, beta, lambda, dt;
  int kernel;
  double mu;
  double dip_n[3];
  double gamma[3];
  double gs_delta, gs_h, gs_tmin;
  int prec;
  int renormalize;
  int order;
  double lat_amp;
  double lat_k[3];
  int quad_nodes;
} fse_params;

/* Observables (Eqs. mass, energy, AME, CoM, ConWidth) at time t, in float64.
 * energy = e_kin + e_pot + e_int + e_non + e_rot with e_rot = -Omega <L_z>;
 * xc and width are in the frame of Eq. SFSE (x = A(t) x~); unused z entries 0. */
typedef struct {
  double mass, e_kin, e_pot, e_int, e_non, e_rot, energy, lz;
  double xc[3], width[3];
} fse_obs;

/* Validate *params, create a plan bound to cuda_stream (a cudaStream_t; NULL
 * = legacy default stream) on the current CUDA device, and return in
 * *workspace_bytes the size of the device workspace the caller must supply.
 * Errors: FSE_ERR_INVALID (null pointers, dim, s <= 0, box, dt = 0, kernel
 * and dim mismatch, mu outside (0, dim - 1] for the Coulomb-type kernel or
 * mu != 1 for a DDI kernel, order not 0, 2 or 4, non-finite lattice
 * parameters or quad_nodes outside 0..16), FSE_ERR_UNSUPPORTED (a size outside the
 * supported set). On error *out is NULL. */
fse_status fse_plan_create(const fse_params* params, void* cuda_stream, fse_plan_t* out,
                           size_t* workspace_bytes);

/* Attach caller-owned device memory of at least workspace_bytes bytes
 * (256-byte aligned) to the plan; the plan keeps the pointer, not ownership.
 * Errors: FSE_ERR_INVALID (null, misaligned), FSE_ERR_NOMEM (too small). */
fse_status fse_plan_set_workspace(fse_plan_t plan, void* dev_ptr, size_t bytes);

/* Once per plan, after set_workspace: build in the workspace the twiddle
 * tables, the Gaussian-sum tables g_q(k_j) (Eq. tensor) and the kernel
 * transform C^(k) = sum_q w_q prod_j g_q(k_j) + I0 - I2 |k|^2/(2d) on the
 * non-negative padded frequencies (Section 2, Eqs. GS-Gene, tensor, taylor),
 * in float64, stored in the plan's precision. Asynchronous. */
fse_status fse_kernel_precompute(fse_plan_t plan);

/* Advance psi (device, plan layout, in place) by nsteps TS2-GauSum steps
 * from t0 (Eqs. tssp1-tssp3; adjacent kinetic half steps of consecutive
 * steps are merged). gamma_per_step (host, nullable) holds [nsteps][dim]
 * trap frequencies, constant over each step (the parameters' gamma when
 * NULL). Asynchronous. Errors: FSE_ERR_INVALID (null plan/psi, nsteps < 0,
 * precompute not run). */
fse_status fse_step(fse_plan_t plan, void* psi, double t0, int nsteps,
                    const double* gamma_per_step);

/* As fse_step with psi in HOST memory (pinned or pageable): copies psi into
 * the workspace's staging slot, steps, copies it back and synchronises the
 * plan's stream before returning. */
fse_status fse_step_host(fse_plan_t plan, void* psi_host, double t0, int nsteps,
                         const double* gamma_per_step);

/* Pull a cotangent back through the single step t_n -> t_n + dt taken from
 * psi_n (device, unchanged). g (device, plan layout) holds on entry the
 * cotangent dJ/dRe psi_{n+1} + i dJ/dIm psi_{n+1} and on return the cotangent
 * at psi_n. gamma_n (host, nullable, [dim]) are the step's trap frequencies;
 * dgamma_n (host, nullable, [dim]) receives dJ/dgamma_n (the call then
 * synchronises the stream). The paper has no adjoint: this is the transpose
 * of the real-linearised map of Eqs. tssp1-tssp3. Errors: FSE_ERR_INVALID
 * (null or misaligned buffers, precompute not run), FSE_ERR_UNSUPPORTED
 * (a plan with renormalize = 1 or order 4). Uses the workspace's scratch wave function
 * and spectrum, so it must not overlap other calls on the same plan. */
fse_status fse_step_adjoint(fse_plan_t plan, const void* psi_n, void* g, double t_n,
                            const double* gamma_n, double* dgamma_n);

/* Observables of psi (device, unchanged) at time t with trap frequencies
 * gamma (host, nullable, [dim]); float64 reductions on the device, one
 * device-to-host copy; synchronises the plan's stream. */
fse_status fse_observables(fse_plan_t plan, const void* psi, double t, const double* gamma,
                           fse_obs* out);

/* Rebind the plan to another stream (a cudaStream_t on the same device). */
fse_status fse_plan_set_stream(fse_plan_t plan, void* cuda_stream);

/* Release the plan's host memory (never the caller's workspace). NULL is a no-op. */
fse_status fse_plan_destroy(fse_plan_t plan);

/* Static description of a status code. */
const char* fse_status_string(fse_status status);

/* Detail of the last error recorded on this plan ("" if none). */
const char* fse_plan_error(fse_plan_t plan);

/* Number of kernel launches the plan has issued since creation. */
long long fse_plan_launch_count(fse_plan_t plan);

/* Pass kinds for per-kernel timing (see fse_plan_profile). */
typedef enum {
  FSE_PASS_XFWD = 0,    /* forward FFT along x (start of a call) */
  FSE_PASS_XINV = 1,    /* inverse FFT along x (end of a call, or no nonlocal term) */
  FSE_PASS_E = 2,       /* inverse x, density, zero-padded real-to-complex x transform */
  FSE_PASS_A = 3,       /* complex-to-real x transform, potential phase, forward x */
  FSE_PASS_COL = 4,     /* plain transform along y of the wave function */
  FSE_PASS_KIN = 5,     /* forward, kinetic phase, inverse along the last axis */
  FSE_PASS_PAD = 6,     /* zero-padded forward / cropped inverse along y of the density */
  FSE_PASS_KHAT = 7,    /* forward, kernel transform, inverse along the last padded axis */
  FSE_PASS_PRE = 8,     /* once-per-plan tables */
  FSE_PASS_OTHER = 9,   /* observables and adjoint kernels */
  FSE_NPASS = 10
} fse_pass_kind;

/* Per-kernel timing (tracing). With enable != 0 every later launch of the
 * plan is bracketed by two CUDA events on the plan's stream; enable = 0 stops
 * recording. Adds a few microseconds of host time per launch. */
fse_status fse_plan_profile(fse_plan_t plan, int enable);

/* Synchronise on the recorded events and return, per fse_pass_kind, the
 * summed device time in milliseconds (ms[FSE_NPASS]) and the number of
 * launches (count[FSE_NPASS]) since the last read; then clear the record. */
fse_status fse_plan_profile_read(fse_plan_t plan, double* ms, long long* count);

/* ---- Batched 2D runs ------------------------------------------------------
 * Many independent 2D runs (each the scheme of Section 4.2, Eqs. tssp1-tssp3,
 * with its own grid size, s, m, Omega, beta, lambda, dt and trap) advanced
 * together: runs of equal grid size share one launch per pass and one kernel
 * transform; a run advanced in a batch is bit-identical to the same run
 * advanced alone with fse_step. Requirements: dim 2, FSE_F32, renormalize 0, order 2, no lattice,
 * one box, one kernel (none or Coulomb), one exponent mu and one Gaussian-sum
 * fit (gs_delta, gs_h, gs_tmin after defaults) for the whole batch. */
typedef struct fse_batch* fse_batch_t;

/* Validate runs[0..nruns) (every run gets the parameter checks of
 * fse_plan_create), create the batch on cuda_stream and return the device
 * workspace size it needs. Errors: FSE_ERR_INVALID (null, nruns <= 0, DDI
 * kernel, a run that fse_plan_create would reject as invalid),
 * FSE_ERR_UNSUPPORTED (a requirement above not met, or an unsupported grid
 * size). */
fse_status fse_batch_create(const fse_params* runs, int nruns, void* cuda_stream, fse_batch_t* out,
                            size_t* workspace_bytes);
/* Attach caller-owned device memory (256-byte aligned, at least the size
 * reported). Errors as fse_plan_set_workspace. */
fse_status fse_batch_set_workspace(fse_batch_t batch, void* dev_ptr, size_t bytes);
/* Once per batch: twiddles and Gaussian-sum kernel transform per grid size
 * (Section 2) and kinetic phase tables per run. Asynchronous. */
fse_status fse_batch_precompute(fse_batch_t batch);
/* Advance every run by nsteps steps from t0. psi is a HOST array of nruns
 * DEVICE pointers, one wave function per run in that run's layout [ny][nx]
 * (float2). The first call with a given nsteps captures its launches (every
 * size group on a stream of its own) into a CUDA graph, on a stream the batch
 * owns; later calls with that nsteps only upload the pointers and t0 and
 * replay the graph. The capture uses thread-local mode, so the first call with
 * a new nsteps must not be made while this thread captures another stream.
 * Asynchronous, ordered on the batch's stream. Errors: FSE_ERR_INVALID (null
 * or misaligned pointers, precompute not run), FSE_ERR_CUDA (capture or
 * launch failure). */
fse_status fse_batch_step(fse_batch_t batch, void* const* psi, double t0, int nsteps);
/* Release the batch's host memory (never the workspace). */
fse_status fse_batch_destroy(fse_batch_t batch);
/* Detail of the last error on the batch ("" if none). */
const char* fse_batch_error(fse_batch_t batch);
/* Kernel launches issued by the batch since creation. */
long long fse_batch_launch_count(fse_batch_t batch);

/* ---------------------------------------------------------------------------
 * Ground state by GF-GauSum (Section 3.2, Eqs. gf-eq1 to gffg33): the
 * gradient flow with discrete normalisation in the laboratory frame, each
 * backward-Euler step (1/dt + (-Lap+m^2)^s/2 + V + beta|phi^n|^2 + lambda Phi^n
 * - Omega L_z) phi^(1) = phi^n/dt solved by BiCGStab on the system left-
 * preconditioned with P_Delta = [1/dt + (-Lap+m^2)^s/2]^-1 (Eq. precond_type1),
 * then phi^{n+1} = phi^(1)/||phi^(1)||. It uses the plan's grid, s, m, Omega,
 * beta, lambda, kernel (Phi = U * |phi^n|^2 with the un-rotated axis n), the
 * trap gamma and the optical lattice; the plan's dt and order play no part.
 * ------------------------------------------------------------------------- */
typedef struct {
  double dt;        /* gradient-flow time step (> 0) */
  int max_outer;    /* at most this many normalised steps */
  double tol;       /* stop once max |phi^{n+1} - phi^n| / dt <= tol */
  int max_inner;    /* BiCGStab iterations per step, at most */
  double inner_tol; /* BiCGStab stops at ||r|| <= inner_tol ||b|| */
} fse_gs_opts;
typedef struct {
  int outer;        /* normalised steps taken */
  int inner;        /* BiCGStab iterations, all steps */
  double change;    /* max |phi^{n+1} - phi^n| / dt of the last step */
  double residual;  /* ||r|| / ||b|| of the last inner solve */
} fse_gs_info;
/* Device workspace (bytes, 256-byte aligned) that fse_ground_state needs for
 * its Krylov vectors on this plan: ten complex and three real fields. */
fse_status fse_ground_state_workspace(fse_plan_t plan, size_t* bytes);
/* psi (device, plan layout): initial guess on entry (scaled to unit mass),
 * the last iterate on return. The BiCGStab scalars stay on the device, so
 * the launches of one iteration are captured once per call as a CUDA graph
 * and replayed; the host reads the scalars one iteration behind the GPU (one
 * extra, idempotent iteration may run after convergence). The solve runs on
 * a stream the plan creates at the first call, ordered after and before the
 * plan's stream, and the call returns with the plan's stream synchronised. It
 * uses the plan's scratch field and spectrum, and keeps that stream, four
 * events and 256 bytes of page-locked host memory on the plan (released by
 * fse_plan_destroy). info (nullable) receives the counts. Errors: FSE_ERR_INVALID (null
 * or misaligned buffers, precompute not run, dt <= 0, negative counts or
 * tolerances, zero initial field), FSE_ERR_NOMEM (workspace too small),
 * FSE_ERR_NONFINITE (the iteration produced a non-finite field). */
fse_status fse_ground_state(fse_plan_t plan, void* psi, void* workspace, size_t workspace_bytes,
                            const fse_gs_opts* opts, fse_gs_info* info);

/* Initial data of the dynamics runs (Section 4.3, Eq. ini_dyn): psi <-
 * psi(x - x0) exp(i k . x), the translation taken spectrally (the Nyquist mode
 * of each axis takes cos(k_N x0_j), the mean of its two aliases) and the kick
 * exactly; e.g. x0 = (3, 3), k = v0 (0.8, 0.5) turns a ground state into the
 * paper's shifted and moving state. x0 and k are host arrays [dim] (nullable:
 * no shift / no kick); psi is device, plan layout. Asynchronous. Errors:
 * FSE_ERR_INVALID (null or misaligned psi, precompute not run, non-finite x0
 * or k). */
fse_status fse_shift_kick(fse_plan_t plan, void* psi, const double* x0, const double* k);

/* Largest npoints accepted by fse_mass_noalloc (4096 partials of 65536 points). */
#define FSE_NOALLOC_MAX_POINTS (4096LL * 65536LL)

/* Mass h^d sum |psi|^2 of npoints complex values at psi (device, float2 when
 * prec = FSE_F32, double2 when FSE_F64), written as one double to mass_out
 * (device) on cuda_stream (NULL = legacy default stream); cell_volume is h^d.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- e.g. a monitoring hook between steps inside
 * a framework whose caching allocator owns the device memory, where a
 * cudaMalloc would fail or synchronise the device -- and that have no plan
 * workspace. It allocates nothing: its scratch is a static 32 KB device array
 * (4096 float64 partials) that every GPU loading the library holds until the
 * process exits. The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture. Every call overwrites the partials it reads, so
 * nothing needs clearing, but all calls share the one array: calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * ordered by the caller. Asynchronous. Errors: FSE_ERR_INVALID (null or
 * misaligned pointers, npoints < 0, prec), FSE_ERR_UNSUPPORTED (npoints >
 * FSE_NOALLOC_MAX_POINTS, the size the static scratch holds; or a device
 * index >= 64), FSE_ERR_CUDA (symbol lookup or launch failure). */
fse_status fse_mass_noalloc(const void* psi, int prec, long long npoints, double cell_volume,
                            double* mass_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FSE_H_ */

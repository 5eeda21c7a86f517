/*
 * etd.h -- C ABI of the GB300 ETD step for the phase-field model of multicomponent
 * membranes (Luo, Qiao, Zhao: exponential time differencing schemes for a phase-field
 * model of multicomponent membranes).
 *
 * The library advances the phase field phi (membrane) and the protein density u on a
 * periodic 2D/3D grid with the FFT-based stabilised ETD1/ETDRK2 schemes of Sec. 3.3 and
 * Algorithm 1, or (model = ETD_MODEL_FIXED) the protein density alone on a frozen membrane.
 * model = ETD_MODEL_FIXED_SQRTG runs the frozen-membrane scheme of Sec. 2.2 instead: the
 * equation divided by g^{1/2}, d(g^{1/2} u)/dt + L_phi (g^{1/2} u) = R_phi(u) with
 * L_phi = B - eps_u g^{-1/2} Delta_{S,h} g^{-1/2} (B = params.B2), ETD1 (Eq. (2.8)) or ETDRK2
 * (Eq. (2.9)-(2.10)), on the narrow band with zero-flux band edges; phi_j(tau L_phi) acts
 * through Lanczos Krylov spaces (L_phi is not diagonal in Fourier space).  u off the band is
 * left unchanged.
 *
 * Conventions shared by every entry point:
 *  - Fields are dense, C-ordered, x fastest: index (k*Ny + j)*Nx + i for 3D, j*Nx + i for
 *    2D.  Grid point (i,j,k) sits at (-X + i*hx, -Y + j*hy, -Z + k*hz), h = 2X/N (Sec. 2.1).
 *  - Element type is double for ETD_FP64 and float for ETD_FP32_MIXED.  FP32_MIXED keeps
 *    the phi-function tables (built in FP64, rounded once), every reduction (mass, volume,
 *    energy, CG dot products) and the scalar constraint terms in FP64.
 *  - Field pointers are DEVICE pointers owned by the caller (for example PyTorch tensors
 *    on the plan's device).  They must stay valid until the enqueued work completes.  The
 *    library never frees them.  All work is enqueued on the stream given to etd_plan.
 *  - The plan owns its workspace (spectra, band list, CG vectors, tables) and frees it
 *    in etd_free.  A plan is not thread-safe; use one plan per host thread.
 *  - No C++ exception crosses this boundary.  Errors come back as etd_status; the
 *    message of the last error of the calling thread is returned by etd_last_error().
 *  - Supported grids: every N a power of two from 8 to 256, or 96, along x and y; N_z = 1
 *    (2D) or one of the same lengths; cubic boxes X = Y (= Z).  The FP32-mixed coupled form
 *    needs powers of two.  Other sizes return ETD_EINVAL.  (etd_fft_forward_noalloc: powers
 *    of two only.)
 */
#ifndef ETD_H
#define ETD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct etd_plan_s *etd_plan_t;

typedef enum {
  ETD_OK = 0,
  ETD_EINVAL = 1,      /* invalid argument or unsupported size                        */
  ETD_ENOMEM = 2,      /* device allocation failed                                    */
  ETD_ECUDA = 3,       /* a CUDA runtime call failed                                  */
  ETD_ENONFINITE = 4,  /* a non-finite value appeared in the state                    */
  ETD_ENOTCONV = 5,    /* band CG did not reach cg_rtol within cg_maxit iterations     */
  ETD_ETIMEOUT = 6,    /* a bounded device wait gave up (grid barrier, tensor copy)     */
  ETD_EMBP = 7         /* reserved, never returned: the spectral schemes of Sec. 3 do not
                          guarantee the maximum bound (etd_diag reports max |2U-1|)      */
} etd_status;

typedef enum { ETD_ETD1 = 1, ETD_ETDRK2 = 2 } etd_scheme;
typedef enum {
  ETD_MODEL_FIXED = 0,        /* frozen membrane, FFT-diagonal split of Sec. 3 (Eq. (2.1))    */
  ETD_MODEL_COUPLED = 1,      /* phi-u system, Algorithm 1                                   */
  ETD_MODEL_FIXED_SQRTG = 2   /* frozen membrane, g^{1/2}-split scheme of Sec. 2.2 (Krylov)   */
} etd_model;
typedef enum { ETD_FP64 = 0, ETD_FP32_MIXED = 1 } etd_precision;

/* Problem statement (Sec. 1 model, Sec. 3.1 splittings, Sec. 3.3 schemes). */
typedef struct {
  int dim;                 /* 2 or 3                                                  */
  int n[3];                /* (Nx, Ny, Nz); Nz = 1 when dim = 2                        */
  double half_len[3];      /* (X, Y, Z): box [-X,X) x [-Y,Y) x [-Z,Z)                   */
  int scheme;              /* etd_scheme                                              */
  int model;               /* etd_model                                               */
  int precision;           /* etd_precision                                           */
  double tau;              /* time step (Sec. 2.2, Sec. 3.3)                          */
  double eps_phi, eps_u;   /* interface widths of phi and u (Eq. (1.1)-(1.2))          */
  double mu, lambda_surf, kappa, lambda_line, M_area, A0, alpha, u0;  /* Eq. (1.1)     */
  double gamma, M, ubar;   /* nonlocal strength, mass penalty, mean density (Eq. (1.2)) */
  double A1, A2, B1, B2;   /* stabilisers of Eq. (3.1) and Eq. (3.2)                  */
  double band_mask_hi;     /* narrow band = {|2 phi - 1| < band_mask_hi}, e.g. 0.99    */
  double recover_delta;    /* U = GU/G where G > recover_delta (Sec. 3.3), e.g. 1e-3    */
  double cg_rtol;          /* relative residual of the band CG                         */
  int cg_maxit;            /* iteration cap of the band CG                             */
  int linear_only;         /* 1: drop R1 and R2 (the exact linear flow; tests)          */
  double cg_rtol_pred;     /* ETDRK2 only: relative residual of the predictor-stage
                              band solves, whose result reaches u^{n+1} only through the
                              corrector's tau phi2 (R2(U~) - R2(U^n)) term; 0 = cg_rtol  */
  double krylov_tol;       /* ETD_MODEL_FIXED_SQRTG: a Krylov space grows (8 Lanczos steps
                              at a time, at most 128) until the estimated error of
                              tau phi_j(tau L_phi) x, |x| beta_m tau |e_m^T phi_{j+1}(tau T_m) e_1|,
                              is below krylov_tol times the result's norm; 0 = 1e-12 (FP64),
                              1e-6 (FP32-mixed); a space that reaches 128 steps without it
                              makes etd_step return ETD_ENOTCONV.  Ignored by the other
                              models.                                                       */
} etd_params;

/* Diagnostics of the current state (Eq. (2.16) energy and the bound of Sec. 2.2). */
typedef struct {
  double energy;           /* E_{phi,h}[U] of Eq. (2.16), band-restricted inverse      */
  double mass;             /* etd_step: fixed <g (f(U)-ubar),1>_h, coupled <g (U-ubar),1>_h;
                              etd_energy: <g (f(U)-ubar),1>_h (the energy term), both models */
  double max_bound;        /* max |2U-1| over {G > recover_delta}                       */
  double umin, umax;       /* min/max U over {G > recover_delta}                        */
  double volume;           /* <phi,1>_h                                                */
  long band_size;          /* number of band nodes                                     */
  int cg_iters_last;       /* iterations of the last band solve                        */
  double cg_resid_last;    /* relative residual reached by the last band solve         */
  int krylov_dim_last;     /* ETD_MODEL_FIXED_SQRTG: largest Krylov dimension of the call  */
} etd_diag;

/* Create a plan: validates `params`, allocates the workspace on the current device and
 * builds the phi-function tables in FP64 (phi_0, tau phi_1, tau phi_2 of tau l^phi and
 * tau l^u, Sec. 3.2-3.3).  `cuda_stream` is a cudaStream_t (NULL = legacy stream).
 * Returns ETD_EINVAL for unsupported sizes or non-positive tau/eps, ETD_ENOMEM when the
 * workspace does not fit.  On failure *out is NULL.
 * In 3D the FFT's first pass moves its four-step intermediate with tensor copies (TMA);
 * the environment variable ETD_PASSA_DIRECT=1, read here, selects direct loads and stores
 * instead (same arithmetic, bit-identical results; for verification).
 * Every device wait is bounded: a grid barrier of the band solve gives up after
 * ETD_WAIT_BUDGET clock cycles (default 4e9) and a tensor copy of the FFT after
 * ETD_WAIT_TRIES mbarrier polls (default 2^22); both environment variables are read here.
 * A wait that gives up makes the call that observes it return ETD_ETIMEOUT, the device
 * context stays usable (the waiting blocks return, a block whose copy is late waits for it
 * once more before it leaves). */
etd_status etd_plan(const etd_params *params, void *cuda_stream, etd_plan_t *out);

/* Advance `nsteps` steps in place (Algorithm 1; ETD1 or ETDRK2 per params.scheme).
 * coupled: phi and u are both read and overwritten.
 * fixed:   phi is read when non-NULL (it then fixes G = g(phi) and the band for this and
 *          later calls) and is never written; the first call must pass it.
 * When A0 was NaN at plan time, the first call fixes A0 = <phi,1>_h.
 * Asynchronous unless `last` is non-NULL: then the call synchronises the stream, checks
 * the state for non-finite values and the CG status, and fills *last (band size, CG
 * iterations, volume, mass; energy fields are left at 0 -- use etd_energy). */
etd_status etd_step(etd_plan_t plan, void *phi, void *u, int nsteps, etd_diag *last);

/* Diagnostics of (phi, u): energy of Eq. (2.16) (nonlocal term by a band solve of
 * (-Delta_{S,h}) w = g f(U) - mean), the energy's mass <g (f(U) - ubar), 1>_h (both models),
 * bound statistics, volume.  Plans of ETD_MODEL_FIXED_SQRTG report the same quantity (its
 * gradient term over every face of the grid), not the band system's own energy, whose gradient
 * term counts band faces only.  Synchronous. */
etd_status etd_energy(etd_plan_t plan, const void *phi, const void *u, etd_diag *out);

/* Release the plan and its workspace.  etd_free(NULL) returns ETD_OK. */
etd_status etd_free(etd_plan_t plan);

/* Message of the last error raised on the calling thread ("" if none). */
const char *etd_last_error(void);

/* ---- Operator entry points: single rows of the step, for verification -------------- */

/* Forward FFT (Sec. 3.2): real field -> half spectrum, unnormalised,
 * out[(kz*Ny + ky)*(Nx/2+1) + kx] (complex as interleaved re,im of the element type). */
etd_status etd_fft_forward(etd_plan_t plan, const void *field, void *half_spectrum);

/* Inverse FFT: half spectrum (layout above) -> real field, with the 1/N factor.  The
 * imaginary parts of self-conjugate modes are ignored (real-to-complex convention). */
etd_status etd_fft_inverse(etd_plan_t plan, const void *half_spectrum, void *field);

/* Narrow band of phi (Sec. 3.2): writes the ascending flat indices of the band nodes
 * {|2 phi - 1| < band_mask_hi} to idx (device int32, capacity N) and the count to
 * *count (host).  Synchronous. */
etd_status etd_band(etd_plan_t plan, const void *phi, int *idx, long *count);

/* Band-restricted nonlocal solve: w = (-Delta_{S,h})^{-1}(f - mean) on the band of phi
 * with zero-flux band edges, g = g(phi) (Eq. (2.3)); f and w are full fields, w = 0
 * off the band.  The band operator is singular on each connected band component (6-neighbour,
 * periodic), so the mean of f is removed and w is returned with zero mean on every component
 * separately (the mean removal of Sec. 2.1, per component; up to 4096 components, more
 * return ETD_EINVAL).  Warm start from the incoming w.  Synchronous; reports iterations and
 * relative residual. */
etd_status etd_nonlocal(etd_plan_t plan, const void *phi, const void *f, void *w,
                        int *iters, double *resid);

/* Nonlinear remainders as real fields:
 *   which = 1: R1(phi, u) of the force balance (Sec. 3.1), phi_old unused;
 *   which = 2: R2(phi, u) of the coupled OK equation with advection velocity from
 *              (phi - phi_old)/tau (coupled plans), zero off the band;
 *   which = 3: R2 of the fixed-membrane model with g = g(phi) (fixed plans).
 * Synchronous. */
etd_status etd_remainder(etd_plan_t plan, int which, const void *phi, const void *phi_old,
                         const void *u, void *out);

/* ---- Batched runs (many independent simulations, fixed model or coupled) -------------- */

typedef struct etd_batch_s *etd_batch_t;

/* Create a batch of `nruns` independent runs, params[i] describing run i (grids, precision,
 * model, scheme, tau and coefficients may all differ).  Each run gets its own plan (workspace
 * as etd_plan) and its own CUDA stream, forked from and joined back into `cuda_stream`.
 * autotune_tiles = 1: for every distinct grid and precision, time a forward + inverse
 * transform pair for each candidate tiling (pass-A z-planes per block, pass-B pencil blocks
 * per block, tensor-copy staging of pass A on or off) and give the runs of that grid the
 * fastest; 0: default tiles.  Tiling never changes the results (the same arithmetic per
 * element).  Runs of model ETD_MODEL_FIXED_SQRTG are rejected (ETD_EINVAL): their Krylov
 * spaces are sized on the host between launches, which a recorded graph cannot do.
 * Synchronous; ETD_EINVAL names the first invalid run. */
etd_status etd_plan_batch(const etd_params *params, int nruns, void *cuda_stream, int autotune_tiles,
                          etd_batch_t *out);

/* Advance every run `nsteps` steps in place (as etd_step on each run).  phi[i], u[i] are run
 * i's device fields; phi is read on the first call (it fixes the membrane of fixed-model runs,
 * which may pass NULL afterwards) and on every call of coupled runs.  The first two steps of a
 * batch run eagerly; after that, blocks of 6 steps of all runs are recorded once into a CUDA
 * graph (the runs as parallel branches) and replayed, the rest eagerly.  A graph is tied to
 * the field pointers it was recorded with: other pointers re-record it.  If the graph cannot
 * be recorded (etd_batch_info reports graph = 0), every step runs eagerly.  Asynchronous on
 * the batch stream; errors inside the steps surface in etd_batch_check. */
etd_status etd_batch_step(etd_batch_t batch, void *const *phi, void *const *u, int nsteps);

/* Synchronise and check every run (non-finite state, band-solve convergence, device waits);
 * fills diag[i] (nullable) as etd_step's `last`.  Returns the first run's error. */
etd_status etd_batch_check(etd_batch_t batch, void *const *phi, void *const *u, etd_diag *diag);

/* Tiles run `run` uses (pass-A z-planes, pass-B pencil blocks, tensor-copy staging 1/0) and the
 * batch's graph state (1 replaying, 0 eager, -1 not yet recorded).  Any pointer may be NULL.
 * When the graph could not be recorded, etd_last_error() then gives the reason. */
etd_status etd_batch_info(etd_batch_t batch, int run, int *zb, int *kb, int *tma, int *graph);

/* Release the batch (synchronises its stream).  etd_batch_free(NULL) returns ETD_OK. */
etd_status etd_batch_free(etd_batch_t batch);

/* ---- Per-kernel timing (measurement support; no counterpart in the paper) ----------- */

/* Kernel classes reported by etd_timing_read. */
typedef enum {
  ETD_K_FFT_A_FWD = 0,   /* pass A forward: x real-to-complex + inner y DFT             */
  ETD_K_FFT_A_INV = 1,   /* pass A inverse (+ fused pointwise epilogue)                  */
  ETD_K_FFT_B = 2,       /* pass B: outer y + z DFT, fused spectral ETD update, inverse  */
  ETD_K_CG = 3,          /* persistent band CG (one launch per solve)                    */
  ETD_K_POINTWISE = 4,   /* R1, R2, Delta_S u and other full-grid pointwise kernels      */
  ETD_K_BAND = 5,        /* band compaction and CG set-up                                */
  ETD_K_REDUCE = 6,      /* FP64 reductions                                              */
  ETD_K_KRYLOV = 7,      /* Lanczos steps, Krylov norms and combinations (Sec. 2.2 scheme) */
  ETD_K_NKINDS = 8
} etd_kernel_kind;

/* enable = 1: reset the counters and bracket every later launch with CUDA events on the
 * plan's stream; enable = 0: stop recording (counters are kept). */
etd_status etd_timing(etd_plan_t plan, int enable);

/* Totals since the last etd_timing(plan, 1) for one kernel class: summed event time
 * (ms), launch count, and the algorithmic bytes of those launches (each real field
 * element and each half-spectrum complex element read or written once, at the element
 * size of the plan's precision).  Synchronises the stream. */
etd_status etd_timing_read(etd_plan_t plan, int kind, double *total_ms, long *launches,
                           double *algo_bytes);

/* ---- Host half of the Krylov evaluation (ETD_MODEL_FIXED_SQRTG) ------------------- */

/* For the symmetric tridiagonal Lanczos matrix T_m (diagonal alpha[0..m-1], off-diagonal
 * beta[0..m-2]; host arrays), writes y = phi_j(tau T_m) e_1 (m host doubles) and *tail =
 * |e_m^T phi_{j+1}(tau T_m) e_1|, with phi_0(z) = e^{-z}, phi_1(z) = (1 - e^{-z})/z,
 * phi_2(z) = (e^{-z} - 1 + z)/z^2, phi_3(z) = (1/2 - phi_2(z))/z (Sec. 2.2's convention).
 * The plan of the Sec. 2.2 scheme takes tau phi_j(tau L) x ~ tau |x| V_m y and stops growing
 * the Krylov space when |x| beta_m tau *tail is small against the result.  T_m by cyclic Jacobi
 * rotations; 1 <= m <= 128, j in {0, 1, 2}, tau >= 0, T_m positive semi-definite (the phi_j
 * series and closed forms are evaluated at tau lambda >= 0).  Host computation only: needs no GPU. */
etd_status etd_krylov_coeffs(int m, const double *alpha, const double *beta, double tau, int j, double *y,
                             double *tail);

/* ---- Forward FFT that allocates nothing ------------------------------------------- */

/* The paper has no counterpart to this entry point; it serves callers that may not
 * allocate device memory -- a host application that owns all device memory through its
 * own pool or a fixed footprint, or a latency-critical path on which cudaMalloc/cudaFree
 * could synchronise the device.  Such callers cannot create a plan (etd_plan allocates).
 *
 * Same transform and output layout as etd_fft_forward: real field (dim = 2: Ny x Nx,
 * dim = 3: Nz x Ny x Nx, x fastest) -> unnormalised half spectrum
 * out[(kz*Ny + ky)*(Nx/2+1) + kx]; double/complex double for ETD_FP64, float/complex
 * float for ETD_FP32_MIXED.  `field` and `half_spectrum` are caller-owned device
 * pointers; the work is enqueued on `cuda_stream` (a cudaStream_t, NULL = legacy) and
 * the call returns after the launches.
 *
 * Scratch: a file-scope device array of ETD_STATIC_SCRATCH_BYTES = 8 MiB, held by every
 * GPU that loads the library until the process exits.  The intermediate spectrum
 * ((Nx/2+1)*Ny*Nz complex elements) plus the three twiddle tables must fit, each rounded
 * up to 256 bytes; larger grids return ETD_EINVAL with the sizes in etd_last_error().
 * Every call on a device shares that array and overwrites it (nothing in it needs to
 * start at zero: the intermediate and the twiddles are fully rewritten by each call), so
 * calls whose work overlaps on the GPU -- for example on two streams -- race; order them.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * Sizes: Nx, Ny powers of two in [8, 256]; Nz = 1 (dim 2) or a power of two in [8, 256]. */
etd_status etd_fft_forward_noalloc(int dim, const int *n, int precision, const void *field,
                                   void *half_spectrum, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ETD_H */

/*
 * atkm.h -- C interface of the GB300 PCG-ATKM ground-state solver.
 *
 * Computes ground states of the 3D rotating dipolar Gross-Pitaevskii energy
 * (Tang, Wang, Zhang & Zhang, "An efficient and accurate numerical method for
 * computing the ground states of three-dimensional rotating dipolar
 * Bose-Einstein condensates under strongly anisotropic trap"):
 *   - the dipolar potential by the anisotropic truncated kernel method (ATKM,
 *     §2.2, Eqs. (iden_b2)-(FUk) with the Coulomb reformulation (DDI2Cou3D)),
 *   - the Fourier-spectral Hamiltonian (§2.1 Eq. (Laplacian), §2.3),
 *   - the preconditioner, the Riemannian PCG step and its step control
 *     (§2.3, Algorithm 1).
 *
 * Conventions shared by every call
 *   - Box prod_a [-L_a, L_a]; grid N_a points per axis, N_a even, each N_a a
 *     product of 2, 3 and 5 only, 2 <= N_a <= 1024; h_a = 2 L_a / N_a; grid
 *     point j of axis a sits at -L_a + j h_a (§2.1).
 *   - Arrays are row-major [N_z][N_y][N_x] (x fastest).  Complex arrays are
 *     interleaved (re, im) pairs, i.e. 2*N_x*N_y*N_z doubles (or floats).
 *   - Every array argument is a DEVICE pointer owned by the caller, sized for
 *     the plan's grid, 16-byte aligned (any cudaMalloc / torch allocation is).
 *     Host pointers are only the small parameter/result structs.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous unless the call says otherwise.
 *   - Every call returns an atkm_status; none raises, traps or sets errno.
 *     After a failure atkm_last_error_string(plan) describes it.
 *   - A plan may be used by one host thread at a time; calls on one plan must
 *     use one stream (the plan's workspace is shared between calls).
 */
#ifndef ATKM_H_
#define ATKM_H_

#ifdef __cplusplus
extern "C" {
#endif

typedef enum atkm_status {
  ATKM_OK = 0,
  ATKM_ERR_ARG = 1,              /* bad pointer, size or parameter value         */
  ATKM_ERR_UNSUPPORTED_SIZE = 2, /* N_a odd, not {2,3,5}-smooth, or too large     */
  ATKM_ERR_OOM = 3,              /* device allocation failed                      */
  ATKM_ERR_CUDA = 4,             /* a CUDA runtime call or kernel launch failed   */
  ATKM_NOT_CONVERGED = 5,        /* PCG reached max_iter before the stop rule     */
  ATKM_STAGNATED = 6,            /* three consecutive exhausted halving loops     */
  ATKM_ERR_NAN = 7,              /* a NaN/Inf appeared in the PCG scalars         */
  ATKM_ERR_TIMEOUT = 8           /* the solve reached opts.time_limit_s           */
} atkm_status;

typedef struct atkm_plan atkm_plan;

/* Plan flags (bit set). */
#define ATKM_PLAN_F64 0u   /* FP64 workspaces (always present)                  */
#define ATKM_PLAN_F32 1u   /* also allocate complex64 workspaces for the _f32 calls */
#define ATKM_PLAN_DF32 2u  /* also keep a double-word copy of U0 for the _df32 calls  */
#define ATKM_PLAN_GENERIC_FFT 4u  /* lengths that are not powers of two run on the generic
                                     shared-memory FFT engine also where the mixed-radix
                                     register engine covers them (3 * 2^a and 5 * 2^a,
                                     20 <= L <= 384); for comparisons, same results to
                                     rounding                                            */
#define ATKM_PLAN_AUTOTUNE 8u     /* run atkm_plan_autotune at creation                   */

/*
 * atkm_plan_create -- grid, box, dipole axis; precomputes the truncated-kernel
 * multiplier (the set-up step of Algorithm 1; §2.2 remark: once per domain
 * and mesh).
 *   N[3]  grid sizes (N_x, N_y, N_z), see conventions.
 *   L[3]  box half-lengths, each > 0 and finite.
 *   n[3]  dipole orientation; | |n| - 1 | must be <= 1e-12 (Eq. (DDI-3D)).
 *   flags ATKM_PLAN_F64, or any of ATKM_PLAN_F32, ATKM_PLAN_DF32,
 *         ATKM_PLAN_GENERIC_FFT and ATKM_PLAN_AUTOTUNE.
 * Builds, in FP64 on the device, U0(nu) = int_{D_2L} e^{-i nu.y}/(4 pi|y|) dy on
 * the nonnegative frequency octant of the twofold-padded grid (Eq. (FUk)),
 * and from it the dipolar multiplier K = -1 + 3 (n.nu)^2 U0, symmetrised on the
 * padded Nyquist planes, on the half spectrum kept by the real-data transform
 * (FP64, and a double-word copy with ATKM_PLAN_DF32; FP32 passes form it from
 * an FP32 copy of U0).  Also holds the twiddle tables, per-axis frequency and
 * coordinate tables and the workspaces (atkm_plan_device_bytes gives the
 * total: about 0.5 GB for an FP64 plan at 256 x 256 x 64, more once a solve
 * has allocated its vectors).  Synchronises `stream` before
 * returning.  On success *out owns all device memory of the plan; on failure
 * *out is NULL and nothing is leaked.
 */
int atkm_plan_create(atkm_plan** out, const int N[3], const double L[3], const double n[3],
                     unsigned flags, void* stream);

/* Frees the plan and its device memory (synchronises the device). NULL-safe. */
void atkm_plan_destroy(atkm_plan* plan);

/* Message for the last failing call on `plan` (or a global message when plan is NULL). */
const char* atkm_last_error_string(const atkm_plan* plan);

/* Bytes of device memory held by the plan. */
unsigned long long atkm_plan_device_bytes(const atkm_plan* plan);

/*
 * Per-kernel timing (opt-in).  While profiling is on, every pass kernel of the
 * spectral operators is bracketed by CUDA events recorded on the stream it is
 * launched on, and tagged with the algorithmic HBM bytes and flops of that
 * launch (bytes: each input read once and each output written once; flops:
 * 5 n log2 n per complex FFT of length n).  Library extension for
 * measurement; the paper has no counterpart.
 */
typedef struct atkm_kernel_stat {
  char name[32];            /* pass name, e.g. "atkm_z_f32"                 */
  int launches;             /* launches recorded since profiling was enabled */
  int pad_;
  double ms_total;          /* summed CUDA-event time of those launches      */
  double bytes_total;       /* summed algorithmic bytes                      */
  double flops_total;       /* summed algorithmic flops                      */
} atkm_kernel_stat;

/* Number of CUDA kernels this library has launched in this process (all
 * plans, all calls); the difference around a region counts its launches. */
unsigned long long atkm_launch_count(void);

/*
 * atkm_measure_fp64_fma -- peak binary64 FMA rate of the current device, the
 * denominator of the roofline of the binary64 FFT passes (bound by that
 * pipe on this GPU).  Launches blocks_per_sm x (SM count) CTAs of 256
 * threads, each thread running 8 independent FMA chains of `iters` steps;
 * times `repeats` launches (after one warm-up) with CUDA events on `stream`
 * and writes the best rate in GFLOP/s (2 flops per FMA) to *gflops (host).
 * Allocates and frees a small output buffer; synchronises the stream.
 * Measurement support; the paper has no counterpart.
 */
int atkm_measure_fp64_fma(int blocks_per_sm, int iters, int repeats, double* gflops, void* stream);

/*
 * atkm_plan_autotune -- FFT-tile autotuner: for every line length of the
 * plan's passes that is not a power of two, per arithmetic the plan carries
 * (binary64; FP32 with ATKM_PLAN_F32; double-word with ATKM_PLAN_DF32) and per
 * layout (line-major x pass, strided y / z pass), times the candidates -- the
 * mixed-radix register engine (FP32: lengths 3 * 2^a and 5 * 2^a <= 384;
 * binary64: 3 * 2^a <= 384; not double-word; not with ATKM_PLAN_GENERIC_FFT)
 * and the generic shared-memory engine
 * at its default tile width, 1/2 and 1/4 of it -- on the plan's own ATKM of
 * |psi|^2, H psi and P r (CUDA events on `stream`, best of 3 after a warm-up)
 * and keeps the fastest; every later pass of that length and layout uses it.
 * Power-of-two lengths keep the power-of-two register engine.  Results change
 * only by rounding.  Allocates and frees scratch of about 40 bytes a grid
 * point; synchronises `stream`.  Must run before the plan's first PCG solve
 * (ATKM_ERR_ARG afterwards).  Selection support; the paper has no
 * counterpart.
 */
int atkm_plan_autotune(atkm_plan* plan, void* stream);

typedef struct atkm_tune_info {
  int precision;   /* 0 binary64, 1 FP32, 2 double-word                        */
  int length;      /* line length L                                            */
  int line_major;  /* 1: the x pass (contiguous lines), 0: a strided y / z pass */
  int engine;      /* 1: mixed-radix register engine, 2: generic engine        */
  int tile_shift;  /* generic engine: tile width = default >> tile_shift       */
  int pad_;
  double ms_default;  /* the timed operators under the fixed rule, ms          */
  double ms_best;     /* under the chosen candidate, ms                        */
} atkm_tune_info;

/* Copies up to `cap` of the plan's autotuned choices to out (host); returns
 * how many the plan holds (0 when not tuned), or -ATKM_ERR_ARG. */
int atkm_plan_tuning(const atkm_plan* plan, atkm_tune_info* out, int cap);

/* on != 0 clears the record and starts recording; on == 0 stops. */
int atkm_plan_set_profiling(atkm_plan* plan, int on);

/* Synchronises the device, aggregates the record per pass name into
 * out[0..capacity) and writes the number of distinct passes to *count. */
int atkm_plan_kernel_stats(atkm_plan* plan, atkm_kernel_stat* out, int capacity, int* count);

/*
 * atkm_plan_copy_U0 -- copies the FP64 octant table U0[|k_z|][|k_y|][|k_x|],
 * |k_a| = 0..N_a, (N_z+1)(N_y+1)(N_x+1) doubles, to the device buffer `dst`
 * (ATKM precompute, Eq. (FUk)).  Stream-ordered.
 */
int atkm_plan_copy_U0(const atkm_plan* plan, double* dst, void* stream);

/*
 * atkm_plan_copy_multiplier -- writes the full padded dipolar multiplier
 * K(k) = -1 + 3 (n.nu_k)^2 U0(nu_k) in FFT order, shape [2N_z][2N_y][2N_x]
 * doubles, to `dst` (Eq. (DDI2Cou3D) in Fourier space).  Stream-ordered.
 */
int atkm_plan_copy_multiplier(const atkm_plan* plan, double* dst, void* stream);

/*
 * dipolar_potential -- Phi = U_dip * rho by ATKM (§2.2: twofold zero padding,
 * FFT (Eq. (fouriercoeff)), multiply, inverse FFT (Eq. (U_TrunFour)), real
 * part, crop).  rho, phi: N doubles each (phi may not alias rho).  Phi does
 * not include the factor lambda.
 */
int dipolar_potential(atkm_plan* plan, const double* rho, double* phi, void* stream);

/* Same with rho = |psi|^2 formed on the fly; psi: N complex (2N doubles). */
int dipolar_potential_from_psi(atkm_plan* plan, const double* psi, double* phi, void* stream);

/* Same with rho = Re(conj(a) b) formed on the fly (the density variation
 * of Eq. (Energy_Expend)); a, b: N complex each. */
int dipolar_potential_from_pair(atkm_plan* plan, const double* a, const double* b, double* phi,
                                void* stream);

/* FP32-arithmetic variant of dipolar_potential_from_psi (plan needs
 * ATKM_PLAN_F32): same FP64 interface, but the five FFT passes run in FP32
 * on complex64 workspaces (half the bytes); the multiplier is formed in FP64
 * and rounded per use.  Relative error ~1e-6 of max|Phi|. */
int dipolar_potential_from_psi_f32(atkm_plan* plan, const double* psi, double* phi, void* stream);

/* Double-word variant of dipolar_potential_from_psi (plan needs
 * ATKM_PLAN_DF32): same FP64 interface and the same padded convolution
 * (§2.2), with every FFT pass in double-FP32 arithmetic -- each value is an
 * unevaluated sum of two binary32 numbers, about 48 significant bits --
 * computed on the FP32 pipe, which runs about 57 times the binary64 rate on
 * this GPU.  Uses the FP64 workspaces.  Relative error about 1e-14 of
 * ||Phi|| (the FP64 call reaches about 1e-15). */
int dipolar_potential_from_psi_df32(atkm_plan* plan, const double* psi, double* phi, void* stream);

/* Physical parameters of the energy (Eqs. (DipGPE0), (Vpoten)). */
typedef struct atkm_params {
  double gamma[3]; /* trap frequencies gamma_x, gamma_y, gamma_z */
  double beta;     /* contact interaction strength */
  double lambda;   /* dipolar interaction strength */
  double Omega;    /* rotation frequency */
} atkm_params;

/*
 * apply_H -- Hf = -1/2 [[Delta]] f + V f + beta |phi|^2 f + lambda Phi f
 * - Omega [[L_z]] f (§2.3, the operator H_phi of the energy gradient, with
 * [[.]] the Fourier-spectral operators of Eq. (Laplacian)).
 *   f    N complex: the vector H_phi acts on (f == phi gives H_phi phi).
 *   phi  N complex: the state whose density enters beta |phi|^2.
 *   Phi  N doubles: the dipolar potential of |phi|^2 (from dipolar_potential).
 *   Hf   N complex output; must not alias f, phi or Phi.
 */
int apply_H(atkm_plan* plan, const atkm_params* prm, const double* f, const double* phi,
            const double* Phi, double* Hf, void* stream);

/* Energy terms of the discrete functional (§2.3) and the virial residual
 * I = 2E_kin - 2E_pot + 3E_int + 3E_dip (Eq. (vir_iden)). */
typedef struct atkm_energy {
  double E, E_kin, E_pot, E_int, E_dip, E_rot, mu, virial, norm2;
} atkm_energy;

/*
 * atkm_energy_parts -- evaluates the energy terms and mu = <H_phi phi, phi>
 * for (phi, Phi).  Synchronises `stream` and writes *out (host struct).
 */
int atkm_energy_parts(atkm_plan* plan, const atkm_params* prm, const double* phi,
                      const double* Phi, atkm_energy* out, void* stream);

/*
 * apply_preconditioner -- Pr = P_V^{1/2} P_Delta P_V^{1/2} r (§2.3), with
 * P_Delta = (alpha - [[Delta]]/2)^{-1} and
 * P_V = (alpha + V + beta |phi|^2 + |lambda| (1 + sign Phi) Phi / 2)^{-1}.
 *   alpha  the shift (> 0); pcg_ground_state uses
 *          <-1/2[[Delta]]phi + V phi + beta|phi|^2 phi, phi> + |lambda <Phi phi, phi>|.
 *   r, phi N complex; Phi N doubles; Pr N complex output (no aliasing).
 */
int apply_preconditioner(atkm_plan* plan, const atkm_params* prm, double alpha, const double* r,
                         const double* phi, const double* Phi, double* Pr, void* stream);

/* Precision modes of the PCG driver. */
#define ATKM_PRECISION_F64 0      /* every step in FP64                          */
#define ATKM_PRECISION_F32_F64 1  /* complex64 FFT/ATKM/H/P until switch_tol, two exhausted
                                     halving loops, or f32_window iterations without
                                     the best FP32 residual falling by the factor
                                     f32_gain; then FP64                                */
#define ATKM_PRECISION_F32_SPLIT 2 /* as ATKM_PRECISION_F32_F64, and after the hand-over the
                                     operators that only shape the search direction and
                                     the step-size model (P r, H p and the ATKM of
                                     Re(conj(phi) p)) stay complex64; H phi (residual,
                                     mu), the trial-energy ATKM, every reduction, the
                                     retraction and the stop test are FP64             */
#define ATKM_PRECISION_DF32_SPLIT 3 /* as ATKM_PRECISION_F32_SPLIT, with H phi and the
                                     trial-energy ATKM of the polish in double-FP32
                                     arithmetic (about 48 bits, on the FP32 pipe;
                                     plan needs ATKM_PLAN_F32 | ATKM_PLAN_DF32); the
                                     reductions and the retraction stay FP64, and the
                                     stop test's residual is formed from the double-
                                     word H phi (error about 1e-14 relative)           */

typedef struct atkm_pcg_opts {
  double tol_residual;  /* stop when ||H phi - mu phi|| <= tol_residual (e.g. 1e-8)    */
  double tol_linf;      /* if > 0, also stop when ||phi_{n+1}-phi_n||_inf <= tol_linf  */
  int max_iter;         /* iteration cap (ATKM_NOT_CONVERGED when reached)            */
  int max_halvings;     /* halvings of t per iteration before taking the lowest trial */
  int precision_mode;   /* ATKM_PRECISION_F64 or ATKM_PRECISION_F32_F64               */
  double switch_tol;    /* residual at which the F32 phase hands over (e.g. 1e-5); if
                           < 0, automatic: the larger of |switch_tol| and 4x the
                           FP32 noise of the residual, measured once at phi_0 as
                           ||H phi_0 in FP32 - H phi_0 in FP64|| (each with its
                           own ATKM; about one FP64 iteration of extra work), and
                           the stagnation window's default becomes 2000         */
  int log_capacity;     /* entries available in `log` (0 = no log)                    */
  int resume;           /* != 0: continue the solve this plan ran last (psi_inout is
                           then output only); the iteration count, direction memory,
                           precision phase and energy carry over; max_iter counts
                           the iterations of this call                              */
  int no_graphs;        /* != 0: launch every kernel directly instead of replaying the
                           captured CUDA graph of an iteration (same results)       */
  double time_limit_s;  /* if > 0: stop with ATKM_ERR_TIMEOUT once this many seconds
                           of wall-clock time have passed since the call began,
                           checked at the top of every iteration (on the device,
                           from its global timer, in the device-driven loop); the
                           state reached is returned and can be resumed          */
  int f32_window;       /* precision forms: FP32-phase iterations without halving the
                           best FP32 residual before the hand-over (0: 50)       */
  double f32_gain;      /* precision forms: the factor by which the best FP32
                           residual must fall within f32_window iterations for
                           the FP32 phase to go on (0: 0.5, "halving"; 0.9 lets
                           slow but steady progress continue)                   */
  int mg_f64_levels;    /* pcg_ground_state_mg with a precision form: the number of
                           coarsest levels solved in FP64 (0: none); ignored by the
                           single-level calls                                   */
} atkm_pcg_opts;

/* One record per iteration n (values at phi_n; step fields describe n -> n+1). */
typedef struct atkm_iter_log {
  int n, halvings, reset_to_sd, accepted, f32_phase, pad_;
  double E, mu, residual, linf_step, alpha, beta_cg, d1, curvature, t0, t;
} atkm_iter_log;

typedef struct atkm_result {
  double E, mu, E_kin, E_pot, E_int, E_dip, E_rot, virial;
  double residual, linf_step;
  int iters, halvings, f32_iters, status;
  atkm_iter_log* log;   /* host array of opts.log_capacity entries (may be NULL) */
  int log_count;        /* entries written                                       */
  int device_loop;      /* 1 when the device-driven graph ran the iterations, 0 when
                           the host took the decisions between them              */
  double switch_residual; /* precision forms: the residual at which the FP32 phase
                           hands over (see atkm_pcg_opts.switch_tol); 0 in FP64  */
} atkm_result;

/*
 * pcg_ground_state -- Algorithm 1 (PCG-ATKM) with the step control of §2.3
 * (i) PSD fallback when <H phi, p> >= 0, (ii) quadratic-model step
 * (Eq. (opt_step)) or t = 0.3, (iii) halving until the energy decreases.
 *   psi_inout  N complex: initial guess in, final state out (normalised on entry).
 *   out        host struct; out->log (host) receives per-iteration records.
 * Allocates the PCG vectors, a plan-owned stream and graph state on first use
 * (kept by the plan).  Every decision runs in control kernels on the device:
 * the solve (the FP32 phase, the hand-over and the polish of the precision
 * forms included) is one CUDA graph whose conditional nodes loop over the
 * iterations and the halvings, built once per plan and form and launched once
 * on the plan's stream, which is ordered after `stream`'s prior work on entry
 * and before its later work on return; the host synchronises once at the
 * start (the check of psi_0) and once at the end.  Every graph loop is bounded
 * by a count derived from max_iter and max_halvings.  While per-pass profiling
 * is on, or with no_graphs, the host takes the same decisions between
 * iterations instead (one synchronisation per iteration and per halving);
 * the results are identical.
 * Returns ATKM_OK, ATKM_NOT_CONVERGED, ATKM_STAGNATED, ATKM_ERR_NAN,
 * ATKM_ERR_TIMEOUT or an argument/CUDA error; out->status holds the same value.
 */
int pcg_ground_state(atkm_plan* plan, const atkm_params* prm, const atkm_pcg_opts* opts,
                     double* psi_inout, atkm_result* out, void* stream);

/*
 * pcg_ground_state_batched -- `count` independent solves of Algorithm 1 (an
 * Omega or anisotropy sweep) on one GPU.  Grids may differ: instance i uses
 * plans[i] (each instance needs its own plan), prm[i], psi[i] (device, in/out)
 * and out[i] (its log pointer is honoured); all share `opts`.  The solves of
 * all instances are built into one CUDA graph (one independent chain of
 * conditional loops per instance) and launched once: the instances run
 * concurrently on the GPU and each ends on its own stop rule, with no host
 * work until all have ended.  (With profiling on or graphs off, the host
 * instead polls the instances' streams and relaunches each as soon as its
 * last phase has finished.)  Results are bitwise identical to
 * pcg_ground_state on each instance alone.  Returns
 * ATKM_OK if every instance converged, else the first non-OK status
 * (ATKM_ERR_CUDA takes precedence); per-instance statuses are in out[i].status.
 */
int pcg_ground_state_batched(int count, atkm_plan* const* plans, const atkm_params* prm,
                             const atkm_pcg_opts* opts, double* const* psi, atkm_result* out,
                             void* stream);

/*
 * atkm_spectral_upsample -- psi_f = the Fourier interpolant of psi_c
 * (Eq. (Fourphi): sum over k in Lambda_Nc of coef_k W_k) evaluated on the fine
 * plan's grid; the interpolation step of the cascadic multigrid driver
 * (Algorithm 2, Step 2) and of the learned guess.  Both plans must have the
 * same box; the fine grid may not be coarser on any axis.  psi_c: coarse N_c
 * complex (device), psi_f: fine N_f complex (device, output; must not alias).
 * Uses the coarse plan's T1 workspace.  Stream-ordered.
 */
int atkm_spectral_upsample(atkm_plan* coarse, atkm_plan* fine, const double* psi_c, double* psi_f,
                           void* stream);

/*
 * pcg_ground_state_mg -- the cascadic multigrid driver PCG-ATKM-MG
 * (Algorithm 2): for level i = 0 .. levels-1 (coarse to fine), compute the
 * ground state on plans[i] by Algorithm 1 (pcg_ground_state with `opts`;
 * with a precision form, the opts.mg_f64_levels coarsest levels in FP64)
 * starting from psi[i], then (Step 2) set psi[i+1] to its Fourier interpolant
 * on the next grid (atkm_spectral_upsample).  The plans share the box and the
 * dipole axis; grids must not get coarser.  The paper's setting is three
 * levels with N_a/4, N_a/2, N_a points per axis.
 *   psi     `levels` device buffers, psi[i] of plans[i]'s size; psi[0] holds
 *           the initial guess; every psi[i] ends as level i's ground state.
 *   out     `levels` host result structs (log pointers honoured).
 * Returns the finest level's status (ATKM_OK when it converged); a level
 * ending in NOT_CONVERGED or STAGNATED still seeds the next one; an error
 * stops the cascade.  out[i].status holds each level's status.
 */
int pcg_ground_state_mg(int levels, atkm_plan* const* plans, const atkm_params* prm,
                        const atkm_pcg_opts* opts, double* const* psi, atkm_result* out, void* stream);

/*
 * Learned initial guess.  The paper chooses psi_0 among fixed formulas (§3,
 * ten initial guesses) or interpolates a coarse solution (Algorithm 2); this
 * network maps the 8 workload features (Omega, gamma_x, gamma_y, ln gamma_z,
 * ln beta, lambda/beta, sin theta, cos theta of n = (sin theta, 0, cos theta))
 * to psi_0 on a 16x64x64 (z, y, x) grid: MLP 8 -> 256 (ReLU) -> 8192 = latent
 * 4x8x8 voxels x 32 channels -> transposed 3D convolutions with kernel =
 * stride: 32 -> 16 ch (stride 2, ReLU), 16 -> 8 (stride 2, ReLU), 8 -> 2
 * (stride (1,2,2); Re, Im).  Every layer runs as a GEMM with BF16 operands
 * and FP32 accumulation: the MLP layers and their gradients on the tcgen05
 * tensor cores (accumulator in tensor memory; engine selectable with
 * atkm_guess_net_set_gemm_engine), the transposed convolutions, whose
 * products need at most 4096 weights a row, on the CUDA cores (they are
 * bound by memory traffic, not multiply-adds); parameters are FP32 (master
 * copy) and trained with Adam on the loss 1 - |<u,t>|^2/(|u|^2 |t|^2) (mean
 * over the batch), which ignores the global phase and scale of the targets.
 *   feats    device, batch x 8 floats.
 *   psi      device, batch x 16 x 64 x 64 complex doubles (forward output).
 *   targets  device, batch x 16 x 64 x 64 complex doubles.
 *   grad_out device, atkm_guess_net_num_params() floats (may be NULL).
 *   loss     device, 1 float (batch mean).
 * Parameters are one flat float vector (get/set copy it device to device).
 */
typedef struct atkm_guess_net atkm_guess_net;
unsigned long long atkm_guess_net_num_params(void);
int atkm_guess_net_create(atkm_guess_net** out, unsigned long long seed, void* stream);
void atkm_guess_net_destroy(atkm_guess_net* net);
int atkm_guess_net_get_params(const atkm_guess_net* net, float* dst, void* stream);
int atkm_guess_net_set_params(atkm_guess_net* net, const float* src, void* stream);
int atkm_guess_net_forward(atkm_guess_net* net, int batch, const float* feats, double* psi, void* stream);
int atkm_guess_net_grad(atkm_guess_net* net, int batch, const float* feats, const double* targets,
                        float* grad_out, float* loss, void* stream);
int atkm_guess_net_train_step(atkm_guess_net* net, int batch, const float* feats, const double* targets,
                              float lr, float* loss, void* stream);
/* Engine of the network's dense GEMMs: ATKM_GEMM_TCGEN05 (default; tcgen05.mma
 * with the accumulator in tensor memory, 128-row tiles) or ATKM_GEMM_MMA_SYNC
 * (warp-level mma.sync m16n8k16, kept for comparison).  Both round the
 * operands to BF16 and sum in FP32.  ATKM_GEMM_TCGEN05_WAIT_TEST checks the
 * tensor-core path's error reporting: every such GEMM first waits, at most
 * 1000 polls, on a barrier that nothing completes, gives up before issuing
 * any MMA, and leaves its output unwritten; atkm_guess_net_check then
 * returns ATKM_ERR_TIMEOUT and the context stays usable.  ATKM_ERR_ARG for
 * another value.  Implementation choice; the paper has no counterpart. */
#define ATKM_GEMM_TCGEN05 0
#define ATKM_GEMM_MMA_SYNC 1
#define ATKM_GEMM_TCGEN05_WAIT_TEST 2
int atkm_guess_net_set_gemm_engine(atkm_guess_net* net, int engine);
/* Synchronises `stream` and reports whether any tcgen05 GEMM of this network
 * gave up a bounded wait for its MMAs since the last check (ATKM_ERR_TIMEOUT;
 * that GEMM's output is then not written), else ATKM_OK.  Clears the flag. */
int atkm_guess_net_check(atkm_guess_net* net, void* stream);
/* One training step as atkm_guess_net_train_step, with every GEMM bracketed by
 * CUDA events on `stream`: *gemm_ms = their summed time, *step_ms = the whole
 * step, *gemm_calls = the GEMMs timed, each_ms[i] (if not NULL, up to
 * each_cap entries) the time of GEMM i in launch order: the five forward
 * layers, then per layer from the last the weight gradient and (but for the
 * first layer) the input gradient (host outputs; synchronises `stream`).
 * Measurement support; the paper has no counterpart. */
int atkm_guess_net_profile_step(atkm_guess_net* net, int batch, const float* feats, const double* targets,
                                float lr, float* loss, double* gemm_ms, double* step_ms, int* gemm_calls,
                                double* each_ms, int each_cap, void* stream);

/*
 * atkm_inner_products_noalloc -- out[i] = hvol * Re(sum_j u_i[j] conj(v_i[j]))
 * for i < npairs, without allocating anything.  The paper has no counterpart:
 * this is for callers that cannot call cudaMalloc (code inside a host
 * framework that owns every device allocation, or a process that must not grow
 * its device footprint after start-up).  With hvol = h_x h_y h_z it is the
 * discrete inner product <u_i, v_i> of the solver.
 *   u, v    HOST arrays of npairs DEVICE pointers, each to n interleaved
 *           complex doubles (16-byte aligned).
 *   npairs  1 .. ATKM_NOALLOC_MAX_PAIRS (8); anything else is rejected with
 *           ATKM_ERR_ARG before any work is enqueued.
 *   n       complex elements per vector (> 0).
 *   out     DEVICE array of npairs doubles, written stream-ordered.
 * Scratch: the per-block partial sums live in one file-scope device array of
 * 8 x 1216 doubles (77,824 bytes) that every GPU loading the library holds
 * until the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture.  Every call on a device shares the array: calls
 * whose kernels overlap on the GPU (different streams, no ordering between
 * them) race and may return wrong sums; order them on one stream.  Each call
 * overwrites every partial it reads, so nothing needs clearing between calls.
 * Calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define ATKM_NOALLOC_MAX_PAIRS 8
int atkm_inner_products_noalloc(const double* const* u, const double* const* v, int npairs,
                                unsigned long long n, double hvol, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ATKM_H_ */

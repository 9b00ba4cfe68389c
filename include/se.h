/*
 * libse -- Spectral Ewald summation of the Stokes potentials (stokeslet, rotlet,
 * stresslet) with periodicity in 3, 2, 1 or 0 directions, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Bagge & Tornberg, "Fast Ewald summation for Stokes flow with arbitrary
 * periodicity" (J. Comput. Phys., arXiv 2210.01255). The potential
 *     u^{DP}(x) = sum_n sum_{p in P_DP} G(x - x_n + p) . f(x_n)          (Sec. 2, Eq. periodic-potential)
 * is split (Eq. Dp-ewald-decomp-self) into a real-space part summed over neighbours within
 * r_c (Eq. real-space-potential-Dp), a Fourier-space part computed by the Spectral Ewald
 * method (Sec. 3, Alg. 1: gridding, FFT, scaling by the modified kernel, IFFT, gathering)
 * and the self / zero-mode / gauge corrections (Eqs. self-term, k0-stresslet-3p,
 * 0p-stokeslet-extra-contribution, 1p-stokeslet-extra-contribution).
 *
 * Conventions
 *   - mu = 1 and the kernels exactly as Eq. (stokes-kernels), no 1/(8 pi) factor.
 *   - The first D coordinate directions are periodic (Eq. periodic-images); the primary
 *     cell is [0,L1) x [0,L2) x [0,L3).
 *   - Positions are double [N][3]. Periodic coordinates are wrapped into [0, L_i); a free
 *     coordinate outside [0, L_i) is rejected with SE_ERR_RANGE.
 *   - Strengths and potentials are double in an SE_FP64 plan and float in an SE_FP32 plan:
 *       stokeslet, rotlet: strengths [n_rhs][N][3] = f
 *       stresslet:         strengths [n_rhs][N][6] = (q, nu), source f_lm = q_l nu_m
 *       potential u:       [n_rhs][N_t][3], overwritten.
 *     With kernel_mask = STOKESLET|STRESSLET the strengths are [n_rhs][N][9] = (f, q, nu)
 *     and u is the sum of both flows.
 *       harmonic field:    strengths [n_rhs][N][1] = q; u_j = sum q (x - y)_j / |x - y|^3, the
 *                          field -grad H q of the harmonic kernel H = 1/r (electrostatics: the
 *                          field of point charges). It is split and computed like the rotlet
 *                          (both are first derivatives of H: the rotlet is the curl, this the
 *                          gradient), with the same zero-mode convention (3P k = 0 term dropped,
 *                          i.e. tin-foil boundary conditions) and no self or gauge term.
 *       harmonic potential: strengths [n_rhs][N][1] = q; u = sum q / |x - y| (H = 1/r, Sec.
 *                          2.1: the electrostatic potential of point charges), ONE output
 *                          per target: u is [n_rhs][N_t][1]. Ewald screening and the
 *                          harmonic modified kernels (Eqs. optimal-1p-harmonic,
 *                          vico-harmonic-0p, and the 2P one of Sec. 3.1); the parameter
 *                          rules are the rotlet's (Sec. 4). Self term -2 xi/sqrt(pi) q.
 *                          Zero-mode conventions: 3P zero mean over the cell (for a charged
 *                          system the constant -pi Q / (xi^2 V), Q = sum q, is added); 2P the
 *                          k^P = 0 kernel -2 pi |r_3| of App. A (no constant); 1P the k_1 = 0
 *                          kernel -2 log(rho) of App. B, gauge l_H = 1 (the method's l_H = R
 *                          result is shifted by -2 log(R) Q / L_1); 0P the plain sum.
 *   - targets == NULL selects the star form (targets = sources, the self interaction
 *     omitted, Eq. periodic-potential-star). With explicit targets, a target that
 *     coincides exactly with a source is treated the same way for that source.
 *   - Zero-mode / gauge conventions: 3P stokeslet and rotlet zero mode = 0 and the 3P
 *     stresslet carries Eq. (k0-stresslet-3p) evaluated with the wrapped coordinates;
 *     the 1P stokeslet is reported with l_B = 1, l_H = e^{-1} (the extra contribution of
 *     Eq. 1p-stokeslet-extra-contribution vanishes); the 0P stokeslet goes to zero at
 *     infinity (Eq. 0p-stokeslet-extra-contribution subtracted); 2P needs no constant.
 *
 * Memory ownership: the caller owns every array passed in. The plan owns its grids,
 * tables, FFT plans and scratch; it grows them on demand inside se_eval*.
 * Execution: all device work of a plan is issued on the plan's stream (se_opts.stream),
 * asynchronously; results are complete when that stream is synchronised. Errors of
 * earlier asynchronous work surface at the next call or at se_sync. A plan is not
 * thread-safe; no C++ exception crosses this interface.
 */
#ifndef SE_H
#define SE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct se_plan_t* se_plan_h;

typedef enum {
  SE_OK = 0,
  SE_ERR_ARG = -1,         /* invalid argument (NULL pointer, bad size, bad enum)          */
  SE_ERR_RANGE = -2,       /* a free-direction coordinate outside [0, L_i), or NaN/Inf     */
  SE_ERR_NOMEM = -3,       /* device or host allocation failed                             */
  SE_ERR_CUDA = -4,        /* a CUDA runtime call or kernel launch failed                  */
  SE_ERR_CUFFT = -5,       /* a cuFFT call failed                                          */
  SE_ERR_TIMEOUT = -6,     /* a bounded device-side wait gave up                           */
  SE_ERR_UNSUPPORTED = -7, /* a valid request this build does not implement               */
  SE_ERR_CAPACITY = -8     /* the request exceeds a fixed capacity (see se_real_noalloc)    */
} se_status;

enum { SE_STOKESLET = 1, SE_ROTLET = 2, SE_STRESSLET = 4, SE_HARMONIC_FIELD = 8, SE_HARMONIC = 16 };
enum { SE_WIN_GAUSSIAN = 0, SE_WIN_KB = 1, SE_WIN_PKB = 2 };
enum { SE_FP64 = 0, SE_FP32 = 1 };
/* parts of the decomposition returned by se_eval_parts (bit mask) */
enum { SE_PART_REAL = 1, SE_PART_FOURIER = 2, SE_PART_CORR = 4, SE_PART_ALL = 7 };

typedef struct {
  int prec;          /* SE_FP64 (default) or SE_FP32                                         */
  int f_M;           /* grid sizes rounded to multiples of f_M by the rules of Sec. 4 (4)  */
  double lambda;     /* box padding factor of Eq. (extended-grid-size); 0 = Table 4       */
  int Mext[3];       /* extended grid size M'_i in free directions; 0 = Eq. extended-grid-size */
  double s0;         /* upsampling factor of the k^P = 0 class, Eq. (upsampling-factor-s0); 0 = rule */
  double s_star;     /* upsampling factor of K_*, Eq. (upsampling-factor-sstar); 0 = rule */
  int kbar_star;     /* threshold kbar_* of Eq. (estimate-kbarstar); -1 = rule            */
  double tol_abs;    /* absolute tolerance used by the s_*, kbar_* rules (0 = 1e-10)     */
  double Q;          /* source quantity Q of Eqs. (vector/tensor-source-quantity) for the rules (0 = 1) */
  int kernel_mask;   /* kernels the plan will be used with (for the free-direction rules); 0 = all.
                        SE_HARMONIC_FIELD uses the rotlet's rules and tables             */
  void* stream;      /* cudaStream_t to issue work on; NULL = the legacy default stream   */
  int flags;         /* SE_FLAG_* bits, 0 = defaults                                        */
  double n_rc;       /* se_autotune: average neighbours within r_c used to choose xi when
                        *xi_io <= 0 (Sec. 5.2); 0 = the paper's uniform-case values (Table 5) */
  int P_margin;      /* se_autotune: window points added to the estimate of Eq.
                        (approximation-estimate) by the error-pollution rule, Eq.
                        (error-pollution-fix); -1 = the paper's (4, or 2 for D = 0)          */
  int tile;          /* gridding tile depth TZ along direction 2 (CUDA-core gridding works on
                        tiles of 4 x 4 x TZ grid points, one warp each): 0 = by the number of
                        components per launch (4 for 9-12, 8 for fewer), 4 or 8 forced (a
                        launch of 10-12 components always takes 4); se_autotune_timed
                        chooses it by timing. Same grid to rounding.                     */
} se_opts;

/* se_opts.flags: with SE_FLAG_TC_GRIDDING, FP32 gridding (Alg. 1, gridding step) with window
 * support P <= 16 runs on the tensor cores (tcgen05.mma kind::tf32, operands split into high
 * and low TF32 parts for FP32 accuracy; same results as the CUDA-core gridding to FP32
 * rounding). Without it (default), and always for FP64 or P > 16, gridding runs on the CUDA
 * cores. */
enum { SE_FLAG_TC_GRIDDING = 1 };
/* se_opts.flags, testing aid: with SE_FLAG_TEST_TIMEOUT as well as SE_FLAG_TC_GRIDDING, the
 * tensor-core gridding's bounded waits for finished chunks report a timeout at their first
 * poll, so that the timeout path can be checked without a hang: each CTA flags it, waits for
 * the tensor-core work it has already issued, releases its tensor memory and writes nothing;
 * se_sync then returns SE_ERR_TIMEOUT and the evaluation's result is invalid. */
enum { SE_FLAG_TEST_TIMEOUT = 2 };
/* se_opts.flags: real-space sum with the dense-block path. Targets are grouped in blocks of 32
 * consecutive cell-sorted targets (cells of side >= r_c / 8); a block whose targets lie in a
 * box of side <= r_c is
 * summed by one warp against the candidates of the whole box (staged in shared memory and
 * shared by the 32 targets), the targets of the other blocks one warp per target as without
 * the flag. Pays off where targets have many neighbours (clustered points, large r_c);
 * se_autotune_timed chooses it by timing. Same sums to rounding. */
enum { SE_FLAG_REAL_BLOCKS = 4 };
/* se_opts.flags: FFT-friendly grid sizes. se_autotune rounds every grid extent it chooses (M_i
 * of periodic directions, and M'_i of the free directions) up to the next even number whose
 * prime factors are 2, 3, 5 and 7 only (cuFFT's fastest radices; the D = 0 transform length
 * 2 M' then has them too) instead of a multiple of f_M, and se_plan_create does the same for
 * the upsampled class lengths of Sec. 4.5. The
 * grid only gets finer (h smaller), so the tolerance rules still hold. Without the flag the
 * sizes are the paper's multiples of f_M. */
enum { SE_FLAG_FFT_SIZES = 8 };
/* se_opts.flags: for D = 0, the precomputed truncated biharmonic kernel (stokeslet,
 * stresslet; Sec. 3.5) is split as (B_R - p) + p with p(r) = c0 + c1 r^2 + c2 r^4 + c3 r^6 the
 * least-squares fit of B_R over the 2M' box of offsets (FP64, at plan creation). The
 * Fourier-space step uses B_R - p; the potential of p is added exactly from moment sums of the
 * sources (the operators of the stokeslet and stresslet turn p into polynomials of degree 4
 * and 3 in x - y; the Hasimoto screening changes p only by constants, which they annihilate,
 * and by a multiple of r^2 for the r^6 term, which is included).
 * The potential is the same to the truncation error of the method, but the large values of
 * the truncated biharmonic at small wavenumbers, which multiply the FP32 rounding of the
 * transforms, shrink: in FP32 the rounding of the free-space Fourier part approaches that of
 * the triply periodic one. Rotlet and harmonic kernels are unaffected.
 * se_autotune_timed sets it for D = 0 FP32 stokeslet / stresslet evaluations. */
enum { SE_FLAG_SPLIT_POLY = 16 };
/* se_opts.flags: for D = 0, the extended grid sizes M'_i (given in Mext or from Eq.
 * extended-grid-size) are lower bounds: se_plan_create takes, among the even M'_i up to 25 %
 * larger whose transform lengths 2 M'_i have no prime factor above 7, the ones whose transforms
 * run fastest on this GPU, timing the forward and inverse transforms of one component on
 * scratch memory (cuFFT's speed varies strongly between such lengths: on a GB300 the 0P
 * transforms of 2 M' = 900 took less time than those of 840, 864 or 896). A larger M' only adds
 * zero padding, so the tolerance rules still hold. The choice is kept for the process per
 * (precision, minimum sizes, kernels); se_autotune_timed sets the flag for D = 0. */
enum { SE_FLAG_FFT_TIMED = 32 };

/* Fill *opts with the defaults above. */
se_status se_opts_default(se_opts* opts);

/*
 * Create a plan (Alg. 1 input; Sec. 3.2 discrete formulation).
 *   periodicity  D in {0,1,2,3}: directions 0..D-1 periodic.
 *   box          L_i > 0.
 *   xi           Ewald decomposition parameter (> 0).
 *   rc           real-space cut-off radius (> 0).
 *   M            grid subintervals along each box side; the grid spacing is h = L_0/M_0 and
 *                must be the same in every direction (|L_i/M_i - h| <= 1e-12 h) for the
 *                periodic directions; for free directions M_i only sets h when D = 0
 *                (h = L_0/M_0) and the extended size follows Eq. (extended-grid-size).
 *                Periodic M_i must be even.
 *   P            window support in grid points (even, 2..32), Sec. 3.3.
 *   window       SE_WIN_GAUSSIAN (Eq. TG-window), SE_WIN_KB (Eq. KB-window) or SE_WIN_PKB.
 *   opts         NULL for defaults.
 * Returns SE_OK and a plan in *out, or an error and *out = NULL.
 * Device memory for the plan's tables is allocated here (0P: also the kernel
 * precomputation of Sec. 3.5, which launches GPU work on the plan's stream).
 */
se_status se_plan_create(se_plan_h* out, int periodicity, const double box[3], double xi,
                         double rc, const int M[3], int P, int window, const se_opts* opts);

/*
 * Parameter selection, Sec. 4.6 (steps 1-7), with the relative tolerance converted to an
 * absolute one by tau_abs = tol_rel * U(L,Q,xi) (Sec. 4.2).
 *   kernel_mask  kernels to be evaluated (the strictest parameters over the mask win).
 *   Q            source quantity (Eq. vector-source-quantity / tensor-source-quantity).
 *   N            number of sources (used only when *xi <= 0: xi is then chosen from the
 *                average number of neighbours of Table 5, uniform system).
 *   tol_rel      relative rms tolerance of the Fourier-space part.
 *   io_opts      in: f_M (0 = 4), lambda; out: Mext, s0, s_star, kbar_star, tol_abs filled in.
 *   xi           in/out: the decomposition parameter (<= 0: chosen here).
 *   rc, M, P     out: cut-off radius, grid sizes along the box sides, window support.
 * The window is the PKB window (Sec. 3.3).
 */
se_status se_autotune(int periodicity, const double box[3], int kernel_mask, double Q,
                      long long N, double tol_rel, se_opts* io_opts, double* xi, double* rc,
                      int M[3], int* P);

/*
 * Parameter selection with measured costs. The rules of Sec. 4.6 fix r_c, M and P for a
 * given xi at the tolerance; se_autotune takes xi from an average neighbour count n_rc that
 * holds for uniform systems (Table 5, Sec. 5.2). For other point distributions (a dense
 * cluster multiplies the real-space pairs) and for this GPU's cost balance, this function
 * chooses the split by timing instead: n_rc is scaled by f^3 (r_c by f) over a geometric
 * ladder f = 0.8^k around 1 (starting from io_opts->n_rc, or from the uniform rule when it is
 * 0), se_autotune gives each candidate's parameters, and a plan of each candidate evaluates
 * the caller's own sources and strengths (star form) once untimed and twice timed with CUDA
 * events; the first step decides the direction (towards the faster), and the walk continues
 * until two candidates in a row are invalid (FP32 rounding, below) or more than 10 % slower
 * than the best, a candidate's grids would use more than half of the free device memory, or
 * its grid is unsupported. The real-space path is chosen the same way: both the
 * per-target and the dense-block path (SE_FLAG_REAL_BLOCKS) are timed at the first candidate,
 * the faster is used along the walk, both are timed again at the chosen r_c, and the choice is
 * returned in io_opts->flags (the other flags are kept as given; for D = 0 SE_FLAG_FFT_TIMED
 * is added, and for D = 0 FP32 stokeslet and stresslet evaluations SE_FLAG_SPLIT_POLY). Last,
 * the gridding tile depth
 * (io_opts->tile = 4 and 8, CUDA-core gridding) is timed at the chosen parameters and the
 * fastest of the two and the caller's own value is returned in io_opts->tile. FP32 trials also bound the
 * rounding: each candidate evaluates once more with the linear part of the strengths scaled
 * by 1.3 (f, the stresslet's q, the charges), and the relative rms of u(1.3 f)/1.3 - u(f) over
 * a fixed sample of 2048 targets estimates its rounding. A candidate whose estimate exceeds
 * 3.5 tol_rel is not chosen (the estimate varies between repeated trials by about 2x, so it
 * decides eligibility, not the direction of the walk) (the FP32 rounding of the free-space transforms grows with xi,
 * so large grids can cost more accuracy than the truncation rules allow); if no candidate
 * passes, SE_ERR_UNSUPPORTED. Temporary device memory: one output array (FP32: two, and one
 * copy of the strengths) and the trial plans (one at a time).
 *   periodicity, box, kernel_mask, Q, tol_rel   as se_autotune (kernel_mask: one kernel or
 *                SE_STOKESLET|SE_STRESSLET, as for se_eval; tol_rel > 0, the absolute-tolerance
 *                mode of se_autotune is not offered here). Invalid arguments: SE_ERR_ARG.
 *   n_src, src, strengths, n_rhs   the evaluation to time, as se_eval (device arrays).
 *   window       the window of the plans (SE_WIN_*).
 *   io_opts      in: as se_autotune, plus prec, stream and flags for the trial plans;
 *                out: the chosen candidate's options (n_rc, Mext, s0, s_star, kbar_star, ...).
 *   xi, rc, M, P out: the chosen parameters.
 *   ms           out (may be NULL): the chosen candidate's measured time per evaluation.
 * Synchronous: returns when the trials are done.
 */
se_status se_autotune_timed(int periodicity, const double box[3], int kernel_mask, double Q,
                            long long n_src, const double* src, const void* strengths, int n_rhs,
                            double tol_rel, int window, se_opts* io_opts, double* xi, double* rc,
                            int M[3], int* P, double* ms);

/*
 * Evaluate the potential (Eqs. Dp-ewald-decomp / Dp-ewald-decomp-self).
 *   kernel_mask  SE_STOKESLET, SE_ROTLET, SE_STRESSLET, SE_STOKESLET|SE_STRESSLET,
 *                SE_HARMONIC_FIELD or SE_HARMONIC.
 *   n_src, src   device double [n_src][3].
 *   strengths    device [n_rhs][n_src][c], c = 3 (S, Omega), 6 (T), 9 (S|T) or 1 (harmonic
 *                field, harmonic potential); float in an SE_FP32 plan, double in an SE_FP64
 *                plan.
 *   n_rhs        number of right-hand sides (strength vectors at the same points), >= 1.
 *   n_tgt, tgt   device double [n_tgt][3], or tgt = NULL for the star form (n_tgt ignored).
 *   u            device [n_rhs][N_t][3] (SE_HARMONIC: [n_rhs][N_t][1]) of the plan's
 *                precision, overwritten.
 * Asynchronous on the plan's stream.
 */
se_status se_eval(se_plan_h plan, int kernel_mask, long long n_src, const double* src,
                  const void* strengths, int n_rhs, long long n_tgt, const double* tgt, void* u);

/* As se_eval, returning only the parts selected by parts_mask (SE_PART_*): the real-space
 * sum, the Fourier-space part u_h^{DP,F} (Alg. 1) and the corrections (self term, 3P
 * stresslet zero mode, 0P/1P stokeslet gauge constants). */
se_status se_eval_parts(se_plan_h plan, int kernel_mask, int parts_mask, long long n_src,
                        const double* src, const void* strengths, int n_rhs, long long n_tgt,
                        const double* tgt, void* u);

/* As se_eval with HOST arrays (same layouts): copies in, evaluates and copies the result
 * back through plan-owned pinned staging buffers; returns when u is filled. */
se_status se_eval_host(se_plan_h plan, int kernel_mask, long long n_src, const double* src,
                       const void* strengths, int n_rhs, long long n_tgt, const double* tgt,
                       void* u);

/* Read back plan information: h, the grid sizes actually used (n[3]: FFT grid per
 * direction, m[3]: spread-grid extent per direction), R (truncation radius, 0 for 3P),
 * s0, s_star, kbar_star, the number of kernels launched by the last evaluation and its
 * per-stage device times in ms (times[0..7]: bin, spread, fft, scale, ifft, gather, real,
 * corr; -1 when timing is off; for D < 3 "fft" includes the class copies of the adaptive
 * FFT into their buffers and "ifft" the copies back), and the number of k-space modes per
 * component that the scaling step visited (all classes). Reading the times waits for the
 * last evaluation. */
typedef struct {
  double h, R, s0, s_star, dL[3];
  int n[3], m[3], kbar_star, P;
  float times_ms[8];
  int launches;        /* kernels libse launched in the last evaluation (cuFFT's not counted) */
  long long scale_modes; /* k-space modes per component that the last scaling step visited  */
} se_info;
se_status se_get_info(se_plan_h plan, se_info* info);

/* Copy the plan's spread grid (after the last evaluation, before the FFT) to host memory:
 * component-major [C][n0][n1][n2] (D = 0: [C][m0][n1][n2], the first m0 planes of the zero-
 * padded grid) in the plan's precision; bytes must be >= the grid size.
 * Used to check the gridding step (Eq. SE-gridding-disc) in isolation. */
se_status se_debug_grid(se_plan_h plan, void* host_dst, unsigned long long bytes);

/* Enable per-stage CUDA-event timing of subsequent evaluations (0 = off). */
se_status se_set_timing(se_plan_h plan, int on);

/* Wait for the plan's stream and report any asynchronous device error. */
se_status se_sync(se_plan_h plan);

/* Release the plan and everything it owns. NULL is accepted. */
void se_destroy(se_plan_h plan);

/*
 * Real-space sum without any device allocation (this paper has no counterpart: it is an
 * interface for callers that cannot allocate device memory while they run -- code inside a
 * framework that owns all device memory through its own pre-allocated pool, or a time-step
 * loop that must never stall or fail on an allocation).
 * Computes the same values as se_eval_parts(plan, kernel, SE_PART_REAL, ...) in the star
 * form (targets = sources) for one right-hand side, with the same cut-off rc and, for the
 * stokeslet, the same self term.
 *   periodicity, box, xi, rc  as in se_plan_create; kernel: one of SE_STOKESLET, SE_ROTLET,
 *                             SE_STRESSLET; prec: SE_FP64 (double strengths and u) or SE_FP32.
 *   n_src, src                device double [n_src][3]; strengths device [n_src][c].
 *   u                         device [n_src][3], overwritten.
 *   stream                    cudaStream_t (NULL = legacy default stream).
 * Synchronous: the work is issued on the stream, then the call waits for it and reads the
 * device status word back (4 bytes into a host variable), so that a free-direction coordinate
 * outside [0, L_i) or a non-finite coordinate returns SE_ERR_RANGE as se_eval_parts and
 * se_sync do (u then holds values for the clamped positions and must be discarded).
 * Scratch: a fixed 16 MiB array inside the library (held by every GPU that loads it until
 * the process exits); limits n_src <= 65536 and at most 32 cells per direction; larger
 * requests return SE_ERR_CAPACITY before any work. No cudaMalloc, cudaFree or allocating
 * library call is made. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) once for that device. Every call shares the one array and keeps its
 * last contents (the counters and the status word are cleared at the start of each call);
 * calls that overlap on the GPU (different streams, or host threads) race on it and must be
 * serialised by the caller.
 */
se_status se_real_noalloc(int periodicity, const double box[3], double xi, double rc, int kernel,
                          int prec, long long n_src, const double* src, const void* strengths,
                          void* u, void* stream);

/*
 * A fixed batch of independent evaluations (for example many singly periodic systems of
 * different sizes, each with its own plan and right-hand sides) replayed with one launch.
 * se_batch_create evaluates every configuration once (star form: targets = sources), so
 * that every buffer and cuFFT plan exists, then records all the evaluations into a CUDA
 * graph on the plans' shared stream. All plans must use the same stream, which must not be
 * the legacy default stream (NULL), and must not have timing enabled. The arrays passed here
 * (src, strengths, u of every configuration) are the ones every replay reads and writes:
 * refill the inputs in place between launches. Arguments per configuration i:
 * kernel_mask[i], n_src[i], src[i], strengths[i], n_rhs[i], u[i] as in se_eval.
 * se_batch_launch replays the graph asynchronously on that stream (results are complete
 * when the stream is synchronised); se_batch_destroy releases the graph (not the plans).
 */
typedef struct se_batch_t* se_batch_h;
se_status se_batch_create(se_batch_h* out, int n_cfg, const se_plan_h* plans, const int* kernel_mask,
                          const long long* n_src, const double* const* src,
                          const void* const* strengths, const int* n_rhs, void* const* u);
se_status se_batch_launch(se_batch_h batch);
void se_batch_destroy(se_batch_h batch);

/*
 * Many independent configurations on ONE plan, each stage one launch over all of them
 * (batching of Sec. 5's independent systems; the plan's box, xi, r_c, M, P and window serve
 * every configuration, so pick parameters that meet the tolerance for each, e.g. from the
 * largest N and the smallest source quantity Q).
 *   n_cfg        number of configurations (>= 1).
 *   n_src        HOST long long [n_cfg]: points of each configuration (>= 0, total < 2^31).
 *   src          device double [sum n_src][3]: the configurations' points one after the other.
 *   strengths    device, per configuration a [n_rhs][n_src[c]][c_k] block (c_k as se_eval),
 *                the blocks one after the other.
 *   u            device, per configuration a [n_rhs][n_src[c]][3] block ([...][1] for
 *                SE_HARMONIC), the blocks one after the other, overwritten.
 * Star form (targets = sources of each configuration); a configuration's points interact only
 * with each other. Sorting keys, grid components and outputs are offset per configuration:
 * one gridding launch covers the tiles of all configurations, the transforms and the scaling
 * run over all configurations' components at once, one gathering and one real-space launch
 * cover all targets; the corrections run per configuration. Consecutive configurations are
 * taken together as far as the buffers allow (the adaptive FFT's class buffers of D = 2, 1
 * are indexed with 32-bit offsets, and a group's buffers are held to half the free device
 * memory): a larger group runs as a few such evaluations in sequence. The offsets are copied
 * to the device when they change (so a first call with given n_src comes before any stream
 * capture of a call with the same n_src). Tensor-core gridding is not used for a group.
 * se_get_info reports the kernels of all sub-groups and the stage times of the last one.
 * Asynchronous on the plan's stream. Errors: SE_ERR_ARG (bad argument), SE_ERR_UNSUPPORTED (a
 * key count beyond 2^31), otherwise as se_eval.
 */
se_status se_eval_group(se_plan_h plan, int kernel_mask, int n_cfg, const long long* n_src, const double* src,
                        const void* strengths, int n_rhs, void* u);

/*
 * The same entry points under the names of the problem statement:
 * se_plan         = se_plan_create (same arguments and behaviour).
 * se_eval_batch   evaluates n_cfg independent configurations (star form, targets = sources),
 *                 configuration i as se_eval(plans[i], kernel_mask[i], n_src[i], src[i],
 *                 strengths[i], n_rhs[i], 0, NULL, u[i]), issued in order, each on its plan's
 *                 stream (asynchronous; plans on different streams run concurrently). Returns
 *                 the first error (SE_ERR_ARG for a NULL array or plan, before any work).
 *                 For repeated evaluations of the same configurations, se_batch_create
 *                 records them once into a CUDA graph that se_batch_launch replays.
 */
se_status se_plan(se_plan_h* out, int periodicity, const double box[3], double xi, double rc,
                  const int M[3], int P, int window, const se_opts* opts);
se_status se_eval_batch(const se_plan_h* plans, int n_cfg, const int* kernel_mask,
                        const long long* n_src, const double* const* src,
                        const void* const* strengths, const int* n_rhs, void* const* u);

/* Human-readable name of a status code (static storage). */
const char* se_status_str(se_status s);

#ifdef __cplusplus
}
#endif
#endif

/*
 * fh.h -- C ABI of the GB300 fast-hybrid 2D scattering library (libfh).
 *
 * The library computes the time-domain field scattered by a 2D sound-soft
 * obstacle under single-direction incidence by the frequency/time hybrid
 * method of Anderson, Bruno & Lyon ("fast-hybrid" wave solver, Part I):
 *
 *   F3  J frequency-domain CFIE solves (Sec. 2.3, eq. CFIE_direct), one per
 *       non-zero frequency of a fixed mesh, for plane-wave data e^{i kappa p.r};
 *   F1-F2  recentred window spectra B_k^slow(omega_j) of the incident signal
 *       (Sec. 3.1 eq. window_func; Sec. 3.2 eq. Bkslow_eqn);
 *   F4-F5, T0-T6  target fields V(x, omega_j) = int psi G dsigma and the
 *       band-limited, recentred Fourier synthesis (Sec. 3.2 eqs. Ukslow_repr,
 *       ukW; Sec. 4.1 eqs. fourier_approx, approx) giving u(x, T) at any T at
 *       a cost independent of T.
 *
 * Conventions (all entry points):
 *  - Every call returns an fh_status.  On failure the outputs are untouched,
 *    the context keeps its previous state, and fh_last_error() holds a message.
 *  - Host pointers are owned by the caller and only read/written during the
 *    call.  "_dev" variants take device pointers on the context's device; they
 *    are stream-ordered on the context stream (fh_set_stream) and the caller
 *    keeps them alive until that stream has passed the call.
 *  - Device memory for densities, spectra and work space is owned by the
 *    context and released by fh_destroy().
 *  - Calls out of order (fh_sample before fh_solve_frequencies and
 *    fh_window_spectra) return FH_ESTATE.
 *  - A context is not thread-safe; use one context per thread / serving slot.
 *  - Complex arrays are interleaved (re, im) doubles.
 *  - The library never falls back to the CPU: without a usable CUDA device,
 *    fh_create fails with FH_ECUDA.
 */
#ifndef FH_H
#define FH_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fh_ctx fh_ctx;

typedef enum {
    FH_OK = 0,
    FH_EINVAL = 1,     /* invalid argument (message says which)            */
    FH_ENOMEM = 2,     /* device allocation failed                         */
    FH_ECUDA = 3,      /* CUDA runtime error (message has the CUDA string)  */
    FH_ESTATE = 4,     /* call order: required earlier step missing        */
    FH_ESINGULAR = 5,  /* zero or non-finite pivot in a frequency solve    */
    FH_ENOCONV = 6,    /* iterative refinement did not reach its tolerance */
    FH_ETIMEOUT = 7    /* a bounded device wait gave up                    */
} fh_status;

/* Precision of the frequency solves (fh_create). */
enum {
    FH_FP64 = 0,        /* assembly, LU and solve in IEEE binary64          */
    FH_MIXED_FP32 = 1,  /* FP64 assembly; FP32 LU; FP64 iterative refinement */
    FH_MIXED_TF32 = 2,  /* FP64 assembly; LU with trailing updates on the tensor
                           cores (tcgen05, 3xTF32 split, FP32 accumulation);
                           FP64 iterative refinement; N <= 4096              */
    FH_MIXED_BF16 = 3   /* as FH_MIXED_TF32 with BF16 operands (3xBF16 split) */
};

/* Obstacle descriptions: smooth closed curves, counter-clockwise in t. */
enum {
    FH_CURVE_CIRCLE = 0,  /* z = center + r0 (cos t, sin t)                          */
    FH_CURVE_KITE = 1,    /* z = center + (cos t + 0.65 cos 2t - 0.65, 1.5 sin t)   */
    FH_CURVE_STAR = 2     /* z = center + r(t)(cos t, sin t),
                             r = r0 + sum_{k=1}^{n_harm} amp[k-1] cos(k t + phase[k-1]) */
};
#define FH_MAX_HARMONICS 16

typedef struct {
    int kind;
    double r0;
    int n_harm;
    double amp[FH_MAX_HARMONICS];
    double phase[FH_MAX_HARMONICS];
    double center[2];
} fh_curve;

typedef struct {
    int n_solves;            /* frequency solves performed (omega_j > 0)          */
    int max_N;               /* largest boundary size                             */
    long long matrix_entries;/* sum of N_j^2                                      */
    int refine_iters_max;    /* mixed modes: most refinement sweeps of any solve  */
    double residual_max;     /* mixed modes: largest final relative residual      */
} fh_solve_stats;

/* Create a context on CUDA device `device` with solve precision `precision`
 * (FH_FP64, FH_MIXED_FP32, FH_MIXED_TF32 or FH_MIXED_BF16).  *out receives the context.  The context owns a
 * non-blocking CUDA stream until fh_set_stream selects another one.  Inside a
 * call, independent work may fork onto private helper streams of the context
 * (the near-diagonal band of the assembly, the largest systems started early,
 * the tensor-core LU's cluster sizes); every fork is joined back into the
 * context stream within the same call, so all results are ordered on it.
 * Errors: FH_EINVAL (bad precision / NULL out), FH_ECUDA (no such device). */
fh_status fh_create(fh_ctx **out, int device, int precision);

/* Release all device memory and the owned stream.  NULL is accepted. */
void fh_destroy(fh_ctx *ctx);

/* Message of the last failing call on this context ("" if none). */
const char *fh_last_error(const fh_ctx *ctx);

/* Use `cuda_stream` (a cudaStream_t on the context's device; NULL restores
 * the context's own stream) for all later work of this context. */
fh_status fh_set_stream(fh_ctx *ctx, void *cuda_stream);

/* Steps F3 set-up (Sec. 5 "Overall algorithm", Sec. 2.3): fix the obstacle,
 * the frequency mesh and the incidence direction.
 *   curve   obstacle (host struct, copied)
 *   J       number of frequencies, 2 <= J <= 4097
 *   omega   J frequencies, ascending, uniform, omega[0] == 0 (host).  omega[J-1]
 *           is the band limit W; the synthesis uses M = 2(J-1) full-band nodes.
 *   N       J boundary sizes (host; N[j] even, 8 <= N[j] <= 8192); N[0] is
 *           ignored (no solve at omega = 0).  NULL: N[j] = 64 for all j.
 *   c       wave speed (> 0); kappa_j = omega_j / c
 *   p       unit incidence direction (host, 2 doubles)
 * The Nystrom nodes t_i = pi i / n (i < N = 2n) and z, z', z'' are computed on
 * the device.  Invalidates earlier densities, spectra and target fields. */
fh_status fh_discretize(fh_ctx *ctx, const fh_curve *curve, int J, const double *omega,
                        const int *N, double c, const double p[2]);

/* Step F3 (Sec. 5; eq. CFIE_direct): assemble and solve the J-1 CFIE systems
 * A_j psi_j = g_j, g = dB/dn - i eta B for B = e^{i kappa p.r}.  Densities stay
 * resident on the device.
 *   eta    coupling per frequency (host, J doubles; eta[0] ignored) or NULL
 *          for eta_j = omega_j.
 *   stats  may be NULL.
 * Errors: FH_ESTATE (no fh_discretize), FH_ESINGULAR (zero/non-finite pivot;
 * the message names the frequency), FH_ENOCONV (mixed precision only),
 * FH_ETIMEOUT (a bounded tensor-core completion wait gave up). */
fh_status fh_solve_frequencies(fh_ctx *ctx, const double *eta, fh_solve_stats *stats);

/* Steps F1-F2 (Sec. 3.1 eq. window_func; Sec. 3.2 eqs. ak_signal_def,
 * Bkslow_eqn): window spectra B_k^slow(omega_j) = int_{-H}^{H} w(tau)
 * a(s_k + tau) e^{i omega_j tau} dtau by the trapezoidal rule on the sample
 * grid, for s_k = 1.5 H (k-1), k = 1..K, K = #{k >= 1 : s_k - H < t_last}.
 *   a          n_samples real samples a(t0 + q dt) (host); a = 0 outside them
 *   t0, dt     sample grid; H/dt and (H + t0)/dt must be integers (1e-9)
 *   H          window half-width (the paper uses H = 10)
 * Requires fh_discretize.  Spectra stay resident on the device.  FH_EINVAL if
 * the signal spans more windows than the synthesis weights hold in shared
 * memory (52 K bytes, plus 24 (2J - 2) bytes when J > 1025, at most 204800:
 * K <= 3938 for J <= 1025). */
fh_status fh_window_spectra(fh_ctx *ctx, const double *a, int n_samples, double t0,
                            double dt, double H);

/* As fh_window_spectra with `d_a` in device memory. */
fh_status fh_window_spectra_dev(fh_ctx *ctx, const double *d_a, int n_samples, double t0,
                                double dt, double H);

/* Steps F4-F5 and T0-T6 (Sec. 5): scattered field u(x_i, T_l).
 *   x      2*n_x doubles, interleaved (x0, y0, x1, y1, ...) (host)
 *   T      n_T sample times (host), any real values
 *   u_out  n_x*n_T doubles, row-major by target (u_out[i*n_T + l]) (host)
 * Target fields V(x, omega_j) are recomputed for every call (V(x, 0) := 1, the
 * 2D low-frequency limit); the densities and spectra are reused, never
 * re-solved.  n_x == 0 or n_T == 0 is a no-op.  Requires
 * fh_solve_frequencies and fh_window_spectra. */
fh_status fh_sample(fh_ctx *ctx, const double *x, int n_x, const double *T, int n_T,
                    double *u_out);

/* As fh_sample with device pointers d_x, d_T and d_u (same layouts). */
fh_status fh_sample_dev(fh_ctx *ctx, const double *d_x, int n_x, const double *d_T, int n_T,
                        double *d_u);

/* ---- batches: several problems solved in the same launches ---- */

/* Like fh_discretize for P problems at once (frequency parallelism across
 * problems, Sec. 1 and Sec. 5 step F3): problem q has curve curves[q], J[q]
 * frequencies omega[o_q .. o_q + J[q] - 1] and sizes N[o_q ..] (o_q = sum of
 * J[0..q-1]; N may be NULL), wave speed c[q] and direction p[2q], p[2q+1].
 * fh_solve_frequencies then assembles and factorises the systems of all
 * problems in shared launches (largest first); spectra and sampling are per
 * problem (the _p calls).  The single-problem calls act on problem 0; eta for
 * fh_solve_frequencies is indexed like omega.  Each problem's results equal
 * those of solving it alone. */
fh_status fh_discretize_batch(fh_ctx *ctx, int P, const fh_curve *curves, const int *J,
                              const double *omega, const int *N, const double *c,
                              const double *p);

/* Number of problems of the context (1 after fh_discretize). */
fh_status fh_num_problems(fh_ctx *ctx, int *P);

/* fh_window_spectra / fh_sample (and device variants) for problem `problem`. */
fh_status fh_window_spectra_p(fh_ctx *ctx, int problem, const double *a, int n_samples,
                              double t0, double dt, double H);
fh_status fh_window_spectra_p_dev(fh_ctx *ctx, int problem, const double *d_a, int n_samples,
                                  double t0, double dt, double H);
fh_status fh_sample_p(fh_ctx *ctx, int problem, const double *x, int n_x, const double *T,
                      int n_T, double *u_out);
fh_status fh_sample_p_dev(fh_ctx *ctx, int problem, const double *d_x, int n_x,
                          const double *d_T, int n_T, double *d_u);

/* Time samples on resident target fields (no fresh step F5): u(x_i, T_l)
 * for the targets of the last fh_sample* call of problem `problem` (or of the
 * last fh_synthesize for problem 0), whose V(x_i, omega_j) stay on the device,
 * at new times T (host / device; u as in fh_sample, n_x of that call).  Only
 * the synthesis weights and the contraction run (Sec. 5 T0-T6), so the cost
 * per time sample does not include the target-field evaluation; fields from
 * before a later fh_discretize*, fh_solve_frequencies, fh_set_densities or
 * fh_autotune are not resident (FH_ESTATE). */
fh_status fh_resample_p(fh_ctx *ctx, int problem, const double *T, int n_T, double *u_out);
fh_status fh_resample_p_dev(fh_ctx *ctx, int problem, const double *d_T, int n_T, double *d_u);

/* Density psi_j (N_j complex) of frequency j of problem `problem`. */
fh_status fh_get_density_p(fh_ctx *ctx, int problem, int j, double *psi);

/* Device bytes a context needs for P problems with J[q] frequencies and sizes
 * N (laid out as in fh_discretize_batch) at `precision`, excluding the
 * per-call sampling work space (about 16 (J + n_items) n_x + 16 J n_T bytes).
 * Used for admission by memory footprint.  No device is touched. */
fh_status fh_footprint(const int *J, const int *N, int P, int precision, long long *bytes);

/* Free and total device memory of CUDA device `device` now (cudaMemGetInfo),
 * for admission against what the device actually has.  FH_ECUDA if the
 * device cannot be queried. */
fh_status fh_device_memory(int device, long long *free_bytes, long long *total_bytes);

/* ---- inspection of resident state (host buffers; used by parity tests) ---- */

/* Number of windows K of the last fh_window_spectra. */
fh_status fh_get_num_windows(fh_ctx *ctx, int *K);

/* Window centres s (K doubles) and spectra B (K*J complex, B[k*J + j]). */
fh_status fh_get_window_spectra(fh_ctx *ctx, double *s, double *B);

/* Nodes of frequency j: z, dz, ddz as 2*N_j doubles each, interleaved. */
fh_status fh_get_geometry(fh_ctx *ctx, int j, double *z, double *dz, double *ddz);

/* Assemble the CFIE matrix of frequency j (coupling eta_j) into a scratch
 * buffer and copy it out: A (N_j*N_j complex, row-major A[i*N_j + l]) and the
 * right side g (N_j complex).  Does not change the context's state. */
fh_status fh_assemble_matrix(fh_ctx *ctx, int j, double eta_j, double *A, double *g);

/* Density psi_j of frequency j (N_j complex) after fh_solve_frequencies. */
fh_status fh_get_density(fh_ctx *ctx, int j, double *psi);

/* Replace the resident densities by caller data (all j > 0 concatenated,
 * sum_j N_j complex values) and mark them solved.  Lets the synthesis be
 * checked independently of the solver. */
fh_status fh_set_densities(fh_ctx *ctx, const double *psi_all);

/* Target fields V(x_i, omega_j) of the last fh_sample (n_x*J complex,
 * V[i*J + j]). */
fh_status fh_get_target_field(fh_ctx *ctx, double *V);

/* Synthesis only (steps T0-T6) from caller-given target fields V (n_x*J
 * complex, V[i*J + j], host) and the resident spectra; u_out as fh_sample. */
fh_status fh_synthesize(fh_ctx *ctx, const double *V, int n_x, const double *T, int n_T,
                        double *u_out);

/* ---- synthesis without allocation ---- */

/* The paper has no counterpart to this entry point: it exists for callers that
 * cannot allocate device memory when they need a field (a serving loop with a
 * fixed memory budget, a host whose device memory comes from its own arena, or
 * code that must avoid the implicit synchronisation of cudaMalloc/cudaFree).
 * It runs the synthesis steps T0-T6 (the same kernels as fh_sample's
 * weights and contraction) with all scratch in one static device array
 * (about 14.0 MB, held on every GPU that loads the library until exit); it
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   J, W     frequency mesh: J nodes on [0, W] (2 <= J <= 2049)
 *   K, d_s   K window centres (device, K doubles)
 *   d_B      window spectra B_k^slow(omega_j), K*J complex, B[k*J + j] (device)
 *   d_V      target fields, J*n_x complex, V[j*n_x + i] (device); V[0*n_x + i]
 *            is the omega = 0 value (1 for the 2D low-frequency limit)
 *   d_T      n_T sample times (device);  d_u  n_x*n_T doubles, u[i*n_T + l] (device)
 *   stream   cudaStream_t to launch on (NULL: legacy default stream)
 * Limits: J*n_T <= 524288, and 52 K + 24 M <= 204800 (M = 2(J-1): the weights
 * kernel's per-window and phase arrays in shared memory; K <= 2048 at J = 2049).
 * Larger sizes return FH_EINVAL; nothing is launched.  A CUDA error left
 * pending by earlier work on the calling thread is returned as FH_ECUDA before
 * anything is launched, and left in place for its owner. 
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress) with that device current; make it before any stream
 * capture.  Every call reuses the same array, whose contents are whatever the
 * last call left (each call overwrites all it reads); calls that overlap on
 * the GPU (different streams, or devices sharing nothing but this array's
 * symbol on one device) race on it and must be serialised by the caller. */
fh_status fh_synthesize_static(int J, double W, int K, const double *d_s, const double *d_B,
                               const double *d_V, int n_x, const double *d_T, int n_T,
                               double *d_u, void *stream);

/* ---- 2D synthesis with the low-frequency split; scaled convolutions ---- */

/* The frequency set F^sing of the singular quadrature (Sec. 4.2, eqs.
 * gradedmesh, gradedmeshIntRule): on the graded mesh mu_j = omega_c (j/4)^9.1,
 * j = 1..4, the 8 Clenshaw-Curtis points (a+b)/2 + (b-a)/2 cos(pi c/7), c =
 * 0..7, of each subinterval [a, b] = [mu_{j-1}, mu_j], j = 2..4, interval by
 * interval: out receives 24 doubles (host; shared end points appear twice).
 * Errors: FH_EINVAL (omega_c not positive and finite, NULL out). */
fh_status fh_sing_frequencies(double omega_c, double *out);

/* Steps T1b-T2d and T5 (Sec. 5) for the 2D case: u(x_i, T_l) = sum_k (1/pi)
 * Re[ I_{w_c}^{W}[F_k](T_l - s_k) + I_0^{w_c}[F_k](T_l - s_k) ], F_k(w) =
 * B_k^slow(w) V(x_i, w) (eq. fourier_sing_decomp with F(-w) = conj F(w)).
 * The smooth piece on [w_c, W] (w_c = j_c W/(J-1)) is the term-wise integral
 * (eq. approx) of the FC(Gram) Fourier continuation (Remark Fourier-FC; d = 6
 * matching and C = 31 continuation points) of the samples at omega_j, j =
 * j_c .. J-1; the singular piece on (0, w_c] is the Filon-Clenshaw-Curtis rule
 * on the points of fh_sing_frequencies(w_c).  The smooth piece's sums over the
 * continuation run in compensated double-float on the FP32 pipe, everything
 * else in FP64: u agrees with the FP64 oracle's split synthesis to ~1e-10
 * relative (measured 8.8e-11 on a small kite, 1.1e-12 on the circle).
 *   J, W       uniform mesh omega_j = j W/(J-1); n = J - j_c >= 12 and n + 31 even
 *   j_c        index of w_c (>= 1)
 *   K, d_s     window centres (device, K doubles)
 *   d_B        B_k^slow(omega_j), K*J complex, B[k*J + j] (device)
 *   d_Bs       B_k^slow at the 24 singular frequencies, K*24 complex (device)
 *   d_V        V(x_i, omega_j), J*n_x complex, V[j*n_x + i] (device)
 *   d_Vs       V(x_i, .) at the singular frequencies, 24*n_x complex (device)
 *   d_T, d_u   n_T times; u as n_x*n_T doubles, u[i*n_T + l] (device)
 *   stream     cudaStream_t (NULL: legacy default stream); work is stream-ordered
 * Work space is taken from the device's stream-ordered allocator and returned
 * on the same stream.  FH_EINVAL (sizes), FH_ENOMEM, FH_ECUDA (also for a
 * CUDA error pending from earlier work, which is left in place). */
fh_status fh_synthesize_sing(int J, double W, int j_c, int K, const double *d_s, const double *d_B,
                             const double *d_Bs, const double *d_V, const double *d_Vs, int n_x,
                             const double *d_T, int n_T, double *d_u, void *stream);

/* Sec. 4.1.2, eqs. conv_sum, conv_sum_2, approx_conv_sum: for each of `batch`
 * coefficient vectors c (M complex, c_m for m = -M/2 .. M/2-1; device,
 * consecutive) the scaled convolution d_n = sum_m c_m b(beta n - gamma m) with
 * b(q) = 2A sinc(2A q / P) (eq. discConv; normalised sinc), approximated by
 * (1/L) sum_p C_p^{(gamma)} B_p e^{2 pi i beta n p / L} for n = n0 - L/2 ..
 * n0 + L/2 - 1: C^{(gamma)} the gamma-fractional DFT of c zero-padded to L, B
 * the DFT of b at the integers -L/2 .. L/2-1, each fractional DFT by the chirp
 * factorisation as a circular convolution of radix-2 FFTs.  d_d receives
 * batch*L complex (device).  L even, M <= L <= 2^24.  Work space as for
 * fh_synthesize_sing.  The error of the approximation is O(L^-2) for P > 2A. */
fh_status fh_scaled_convolution(const double *d_c, int M, int batch, double beta, double gamma,
                                long long n0, int L, double A, double P, double *d_d, void *stream);

/* Window count and spectra of problem `problem` of a batch: as
 * fh_get_num_windows and fh_get_window_spectra (s: K doubles, B: K*J complex). */
fh_status fh_get_num_windows_p(fh_ctx *ctx, int problem, int *K);
fh_status fh_get_window_spectra_p(fh_ctx *ctx, int problem, double *s, double *B);

/* ---- kernel timing and launch accounting ---- */

/* Phases of the path, in order: nodes and tables (a1), CFIE assembly with
 * right sides (a2), LU + solve (FP64) or the factorisation of the mixed paths
 * (a3), the mixed paths' FP64 iterative refinement (a3), window spectra (a4),
 * target fields (a5), synthesis weights (a6), synthesis contraction (a7). */
enum { FH_PH_GEOMETRY = 0, FH_PH_ASSEMBLE, FH_PH_FACTOR, FH_PH_REFINE, FH_PH_SPECTRA, FH_PH_FIELD,
       FH_PH_WEIGHTS, FH_PH_CONTRACT, FH_NUM_PHASES };

typedef struct {
    double ms[FH_NUM_PHASES];           /* device time per phase (CUDA events) */
    long long launches[FH_NUM_PHASES];  /* kernels launched per phase            */
    long long events[FH_NUM_PHASES];    /* timed launch groups per phase         */
} fh_timings;

/* enable != 0 (the default): fh_solve_frequencies and fh_sample run their
 * launch sequences as CUDA graphs.  The first call with a given
 * discretization, buffer set and (for fh_sample) problem, sizes and pointers
 * launches directly, the second captures the sequence and later calls replay
 * it; fh_discretize with unchanged inputs keeps its tables and buffers, so the
 * graphs stay valid across repeated discretize-solve-sample cycles.  The
 * kernels and their results are the same either way.  Graphs are not used
 * while kernel timing (fh_set_timing) is on. */
fh_status fh_set_graphs(fh_ctx *ctx, int enable);

/* Schedule parameters of the batched kernels (launch shapes only: every
 * setting computes the same discrete quantities, equal up to rounding order).
 *   assemble_group   frequencies of equal N assembled together per CTA tile
 *                    (1..8; they share the geometry of each node pair)
 *   field_group      frequencies of equal N per target-field work item (1..8)
 *   field_chunk      source nodes per target-field work item (16, 32 or 64)
 *   lu_rows_per_cta  tensor-core LU: a system of order N is factored by the
 *                    smallest power of two of CTAs, at most 8, that is
 *                    >= N / lu_rows_per_cta (128, 256 or 512)
 *   lu_early         tensor-core LU: the largest systems, at least this
 *                    percentage of them (0..50, whole assembly subgroups), are
 *                    assembled and factored on a second stream while the
 *                    others are assembled (0: one sequence).  Kernel timing
 *                    (fh_set_timing) runs the single sequence.
 *   contract_tc      mixed paths, 2J <= 512: 1 contracts u = [Vr | Vi][Gr ; Gm]
 *                    on the tensor cores (operands cut into eight 6-bit
 *                    slices held exactly in BF16, exact FP32 sums per slice
 *                    level, levels combined in double-float; ~2^-48 of
 *                    max|row| max|column| per term), 0 in double-float on the
 *                    FP32 pipe.  fh_sample and fh_synthesize (host pointers)
 *                    report a tensor-core completion wait that gave up as
 *                    FH_ETIMEOUT.
 * Defaults {8, 8, 64, 512, 0, 1}. */
typedef struct {
    int assemble_group;
    int field_group;
    int field_chunk;
    int lu_rows_per_cta;
    int lu_early;
    int contract_tc;
} fh_tuning;

fh_status fh_get_tuning(const fh_ctx *ctx, fh_tuning *out);

/* Applies t (FH_EINVAL for a value outside the sets above; nothing changes).
 * With a discretization present its work lists are rebuilt at once; densities,
 * spectra and target fields already computed stay valid. */
fh_status fh_set_tuning(fh_ctx *ctx, const fh_tuning *t);

/* Autotuner (schedule selection by measurement): after fh_discretize[_batch],
 * times each candidate of the assembly (assemble_group 2, 4, 8), the
 * tensor-core factorisation (lu_rows_per_cta 512, 256, 128, then lu_early 0,
 * 10, 20, 35 over assembly plus factorisation; mixed TF32/BF16 only) and the
 * target fields at the n_x targets x (host, 2 n_x interleaved;
 * field_group 2, 4, 8 x field_chunk 16, 32, 64; skipped when n_x == 0), each
 * as the fastest of `reps` (>= 1) runs on the context stream, one phase at a
 * time with the others at their current settings, and applies the fastest.
 * The runs overwrite the matrices, factors and target-field scratch but not
 * the densities: a solved context stays solved (densities from the previous
 * schedule), and target fields are recomputed by the next fh_sample.  Before
 * the first solve the densities are zeroed for the field runs.  chosen (may
 * be NULL) receives the applied tuning; ms (may be NULL) receives the best
 * time of each tuned stage {assembly, factorisation, target fields, assembly
 * plus factorisation with lu_early} in ms (0 for a stage not tuned).  Blocks
 * until done. */
fh_status fh_autotune(fh_ctx *ctx, const double *x, int n_x, int reps, fh_tuning *chosen,
                      double ms[4]);

/* enable != 0: bracket every kernel group with CUDA events on the context
 * stream (adds two event records per group).  Launch counts are always kept. */
fh_status fh_set_timing(fh_ctx *ctx, int enable);

/* Synchronise the context stream, fold pending event pairs into the totals,
 * copy them to *out, and zero them if reset != 0. */
fh_status fh_get_timings(fh_ctx *ctx, fh_timings *out, int reset);

/* The kernels' Bessel routine on n host arguments x > 0 (current device):
 * out[6i .. 6i+5] = J0, Y0, J1, Y1 from the joint routine used in assembly,
 * then J0, Y0 from the H0 routine used for target fields.  Diagnostic entry
 * point for checking the Hankel kernels of Sec. 2.3 against reference values;
 * allocates its own device scratch. */
fh_status fh_eval_bessel(const double *x, int n, double *out);

/* J0, Y0, J1, Y1 at host points x[0..n-1] through the double-float
 * (FP32-pair) Hankel form used by the mixed-precision kernels for x >= 8
 * (Sec. 2.3 kernels; Hankel's asymptotic form with binary32 remainder
 * polynomials); x < 8 uses the FP64 series.  out[4i .. 4i+3] (host,
 * caller-owned).  Diagnostic entry point; allocates its own device scratch.
 * Errors: FH_EINVAL (NULL pointers, n < 0), FH_ENOMEM, FH_ECUDA. */
fh_status fh_eval_bessel_df(const double *x, int n, double *out);

/* Tensor-core (tcgen05) check: C = A B^T for host FP32 arrays A (M x K) and
 * B (N x K), row-major, with the operands taken as BF16 (kind = 1, rounded to
 * nearest) or TF32 (kind = 2) and FP32 accumulation in tensor memory; C is
 * M x N row-major.  M % 128 == 0, N % 256 == 0, K % 64 == 0.  Diagnostic for
 * the tensor-core building blocks used by the solver; allocates its own
 * device buffers.  FH_ETIMEOUT if an MMA completion wait gave up. */
fh_status fh_tc_gemm_test(int kind, int M, int N, int K, const float *A, const float *B,
                          float *C);

/* Measured FMA throughput of device `device` in TFLOP/s (2 flops per FMA):
 * fp64 != 0 for binary64, else binary32; `iters` FMAs per chain (e.g. 4096).
 * Not part of the scattering path: it gives the arithmetic roofline against
 * which the ALU-bound kernels are reported. */
fh_status fh_probe_fma_peak(int device, int fp64, int iters, double *tflops);

/* Measured dense tensor-core throughput of device `device` in TFLOP/s: one
 * CTA per SM issues `iters` (>= 2) back-to-back tcgen05 MMAs of 128 x 256
 * outputs and one K step from operands resident in shared memory, FP32
 * accumulation in tensor memory; kind 1 = BF16 operands (kind::f16), 2 = TF32
 * (kind::tf32).  Best of two timed runs.  Not part of the scattering path: it
 * is the peak against which the tensor-core LU and contraction are reported.
 * FH_ETIMEOUT if the bounded completion wait gave up. */
fh_status fh_probe_mma_peak(int device, int kind, int iters, double *tflops);

#ifdef __cplusplus
}
#endif
#endif /* FH_H */

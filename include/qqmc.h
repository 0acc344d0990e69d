/*
 * qqmc.h -- C ABI of the GB300 quantum quasi-Monte Carlo (QQMC) library.
 *
 * The library evaluates order-n perturbative coefficients of the Anderson
 * single-level dot at T = 0 -- the charge Q_n (wide-band or semicircular
 * leads) and the current I_n (semicircular leads under a symmetric bias) --
 * by the QQMC method: digitally shifted Sobol' points are warped through the product
 * model function p_n(u) = prod_i exp(-(u_{i-1}-u_i)/tau) into ordered vertex
 * times t = u_0 > u_1 > ... > u_n > 0, the Keldysh integrand (sum over the
 * 2^n Keldysh index vectors of det M_up * det M_down) is evaluated there, and
 * the weighted values are reduced per shifted sequence into Q_n and its
 * shift-to-shift error bar.
 *
 * Conventions shared by every call:
 *  - Green functions: g^<(tau), g^>(tau) of the dot with g^<(0) = i<n>;
 *    tables hold L nodes tau_k = -t_max + k * 2 t_max / (L-1), k = 0..L-1,
 *    as interleaved (re, im) doubles, linearly interpolated in re and im.
 *  - Integrand c_n(u) = i^n sum_a (-1)^{|a|} det M_up(a) det M_down(a),
 *    paper App. E Eq. (integral_gf) over the ordered simplex (the 1/n! of the
 *    cube form is absorbed by ordering the vertices).
 *  - Charge readout Q_n = -2i * (1/N) sum_i w_i c_n(u_i), paper Eq.
 *    (warped_int2) with w = C/p_n, C = tau^n; points with u_n <= 0 add 0.
 *  - Current (App. E, measurement column on lead site 1): the column of
 *    M_up holds gamma g^<_01(u_k - t) (a_k = 0) or gamma g^>_01 (a_k = 1),
 *    and I_n = -4 Re (1/N) sum_i w_i c_n(u_i): the current from the dot into
 *    the lead at -V/2, both spins, e = hbar = 1 (per spin -2 gamma Im<c_0^+ c_1>).
 *  - Error bar: sample standard deviation over the K shifted sequences
 *    (ddof = 1) divided by sqrt(K), paper App. G and App. H.
 *  - Sobol' points in Gray-code order, X_i = XOR of the direction words
 *    selected by the bits of gray(i); shifted by XOR with one 32-bit word per
 *    dimension; x = X * 2^-32.  Dimension m-1 drives the gap v_m.
 *  - Shift words, when not given, are the high 32 bits of
 *    splitmix64(seed XOR (k * 65536 + d)) for shift k and dimension d.
 *
 * Memory and errors: every pointer argument is HOST memory unless its
 * description says device.  The library allocates its own device memory
 * (tables, shift words, partial sums) and frees it in the matching destroy
 * call.  Calls return QQMC_OK (0) or a negative QQMC_E_* code; no call
 * throws, aborts or exits.  qqmc_last_error() describes the last failure of
 * the calling thread.  Objects may be used from several threads, but one
 * problem or plan must not be used by two threads at once; a server is
 * fully thread-safe.
 */
#ifndef QQMC_H
#define QQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QQMC_OK 0
#define QQMC_PENDING 1
#define QQMC_RUNNING 2
#define QQMC_E_INVAL (-1)     /* malformed argument */
#define QQMC_E_RANGE (-2)     /* order outside 1..QQMC_MAX_ORDER */
#define QQMC_E_NOMEM (-3)     /* device or host allocation failed */
#define QQMC_E_CUDA (-4)      /* CUDA runtime error (no device, launch failure) */
#define QQMC_E_BUSY (-5)      /* server queue full */
#define QQMC_E_TIMEOUT (-6)   /* request or wait exceeded its limit */
#define QQMC_E_CANCELLED (-7) /* request cancelled before completion */
#define QQMC_E_NOTFOUND (-8)  /* unknown handle */
#define QQMC_E_NONFINITE (-9) /* an integrand sum came out NaN or infinite (results still filled) */

#define QQMC_MAX_ORDER 22
#define QQMC_MAX_POINTS_LOG2 30 /* N <= 2^30 points per shifted sequence */

/* Observable (qqmc_params.observable). */
#define QQMC_OBS_CHARGE 0  /* Q: G^<_00(t,t) */
#define QQMC_OBS_CURRENT 1 /* I: G^<_01(t,t), needs half_bandwidth > 0 */

/* Arithmetic of the determinant stage. */
#define QQMC_PREC_FP64 0  /* tables, Schur updates and sums in FP64 */
#define QQMC_PREC_MIXED 1 /* tables and Schur updates in FP32; leaf sums and a
                             work unit's 32 weighted point values as two-sum
                             float-float pairs (48 bits); weights, sums over
                             units and shift sums in FP64 two-sum */

/* Elimination order of the Keldysh sum (qqmc_set_elimination).  Every vertex
 * diagonal of M_down is g^<(0) - i alpha (App. E), which is zero at the
 * Hartree-cancelling alpha = Im g^<(0); at particle-hole symmetry every odd
 * leading minor of M_down then vanishes too.
 *   QQMC_ELIM_SINGLE  one vertex per tree level, 1x1 pivots (the fastest; its
 *                     pivots are ratios of consecutive leading minors);
 *   QQMC_ELIM_PAIRS   vertex pairs (1,2), (3,4), ... with 2x2 block pivots
 *                     (the even leading minors) and a lone last vertex without
 *                     a reciprocal: exact where the vertex diagonal vanishes,
 *                     about 10 % (FP64) to 30 % (mixed) more work;
 *   QQMC_ELIM_AUTO    (default) pairs when |g^<(0) - i alpha| is below 0.01
 *                     (FP64) or 0.25 (mixed) of max(|g^<(0)|, |g^>(0)|), with
 *                     g^>(0) = g^<(0) - i; the single-vertex tree otherwise. */
#define QQMC_ELIM_AUTO 0
#define QQMC_ELIM_PAIRS 1
#define QQMC_ELIM_SINGLE 2

/* Physical problem and warp (paper: App. E model, App. F exponential h). */
typedef struct qqmc_params {
    double gamma;       /* tunnelling rate Gamma at the Fermi level (Lorentzian half-width), > 0 */
    double eps_d;       /* level E_d of the non-interacting dot (App. E: eps_d = E_d - alpha U) */
    double t_max;       /* measurement time t = u_0; tables cover [-t_max, t_max]; > 0 */
    double tau;         /* model-function decay: h(v) = exp(-v / tau), > 0 */
    int32_t n_table;    /* L, number of table nodes; even, 4 <= L <= 2^20 */
    int32_t observable; /* QQMC_OBS_CHARGE or QQMC_OBS_CURRENT */
    uint64_t seed;      /* digital-shift seed (used when no shift words are given) */
    double alpha;       /* quadratic shift of the interaction, U (n_up - alpha)(n_dn - alpha) (App. E):
                           the diagonal of every Wick determinant becomes g^<(0) - i alpha, except the
                           entry of the measurement pair; 0 for the plain expansion */
    double half_bandwidth; /* D of the semicircular lead density of states (App. E); 0 = wide band
                              (Delta = -i Gamma).  D > 0 needs |eps_d| + gamma < D. */
    double bias;        /* symmetric bias V >= 0: lead L at +V/2, lead R (holding site 1) at -V/2;
                           V > 0 needs D > 0 */
} qqmc_params;

typedef struct qqmc_problem qqmc_problem;

/*
 * Build a problem: the Green-function tables are computed on the device and
 * kept resident in device memory.
 *  - half_bandwidth = 0 (wide band, V = 0): g^<, g^> by the App. E
 *    contour-deformed Fourier integral (vertical ray into the half plane
 *    where e^{-i w tau} decays, plus the real segment up to the Fermi level;
 *    composite Gauss-Legendre), g^> from the exact sum rule
 *    g^> - g^< = -i exp(-i eps_d tau - Gamma |tau|); g^<(0) = i<n> in closed form.
 *  - half_bandwidth = D > 0 (semicircular leads, App. E, bias V): g^<_00,
 *    g^>_00 and, for the current, gamma g^<_01, gamma g^>_01 from their
 *    spectral forms (Eq. (lesser_greater_freq); textbook normalisation
 *    g^< = i A f) by composite Gauss-Legendre in w = D sin(theta), split at
 *    the Fermi steps +-V/2; the equal-time values from the same quadrature.
 * *out is owned by the caller until qqmc_destroy_problem.
 * Errors: E_INVAL (bad params), E_NOMEM, E_CUDA.
 */
int qqmc_create_problem(const qqmc_params *p, qqmc_problem **out);

/*
 * Build a problem from caller tables (any Green function known on the mesh,
 * paper App. E: the integrand is defined once g is known in time).
 * g_lesser, g_greater: 2*L doubles each (interleaved complex) on the nodes
 * above; only the nodes with tau > 0 and the node next to 0 are read (the
 * tables are assumed to obey g(-tau) = -conj g(tau)).  g0 = g^<(0), used on
 * the diagonal of every Wick determinant.  Copied; the caller keeps its
 * buffers.  Errors: E_INVAL, E_NOMEM, E_CUDA.
 */
int qqmc_create_problem_tables(const qqmc_params *p, const double *g_lesser, const double *g_greater,
                               double g0_re, double g0_im, qqmc_problem **out);

/*
 * Switch a problem to the current observable with caller dot-lead tables:
 * cl = gamma g^<_01, cg = gamma g^>_01, 2*L doubles each (interleaved
 * complex) on the problem's mesh; only the nodes k = 0 .. L/2 (tau <= h/2)
 * are read, since the column entries sit at tau = u_k - t < 0.
 * c0 = gamma g^<_01(0) (the measurement pair; it cancels from every order
 * n >= 1 and gives I_0 = -4 Re c0).  Copied.  Errors: E_INVAL, E_NOMEM, E_CUDA.
 */
int qqmc_set_current_tables(qqmc_problem *pr, const double *cl, const double *cg, double c0_re, double c0_im);

/* Copy a current problem's dot-lead tables to host: nodes k = 0 .. L/2 only,
 * (L/2 + 1) complex values each; c0 (optional) = gamma g^<_01(0).
 * E_INVAL for a charge problem. */
int qqmc_problem_current_tables(const qqmc_problem *pr, double *cl, double *cg, double *c0);

/* Free a problem and its device memory.  NULL is accepted. */
int qqmc_destroy_problem(qqmc_problem *pr);

/* Copy the problem's tables to host: 2*L doubles each, full [-t_max, t_max]
 * mesh (negative nodes filled by g(-tau) = -conj g(tau)). */
int qqmc_problem_tables(const qqmc_problem *pr, double *g_lesser, double *g_greater, double *g0);

/*
 * Rank-1 lattice point set (the lattice rules the paper cites as the other
 * randomised low-discrepancy family) instead of Sobol': N = 2^log2_n points
 * x_i = frac(i z / N + Delta), z = generating vector (dims odd components),
 * Delta the random shift.  Points are 32-bit fixed point like the Sobol'
 * words: word_d = ((i z_d mod N) << (32 - log2_n)) + S_d mod 2^32, with the
 * shift words S (caller or seed, as for Sobol') added instead of XORed.
 * Every later integration on the problem uses the lattice; items must stay
 * inside it (order <= dims, first_index + n_points <= N; E_INVAL otherwise).
 * bakers != 0 applies the baker's (tent) transform x -> 1 - |2x - 1| after the
 * shift (measure preserving; lets the lattice integrate non-periodic
 * integrands at its higher rate; the word 2^31 maps to 1 - 2^-32).
 * z = NULL restores Sobol'.  Errors: E_INVAL, E_NOMEM, E_CUDA.
 */
int qqmc_set_lattice(qqmc_problem *pr, int log2_n, const uint32_t *z, int dims, int bakers);

/*
 * Where the Schur-tree stack of the determinant kernel lives: from order
 * min_order on (per precision) its wide top levels (matrices of more than
 * S_g rows, 14 <= S_g <= 20 chosen so that an SM holds up to 9 FP64 or 12
 * mixed-precision warps) and the chunk's point times move from shared memory to a per-warp
 * slice of device memory allocated with each plan, so that high orders keep
 * more warps per SM.  Orders whose stack does not fit in shared memory at all
 * always split it.  min_order > QQMC_MAX_ORDER: only those; min_order <= 0:
 * the built-in default (FP64: 5, mixed: 11).  Process-wide; set
 * before creating plans.  Errors: E_INVAL.
 */
int qqmc_set_stack_policy(int precision, int min_order);

/* Elimination order of a problem's Keldysh sums (QQMC_ELIM_*, see above);
 * applies to plans and calls made afterwards.  Errors: E_INVAL. */
int qqmc_set_elimination(qqmc_problem *pr, int mode);
/* The order a problem's sums use at the given precision: QQMC_ELIM_PAIRS or
 * QQMC_ELIM_SINGLE (QQMC_ELIM_AUTO resolved), or a negative error code. */
int qqmc_elimination(const qqmc_problem *pr, int precision);

/*
 * Component-by-component construction of a generating vector for N = 2^log2_n
 * (3 <= log2_n <= 24): z_1 = 1, then each z_d the odd number <= N/2 minimising
 * the shift-averaged worst-case error e^2 = -1 + (1/N) sum_k prod_d
 * (1 + gamma_d 2 pi^2 B_2({k z_d / N})) (weighted Korobov space of smoothness 2,
 * product weights gamma[0..dims-1] > 0), ties to the smallest z.  Host only,
 * O(N log N) per component (FFT over the group of odd residues mod 2^m).
 */
int qqmc_lattice_cbc(int log2_n, int dims, const double *gamma, uint32_t *z);

/*
 * Learned warp (paper App. F, "learning h from the integrand"): a second
 * change of variables w -> x on top of the exponential one, with
 * w_m = 1 - exp(-v_m / tau) in [0, 1).  Per dimension m the density of w_m is
 * piecewise constant on `cells` equal cells; cdf (host [order][cells + 1],
 * cdf[m][0] = 0, cdf[m][cells] = 1, non-decreasing) is its cumulative
 * distribution.  A Sobol' coordinate x is mapped to w by inverting the CDF and
 * the point weight gains prod_m dw_m/dx_m.  Installed per (problem, order):
 * every later integration of that order on the problem uses it (plans capture
 * it at creation).  cdf = NULL or cells <= 0 restores the plain warp.
 */
int qqmc_set_projection(qqmc_problem *pr, int order, const double *cdf, int cells);

/*
 * Learn and install the warp above from M integrand samples: the first M
 * Sobol' points shifted by the words of shift index 65535 of the problem's
 * seed, plain exponential warp; |w c_n(u)| of the in-domain points (FP64,
 * device) is binned in each w_m into n_bins bins (the projection of the
 * integrand onto dimension m), smoothed with the Gaussian kernel
 * exp(-(w - w')^2 / lambda^2) onto the cells, floored at floor_frac times its
 * maximum (every region keeps a sampling density), and accumulated into the
 * CDF.  cdf_out (optional, host [order][cells + 1]) receives the table.
 * The paper uses N_b = 100..250 bins, M = 2e4..1e5, lambda = 0.05.
 */
int qqmc_learn_projection(qqmc_problem *pr, int order, uint64_t M, int n_bins, double lambda, double floor_frac,
                          int cells, double *cdf_out);

/* Result of one order-n integration. */
typedef struct qqmc_result {
    int32_t order;
    int32_t n_shifts;          /* K */
    uint64_t n_points;         /* N per shifted sequence */
    double q_mean;             /* mean over shifts of Q_n^(k) (current: I_n^(k)) */
    double q_err;              /* std_{ddof=1} over shifts / sqrt(K) (0 if K == 1) */
    double q_imag_absmax;      /* charge: max_k |Im Q_n^(k)| (zero in exact arithmetic);
                                  current: max_k |-4 Im S_k / N| (not a check) */
    uint64_t n_in_domain;      /* points with u_n > 0, summed over shifts */
    double device_ms;          /* device time of the launch that produced it */
    uint64_t n_nonfinite;      /* work units whose partial sum was NaN or infinite (0 when valid);
                                  any nonzero count makes the call return QQMC_E_NONFINITE */
} qqmc_result;

/*
 * One order-n integration (paper App. B main loop, Eq. (warped_int2)),
 * blocking.  order in 1..QQMC_MAX_ORDER (else E_RANGE); 1 <= n_points <=
 * 2^QQMC_MAX_POINTS_LOG2, 1 <= n_shifts <= 1024 (else E_INVAL).
 * shift_words: host [n_shifts][order] uint32 or NULL (then from the seed).
 * per_shift: host [n_shifts][2] doubles or NULL; receives
 *   S_k = (1/N) sum_i w_i c_n(u_i) (complex), so Q_n^(k) = -2i S_k.
 * precision: QQMC_PREC_FP64 or QQMC_PREC_MIXED.
 */
int qqmc_integrate(qqmc_problem *pr, int order, uint64_t n_points, int n_shifts, int precision,
                   const uint32_t *shift_words, double *per_shift, qqmc_result *out);

/* One work item of a batched launch: an order-n integration of a problem. */
typedef struct qqmc_item {
    qqmc_problem *problem;
    int32_t order;
    int32_t n_shifts;
    uint64_t n_points;
    uint64_t first_index;         /* first Sobol' index (0 normally; resume point otherwise) */
    const uint32_t *shift_words;  /* host [n_shifts][order] or NULL (from the problem seed) */
} qqmc_item;

typedef struct qqmc_plan qqmc_plan;

/*
 * Batched, device-resident execution.  qqmc_plan_create uploads the items'
 * shift words and allocates the partial-sum buffers and, where the stack
 * policy in force at creation splits the Schur-tree stack, its device-memory
 * part (the problems must outlive the plan).  Items with few chunks of 32
 * points are cut into finer work units -- a chunk's points into groups, then
 * each point's Keldysh tree into subtrees -- until an item has about 16384
 * units; the cut depends on the item alone.  qqmc_plan_launch enqueues the
 * whole batch -- one persistent launch per tuned flat depth (uneven orders
 * and point counts share it), one for the orders tuned to one point per
 * lane, and one reduction kernel -- on `stream` (a cudaStream_t, or NULL for
 * the legacy default stream) and returns without waiting; with use_graph !=
 * 0 the launches are captured once into a CUDA graph and replayed.
 * qqmc_plan_results waits for the last launch and copies per-item results
 * (results: [n_items]; per_shift: concatenated [sum_k n_shifts][2] S_k, or
 * NULL).
 */
int qqmc_plan_create(const qqmc_item *items, int n_items, int precision, qqmc_plan **out);
int qqmc_plan_launch(qqmc_plan *plan, void *stream, int use_graph);
int qqmc_plan_results(qqmc_plan *plan, qqmc_result *results, double *per_shift);
int qqmc_plan_destroy(qqmc_plan *plan);
/* Kernel launches a plan issues per qqmc_plan_launch (for launch accounting). */
int qqmc_plan_kernel_count(const qqmc_plan *plan);
/* Device time of the last launch, after qqmc_plan_results: the determinant
 * kernel alone (events on the launch stream around it; 0 when the launch was a
 * graph replay) and the whole launch. */
int qqmc_plan_timing(const qqmc_plan *plan, double *kernel_ms, double *total_ms);
/* Execution span of the last launch on the device clock (%globaltimer, ns):
 * the earliest start and the latest exit of any warp of its determinant
 * launches.  Spans of plans launched on different streams can be compared to
 * see whether their kernels ran at the same time.  Waits for the launch. */
int qqmc_plan_device_span(const qqmc_plan *plan, uint64_t *start_ns, uint64_t *end_ns);

/*
 * Partial sums of single chunks of the last launch (after qqmc_plan_results):
 * for item `item` (caller order), shifted sequence `shift` and chunks
 * chunk[0..count-1] (chunk c holds Sobol' indices first_index + 32c ..
 * first_index + 32c + 31 of that sequence), out[4*q..4*q+3] = (sum.re,
 * sum.im, compensation.re, compensation.im) of w_i c_n(u_i) over the chunk's
 * in-domain points: the sum of the partials of the chunk's work units
 * (point groups and subtrees, in unit order).  For checking a full-size
 * launch point by point against a reference.  E_INVAL on bad indices.
 */
int qqmc_plan_chunk_sums(const qqmc_plan *plan, int item, int shift, const int64_t *chunk, int count, double *out);

/*
 * Tuning of the determinant kernel (the autotuner writes these): for
 * each order, the number of warps per block and the number of vertices
 * resolved per lane in the flat (per-lane) phase, 2..5 (the levels between
 * the depth-first tree leaf, 5 vertices, and the flat phase are expanded
 * breadth first), or 1 for one point per lane (orders <= 4: each lane runs
 * the whole Keldysh sum of its own point).  Values <= 0 restore the built-in defaults.  Applies to
 * plans created afterwards; in a plan every item runs with its own order's
 * flat depth, and the items of one flat depth share a launch with the warps
 * per block of their highest order.  Each elimination order has its own table:
 * precision | QQMC_TUNE_PAIRS addresses the pair-block tree's (its flat depth
 * counts vertices resolved per lane as well; with vertex pairs a lane takes
 * flat_vertices or one fewer).
 */
#define QQMC_TUNE_PAIRS 16
int qqmc_set_tuning(int precision, int order, int warps_per_block, int flat_vertices);
int qqmc_get_tuning(int precision, int order, int *warps_per_block, int *flat_vertices);

/*
 * Allocation-free integration (the paper has no counterpart; this is a
 * deployment convenience).  Same computation as qqmc_integrate, for callers
 * that cannot allocate device memory where they integrate -- e.g. a host
 * framework whose own memory pool owns the device, or a real-time loop that
 * must not enter the driver's allocator.  All scratch (work counter, chunk
 * partial sums, item descriptor) lives in one 16 MiB static device array
 * inside the library, which every GPU that loads the library holds until
 * the process exits; no cudaMalloc/cudaFree or allocating routine is called.
 *   d_shift_words: DEVICE [n_shifts][order] uint32 (caller-owned);
 *   d_sums: DEVICE [n_shifts][2] doubles, receives sum_i w_i c_n(u_i) per
 *           shift, NOT divided by N (Q_n^(k) = -2i d_sums[k] / N);
 *   d_counts: DEVICE [n_shifts] uint64 in-domain counts, or NULL;
 *   stream: cudaStream_t or NULL.  The call only enqueues work (the item
 *   descriptor travels as a kernel argument; no host buffer is read after the
 *   call returns); the outputs are ready when the stream reaches that point.
 *   NaN or infinite integrand values show up in d_sums; there is no
 *   QQMC_E_NONFINITE here, since the call does not wait for the device.
 * The current device must be the problem's (E_INVAL otherwise).
 * Limits (E_INVAL beyond): n_shifts * ceil(n_points / 32) <= 465792; the
 * whole Schur-tree stack in shared memory (every order up to
 * QQMC_MAX_ORDER fits, one warp per block at the highest FP64 orders; a
 * stack that did not fit would be refused).  No work-unit cut: one unit per
 * chunk, so orders with few chunks, and those from the stack-policy order
 * up, can run slower than in qqmc_integrate.
 * The first call on a device resolves the array's device address and uploads
 * the kernels' constant tables; make that first call before any stream
 * capture.  Every call shares the array and leaves its contents behind (the
 * work counter is cleared at the start of each call), so calls whose work
 * overlaps on the GPU -- on different streams, or from different threads --
 * race and must be serialised by the caller.
 */
int qqmc_integrate_noalloc(const qqmc_problem *pr, int order, uint64_t n_points, int n_shifts, int precision,
                           const uint32_t *d_shift_words, double *d_sums, unsigned long long *d_counts,
                           void *stream);

/* ---------------------------- inspection calls ---------------------------- */

/* Sobol' direction words of the product generator (Joe-Kuo primitive
 * polynomials and initial values, standard recurrence): out [n_dims][32]. */
int qqmc_direction_numbers(int n_dims, uint32_t *out);

/* Shift words derived from a seed: out [n_shifts][n_dims] (splitmix64 rule above). */
int qqmc_shift_words(uint64_t seed, int n_shifts, int n_dims, uint32_t *out);

/* Shifted Sobol' integers Y_i = X_i XOR shift computed on the device for
 * indices first_index .. first_index+count-1: out [count][order] (host).
 * shift: host [order] or NULL (zero shift). */
int qqmc_sobol_points(int order, uint64_t first_index, uint64_t count, const uint32_t *shift, uint32_t *out);

/* Warped points on the device: u [count][order], weight C/p_n [count],
 * inside [count] (1 iff u_n > 0), for the problem's t_max and tau. */
int qqmc_warp_points(const qqmc_problem *pr, int order, uint64_t first_index, uint64_t count,
                     const uint32_t *shift, double *u, double *w, int32_t *inside);

/* Integrand c_n(u) at caller points u [count][order] (host, strictly
 * decreasing within t_max > u_1 > ... > u_n > 0), evaluated by the same
 * device code as the integration: out [count][2] (complex). */
int qqmc_integrand(const qqmc_problem *pr, int order, uint64_t count, const double *u, int precision,
                   double *out);

/*
 * Conformal resummation of a truncated perturbation series F(U) =
 * sum_{n=0}^{N} a_n U^n beyond its radius of convergence, paper App. H
 * (parabola transform W = -tan^2(sqrt(U/p)) with a real negative parameter
 * p; for U >= 0 this is W = tanh^2(sqrt(U/|p|)) in [0, 1)).  The series is
 * re-expanded in powers of W through U(W) = |p| artanh^2(sqrt W), truncated at
 * W^N and evaluated at W(U).  invert != 0 resums 1/F (a_0 != 0) and returns
 * the reciprocal.  a_err (optional, host [N+1]): standard errors of the a_n,
 * propagated linearly into *err; *tail (optional) = |b_N W^N|, the size of
 * the last re-expanded term, a truncation estimate.  Host-only, no device.
 * Errors: E_INVAL (N outside 0..QQMC_MAX_ORDER, p >= 0, U < 0, a_0 = 0 with
 * invert).
 */
int qqmc_resum_parabola(const double *a, const double *a_err, int n, double p, double U, int invert, double *value,
                        double *err, double *tail);

/* ------------------------------- serving ---------------------------------- */

typedef struct qqmc_server qqmc_server;

typedef struct qqmc_server_opts {
    uint64_t device_memory_limit; /* bytes the server may hold on the device (0: 4 GiB) */
    int32_t max_queue;            /* pending requests before E_BUSY (0: 4096) */
    int32_t max_batch_items;      /* items per persistent launch (0: 256) */
    int32_t precision;            /* QQMC_PREC_* used for every request */
    int32_t use_graph;            /* capture each batch launch in a CUDA graph */
    double request_timeout_s;     /* 0: none */
} qqmc_server_opts;

/* A request: Q_1..Q_{n_max} (or I_1..I_{n_max} when params.observable is the
 * current) of one dot (paper App. H parameter sweep). */
typedef struct qqmc_request {
    qqmc_params params;
    int32_t n_max;      /* 1..QQMC_MAX_ORDER */
    int32_t n_shifts;   /* K >= 2 */
    uint64_t n_points;  /* N per shift */
    double U;           /* interaction for the truncated series sum_n Q_n U^n */
} qqmc_request;

typedef struct qqmc_series {
    int32_t n_max;
    int32_t status;                    /* QQMC_OK or an error code */
    double q[QQMC_MAX_ORDER + 1];      /* q[0] = Q_0 = -2i g^<(0) (current: I_0 = -4 Re gamma g^<_01(0));
                                          q[n] = Q_n (I_n) */
    double q_err[QQMC_MAX_ORDER + 1];
    double series_sum;                 /* sum_{n <= n_max} Q_n U^n (truncated, not resummed) */
    double latency_ms;                 /* submit -> completion */
    double queue_ms;                   /* submit -> admission */
    uint64_t n_in_domain;
    uint64_t batch;                    /* admission round that carried the request (1, 2, ...) */
    uint64_t device_start_ns;          /* execution span of that round's kernels on the device */
    uint64_t device_end_ns;            /*   clock (%globaltimer, ns); see qqmc_plan_device_span */
} qqmc_series;

int qqmc_server_create(const qqmc_server_opts *opts, qqmc_server **out);
/* Non-blocking.  E_BUSY when the pending queue is full. */
int qqmc_submit(qqmc_server *s, const qqmc_request *r, uint64_t *handle);
/* QQMC_PENDING, QQMC_OK (out filled; the handle is released) or an error code
 * (out->status set; the handle is released). */
int qqmc_poll(qqmc_server *s, uint64_t handle, qqmc_series *out);
/* Where a request stands, without releasing it: QQMC_PENDING (queued),
 * QQMC_RUNNING (admitted: its round is on the device), or its final status
 * (QQMC_OK or an error code) once done; E_NOTFOUND for an unknown handle. */
int qqmc_request_state(qqmc_server *s, uint64_t handle);
int qqmc_cancel(qqmc_server *s, uint64_t handle);
/* Waits for in-flight work, fails pending requests with E_CANCELLED, frees all. */
int qqmc_server_destroy(qqmc_server *s);

/*
 * Measured FMA throughput of the CUDA cores (the paper has no counterpart; it
 * is the denominator of the determinant kernels' roofline, which are bound by
 * the FP64 or FP32 FMA pipes).  A register-resident kernel runs independent
 * multiply-add chains on every resident warp of every SM; *tflops receives
 * 2 x FMAs / second of the last launch, each launch lasting about
 * seconds / 4 (0 < seconds <= 60).  precision: QQMC_PREC_FP64 (DFMA) or
 * QQMC_PREC_MIXED (FFMA).  Blocking.  Errors: E_INVAL, E_CUDA.
 */
int qqmc_fma_peak(int precision, double seconds, double *tflops);

/* Copy the calling thread's last error message (NUL-terminated, truncated). */
int qqmc_last_error(char *buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif /* QQMC_H */

/*
 * ewos.h -- C ABI of the B300 extended Walk-on-Spheres operator toolbox.
 *
 * The library builds, on one GPU, the Laplacian Operator Toolbox of the paper "Extended
 * Walk-on-Spheres Algorithm for Linear and Nonlinear Elliptic Problems of Divergence-type"
 * (the matrices A, B^(j), H, K^(j) of Sec. 2.3, eq. LOT, computed as in Algorithm 5) and
 * uses it to solve divergence-form Dirichlet problems (Sec. 3).
 *
 * Conventions used by every entry point:
 *   - G := A/2 and gradG := B/2, so that G is the inverse of -Laplace with zero boundary
 *     values (G 1 = (1-|x|^2)/(2d) on the unit ball).  H and gradH := K are the paper's.
 *   - d in {2, 3}; n interior nodes x_i (the W and V centres, m = n); p boundary nodes z_j;
 *     N walks per node; eps the width of the stopping shell.
 *   - Arrays are dense, row-major, double precision unless stated.  A pointer argument is
 *     host memory unless the argument's documentation or a flag says it is device memory.
 *   - The caller owns every input and output buffer.  The library owns a toolbox and its
 *     device memory until ewos_toolbox_free.
 *   - Every entry point returns an ewos_status; nothing aborts, traps or prints.  On an
 *     error the output arguments are left unspecified and ewos_last_error() holds a message.
 *   - All entry points run on one CUDA device (the current device at build time) and may be
 *     called from one host thread at a time per toolbox.
 */
#ifndef EWOS_API_H_
#define EWOS_API_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EWOS_OK = 0,
    EWOS_EINVAL = 1,      /* bad argument: sizes, a node outside the domain, NULL pointer   */
    EWOS_ENOMEM = 2,      /* device or host allocation failed                              */
    EWOS_ECUDA = 3,       /* a CUDA runtime call failed (message in ewos_last_error)       */
    EWOS_ESINGULAR = 4,   /* LU met an exactly zero pivot                                  */
    EWOS_ENOCONV = 5,     /* Newton / Picard / refinement did not reach the tolerance     */
    EWOS_ETIMEOUT = 6,    /* a bounded device-side wait gave up                            */
    EWOS_ESTEPCAP = 7,    /* warning: some walks hit max_steps (reported, results valid)   */
    EWOS_EIO = 8          /* a toolbox file could not be written or read, or is not one    */
} ewos_status;

typedef enum {
    EWOS_SDF_BALL = 0,    /* params: centre (d), radius                r = R - |x - c|     */
    EWOS_SDF_BOX = 1,     /* params: lo (d), hi (d)                    r = min_k min(x-lo, hi-x) */
    EWOS_SDF_POLYGON = 2  /* d = 2; params: vertices x0,y0,x1,y1,... (closed polygon, <= 256
                             vertices); r = distance to the nearest edge, signed by an
                             even-odd inside test (an approximate distance, Rem. 2.14 (i)) */
} ewos_sdf_kind;

/* Distance to the boundary r(x) of eq. (r), Sec. 2.1. */
typedef struct {
    int kind;                 /* ewos_sdf_kind */
    int dim;                  /* 2 or 3 */
    const double* params;     /* host */
    int64_t nparams;
} ewos_domain;

typedef struct {
    int precision;            /* 32 (FP32 walks, default) or 64 (FP64 walks)                 */
    int64_t max_steps;        /* cap on work steps per walk; 0 -> 10000                      */
    void* stream;             /* cudaStream_t to run on; NULL -> the legacy default stream   */
    const double* cell_weights; /* optional host n-vector lambda_i; NULL -> Monte Carlo      */
    int64_t cell_samples;     /* Monte Carlo samples for lambda_i; 0 -> 10^7                 */
    int threads_per_block;    /* walk kernel block size; 0 -> autotuned/default             */
    int ctas_per_sm;          /* walk kernel CTAs per SM; 0 -> as many as fit               */
    int hash_in_smem;         /* -1 auto, 0 keep the Voronoi lookup in global memory, 1 SMEM */
    int record_walks;         /* 1 -> keep per-walk records (exit cell, steps, G mass)      */
    uint32_t instance;        /* Philox instance word (separates independent builds)         */
    int inputs_on_device;     /* 1 -> x and z are device pointers                            */
    double lookup_grid_scale; /* Voronoi grid spacing in units of (volume/n)^(1/d); 0 -> autotuned */
    const double* v_nodes;    /* V-centres y [m][d] of the source partition (Sec. 2.3: the
                                 paper's V-cells, a partition independent of the W-cells of the
                                 nodes x); NULL -> y = x, m = n.  Host or device per
                                 inputs_on_device.  Rows stay indexed by x (n), columns of G and
                                 grad G by y (m); the solve's unknown s has m entries.        */
    int64_t m;                /* number of V-centres when v_nodes is set                     */
    int walk_kernel;          /* 0 -> autotuned; 1 -> the row's G and grad G accumulators in
                                 global memory (one 16-byte L2 reduction per walk point;
                                 16 m bytes per CTA of device memory during the build, 32 m
                                 for FP64 walks);
                                 2 -> the accumulators in shared memory (one atomic per value) */
} ewos_build_opts;

typedef struct {
    int64_t walks;            /* n * N                                                       */
    int64_t steps;            /* WoS steps: 1 (first step) + work steps, summed over walks   */
    int64_t capped;           /* walks that hit max_steps                                    */
    double ms_total;          /* device time of the whole build (events on the stream)       */
    double ms_walk;           /* device time of the walk kernel alone                       */
    double ms_lookup;         /* Voronoi lookup structures                                   */
    double ms_cells;          /* lambda_i Monte Carlo                                        */
    int threads_per_block, ctas_per_sm, grid, hash_in_smem;
    int64_t smem_bytes;
    double lookup_grid_scale; /* V grid spacing used                                            */
    int lookup_candidates;    /* fixed candidate slots per V grid cell (0: variable lists)      */
    int walk_kernel;          /* walk kernel used: 1 accumulators in global memory, 2 in
                                 shared memory                                                  */
} ewos_build_report;

typedef struct ewos_toolbox ewos_toolbox;

/*
 * Build the toolbox (Algorithm 5 with eqs. Estimator_A, Estimator_B, Estimator_H,
 * Estimator_K; samplers of Prop. 2.6; Voronoi binning of Sec. 2.3).
 *   x: n x d interior nodes (walk starts, and V centres), all with r(x_i) > 0.
 *   z: p x d boundary nodes (Gamma centres).
 *   walks: N >= 1 per node; eps > 0; seed: Philox key.
 *   opts may be NULL (defaults).  *out receives the toolbox.
 * Random numbers: Philox4x32-10, key (seed_lo, seed_hi), counter (walk, step, node,
 * tag<<24 | instance<<8 | slot); step k >= 0 (k = 0 at x_i) d = 2 slot 0 = (radius of Y,
 * angle of Y, angle of U, -), d = 3 slot 0 = (median uniforms x3, z of Y), slot 1 = (phi of Y,
 * z of U, phi of U, -); ball term: step word 0xFFFFFFFF, slot 0 = (S, angle or z, phi, -).
 * The CPU oracle of the repository replays the same stream.
 * Returns EWOS_ESTEPCAP (with a valid toolbox) when walks were capped.
 */
ewos_status ewos_toolbox_build(const ewos_domain* domain, const double* x, int64_t n,
                               const double* z, int64_t p, int64_t walks, double eps,
                               uint64_t seed, const ewos_build_opts* opts, ewos_toolbox** out);

/*
 * Build without allocating (no counterpart in the paper).  For callers that cannot call
 * cudaMalloc -- code under an allocator that owns all device memory (a framework's caching
 * pool, a serving process with a fixed memory budget) or code that must not allocate while
 * other work is in flight.  FP32 walks, the same kernels and random numbers as
 * ewos_toolbox_build; cell weights are not computed.
 *   x [n][d], z [p][d]: device pointers (double).  Outputs, caller-owned device buffers:
 *   P [(d+1)][n][n] float = [d_1 G, .., d_d G, G], KH [(d+1)][n][p] float = [d_1 H, .., H],
 *   Hc [n][p] uint32 exit counts.  rep may be NULL.  max_steps <= 0 -> 10000.
 * Temporaries live in one static 4 MiB device array per GPU that loads the library (held
 * until the process exits); a build whose node arrays or lookup grids need more is rejected
 * with EWOS_EINVAL and a message (ewos_last_error) before any walk runs (the square workload
 * with n = 4096, p = 512 needs about 0.6 MiB).  The call waits on `stream` (it reads the node
 * check, the lookup sizes and the step counts back) and returns when the build is done.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  Every call shares
 * the array and clears the counters it needs; calls whose work overlaps on the GPU race on
 * the array and must not be issued concurrently (same or different streams).
 */
ewos_status ewos_toolbox_build_noalloc(const ewos_domain* domain, const double* x, int64_t n,
                                       const double* z, int64_t p, int64_t walks, double eps,
                                       uint64_t seed, int64_t max_steps, void* stream, float* P,
                                       float* KH, uint32_t* Hc, ewos_build_report* rep);

/* Build a toolbox from matrices the caller already has (e.g. a toolbox saved earlier):
 * G [n][m], gradG [d][n][m], H [n][p] (frequencies), gradH [d][n][p], lambda [n], host
 * doubles; x [n][d], z [p][d].  precision 32 stores them as FP32 like a built toolbox. */
ewos_status ewos_toolbox_from_host(int dim, int64_t n, int64_t p, const double* x, const double* z,
                                   const double* G, const double* gradG, const double* H,
                                   const double* gradH, const double* lambda, int precision,
                                   void* stream, ewos_toolbox** out);

typedef enum {
    EWOS_G = 0,          /* [n][m]       G = A/2                (double)                    */
    EWOS_GRAD_G = 1,     /* [d][n][m]    gradG = B/2            (double)                    */
    EWOS_H = 2,          /* [n][p]       H = counts / N         (double)                    */
    EWOS_GRAD_H = 3,     /* [d][n][p]    gradH = K              (double)                    */
    EWOS_H_COUNTS = 4,   /* [n][p]       exit counts            (uint32)                    */
    EWOS_LAMBDA = 5,     /* [n]          cell weights           (double)                    */
    EWOS_WALK_EXIT = 6,  /* [n][N]       boundary cell of each walk's end (int32; record_walks) */
    EWOS_WALK_STEPS = 7, /* [n][N]       work steps of each walk (int32; record_walks)      */
    EWOS_WALK_MASS = 8,  /* [n][N]       unscaled G contribution of each walk (double)      */
    EWOS_WALK_VHASH = 9, /* [n][N]       XOR over the walk's interior binnings of cellmix(tag, cell),
                            cellmix = SplitMix64 finaliser of (tag<<32 | cell) folded to 32 bits;
                            tag = step k (0 for the source at x_i), 0xFFFFFFFF for the ball
                            term (uint32; record_walks)                                    */
    EWOS_WALK_XEXIT = 10 /* [n][N][d]    stopping point of each walk (double; record_walks)  */
} ewos_array;

/*
 * Many toolboxes in one persistent walk launch (uneven node counts): instance k has domain
 * domains[k] (all of one dimension and distance kind), nodes x[k] [n[k]][d] and z[k]
 * [p[k]][d] (host arrays); walks, eps, seed and the options are shared, and instance k draws
 * the Philox stream of opts->instance + k (so each toolbox equals the one ewos_toolbox_build
 * makes with that instance number).  The rows of all instances are one index space: a CTA takes
 * the next row of any instance, switching the instance's arguments in shared memory.  The
 * block size and CTAs per SM are chosen by timing the candidates on a prefix of the rows
 * (cached per batch shape) unless opts->threads_per_block is set.  record_walks, cell_weights
 * and inputs_on_device are not supported (EWOS_EINVAL).  out[k] receives toolbox k (free each
 * with ewos_toolbox_free); batch_report (may be NULL) the totals and the launch shape.
 */
ewos_status ewos_toolbox_build_batch(int count, const ewos_domain* domains, const double* const* x, const int64_t* n,
                                     const double* const* z, const int64_t* p, int64_t walks, double eps,
                                     uint64_t seed, const ewos_build_opts* opts, ewos_toolbox** out,
                                     ewos_build_report* batch_report);

/* Copy one toolbox array to dst (dst_bytes must be at least the array's size in the type
 * listed above; dst_on_device = 1 for a device pointer). */
ewos_status ewos_toolbox_get(const ewos_toolbox* tb, int which, void* dst, size_t dst_bytes,
                             int dst_on_device);
ewos_status ewos_toolbox_report(const ewos_toolbox* tb, ewos_build_report* rep);
ewos_status ewos_toolbox_shape(const ewos_toolbox* tb, int* dim, int64_t* n, int64_t* m,
                               int64_t* p, int* precision);
void ewos_toolbox_free(ewos_toolbox* tb);

/* Resident toolboxes across processes (serving, Sec. 3: the toolbox is built once per node set
 * and reused for every problem on it).  ewos_toolbox_save writes tb to the file at path: a
 * versioned header (dimension, precision, n, m, p, N, eps, seed, instance, build report) and the
 * arrays x, z, the V-centres y (when separate), lambda, P = [grad G, G] and KH = [grad H, H] in the
 * toolbox's precision, and the exit counts Hc (when present), all little-endian and raw; per-walk
 * records are not saved.  ewos_toolbox_load reads such a file into a new toolbox on the current
 * device, allocated on `stream` (NULL: the legacy default stream); the loaded toolbox is
 * bit-identical to the saved one and is freed with ewos_toolbox_free.  Errors: EWOS_EINVAL for
 * NULL arguments; EWOS_EIO when the file cannot be opened, written or read, or when its header
 * is not a toolbox header of this version or does not match the file's size (checked before any
 * device memory is touched); EWOS_ENOMEM / EWOS_ECUDA for device failures (nothing is returned). */
ewos_status ewos_toolbox_save(const ewos_toolbox* tb, const char* path);
ewos_status ewos_toolbox_load(const char* path, void* stream, ewos_toolbox** out);

typedef enum { EWOS_NL_NONE = 0, EWOS_NL_SEMILINEAR = 1, EWOS_NL_QUASILINEAR = 2 } ewos_nl_kind;
typedef enum {
    EWOS_SOLVE_FP64 = 0,   /* FP64 assembly, FP64 LU                                        */
    EWOS_SOLVE_MIXED = 1   /* tensor-core assembly + low-precision LU, FP64 refinement      */
} ewos_solve_mode;

/*
 * Problem (Sec. 3.1 eq. linearPDE written with b -> -b and f -> -f, and Sec. 3.2):
 *     -div(kappa(u) A grad u) + b . grad u + c u + N(u) = f  in D,   u = g on the boundary,
 * with N(u) = sum_k nl_coef[k] u^k (EWOS_NL_SEMILINEAR, Newton), kappa(u) = sum_k nl_coef[k] u^k
 * (EWOS_NL_QUASILINEAR, Picard), both absent for EWOS_NL_NONE.  All coefficient arrays are
 * values at the nodes (Rem. 3.3): A [n][d][d] symmetric elliptic, b [n][d] or NULL,
 * c [n] or NULL, f [nrhs][n], g [nrhs][p].
 * The linear system is (Lambda + alpha I) s = rhs of eq. linear_q with
 * alpha = rcond * ||Lambda||_F (the LU counterpart of the paper's TSVD; rcond < 0 -> 3e-2,
 * rcond = 0 -> no shift), u = G s + H g.  Newton solves R(s) + alpha s = 0 with Jacobian
 * Lambda + alpha I + G^T diag(lambda N'(u)) G from s = 0; Picard starts at u = H g.
 */
typedef struct {
    const double* A;
    const double* b;
    const double* c;
    const double* f;
    const double* g;
    int64_t nrhs;
    int nl_kind;              /* ewos_nl_kind */
    const double* nl_coef;
    int nl_ncoef;
    int mode;                 /* ewos_solve_mode */
    double rcond;             /* < 0 -> default 3e-2 */
    double tol;               /* <= 0 -> 1e-10 (Newton: relative residual; Picard: max |du|) */
    int max_iter;             /* <= 0 -> 30 (Newton) / 100 (Picard)                       */
    int inputs_on_device;     /* 1 -> A, b, c, f, g are device pointers                    */
    void* stream;             /* NULL -> the toolbox's stream                              */
    int pivoting;             /* 0 -> LU with the diagonal pivots, kept only when every
                                 multiplier has |l| <= 1 (then it is the partial-pivoting
                                 factorisation) and otherwise redone with row interchanges;
                                 1 -> always partial pivoting.  Both modes.                   */
    int batched;              /* mixed mode: 1 -> all right-hand sides refined together, one
                                 CUDA-graph launch per sweep; a semilinear problem then runs the
                                 chord iteration s <- s - (Lambda + alpha I)^-1 (R(s) + alpha s)
                                 on one factorisation, and exact Newton per right-hand side when
                                 that does not reach tol (iters = chord sweeps when it does).
                                 0 -> one right-hand side at a time, Newton for semilinear.   */
    int newton_refactor;      /* mixed-mode Newton: 0 -> each Newton system is refined with the
                                 FP32 factors of the last Jacobian factored while that refinement
                                 reaches its inexact-Newton forcing term in 24 sweeps (refactored
                                 otherwise); 1 -> the Jacobian of every step is factored        */
    int assembly;             /* mixed mode, assembly of Lambda on the tensor cores: 0 -> FP16
                                 (P and Q scaled by powers of two, each split into two FP16
                                 halves, three products: twice the TF32 rate); 1 -> TF32 (each
                                 FP32 operand split into two TF32 parts, three products)        */
} ewos_problem;

typedef struct {
    int iters;                /* Newton / Picard iterations (1 for linear)                  */
    int refine_iters;         /* FP64 refinement sweeps of the mixed mode (total)            */
    int converged;
    double alpha;
    double residual;          /* final ||R(s) + alpha s||_2 (FP64)                           */
    double ms_total, ms_assemble, ms_factor, ms_solve;
    int factorizations;       /* LU factorisations run                                       */
    int pivoted_factorizations; /* of which with row interchanges                            */
    /* device time (CUDA events on the solve's stream) of the mixed mode's tensor-core
     * assembly products (Lambda = P^T Q and the Newton Jacobian products G^T diag G) and of
     * its FP32 LU factorisations, with the method's floating-point operations of those
     * products (2 m^2 K each, m (m + 1) K for a symmetric one, which is computed as its lower
     * triangle; the three TF32 split products counted once); 0 in FP64 mode */
    double dev_ms_gemm;
    double gemm_flop;
    double dev_ms_lu;
} ewos_solve_report;

/* Solve; u_out [nrhs][n] and s_out [nrhs][m] (may be NULL) are host buffers unless
 * outputs_on_device = 1.  rep may be NULL. */
ewos_status ewos_solve(ewos_toolbox* tb, const ewos_problem* pb, double* u_out, double* s_out,
                       int outputs_on_device, ewos_solve_report* rep);

/* Euler-Lagrange route (Sec. 3.2): the gradient of the discrete functional,
 *   grad J(s) = R(s) = P^T w,  w_i = M_i (P_i s + KH_i g) + e_d lam_i (N(u_i) - f_i)     (eq. gradJ),
 * for the problem's A, b, c, f, g (first right-hand side) and a semilinear N (a quasilinear
 * equation is not the Euler-Lagrange equation of a functional: EWOS_EINVAL).  s [m] and grad [m]
 * are host buffers (device buffers when pb->inputs_on_device = 1).  FP64 toolbox: FP64
 * products and sums; FP32 toolbox: the stored FP32 entries times a two-float split of s and g,
 * summed in float pairs (about 1e-14 relative, the mixed solve's residual).  Errors:
 * EWOS_EINVAL (a NULL argument, a quasilinear problem, 0 or more than 64 coefficients),
 * EWOS_ENOMEM / EWOS_ECUDA from the device; grad is written only on EWOS_OK. */
ewos_status ewos_gradient(ewos_toolbox* tb, const ewos_problem* pb, const double* s, double* grad);

/* Adam on J (the paper's appendix algorithm; its Examples use beta1 = 0.9, beta2 = 0.999,
 * eps = 1e-10): m_j = beta1 m_{j-1} + (1 - beta1) grad J(s_{j-1}), v_j likewise with the squared
 * gradient, alpha_j = alpha sqrt(1 - beta2^j) / (1 - beta1^j), s_j = s_{j-1} - alpha_j m_j /
 * (sqrt(v_j) + eps), all on the device.  Runs max_iter steps, or stops earlier when the weighted
 * gradient norm (sum_i w_i grad_i^2)^(1/2) <= tol (w = lambda when the V-centres are the nodes,
 * else 1; checked every check_every steps, default 10; tol <= 0: never).  s_inout [m] holds the
 * start and receives the result; u_out [n] (may be NULL) receives u = G s + H g.  Errors: as
 * ewos_gradient, and EWOS_EINVAL for alpha <= 0, beta1 or beta2 outside [0, 1), eps <= 0 or
 * max_iter < 0 (checked before any device work); max_iter = 0 returns the start. */
typedef struct {
    double alpha, beta1, beta2, eps;
    int64_t max_iter;
    double tol;
    int check_every;
} ewos_adam_opts;

typedef struct {
    int64_t iters;            /* Adam steps taken                                            */
    double grad_norm;         /* weighted gradient norm at the returned s                   */
    int converged;            /* grad_norm <= tol                                            */
    double ms_total;
} ewos_adam_report;

ewos_status ewos_minimize_adam(ewos_toolbox* tb, const ewos_problem* pb, const ewos_adam_opts* opts,
                               double* s_inout, double* u_out, ewos_adam_report* rep);

/* Operator estimates (Sec. 3.1, after eq. linear_inversion): the matrices of the linear solve
 * map u = GL f + HL g of ewos_solve for the problem's A, b, c, mode, rcond, pivoting and stream
 * (f, g, nrhs and batched are ignored; nl_kind must be EWOS_NL_NONE, else EWOS_EINVAL; in mixed
 * mode all columns are refined together, as with batched = 1):
 *   GL [n][n] = G (Lambda + alpha I)^(-1) G^T diag(lambda)      (the Green operator G^L at the nodes),
 *   HL [n][p] = H - G (Lambda + alpha I)^(-1) Sigma             (the elliptic measure H^L),
 * both row-major (GL[i][k] weighs f at node k for u at node i).  Computed by solving for the
 * n + p unit right-hand sides (f = e_k; g = e_j) with one assembly and factorisation, in chunks
 * of columns sized so that each triangular solve stays well inside its bounded waits (about
 * 2^31 / m^2 columns in mixed mode, 32 times fewer in FP64 mode; all at once when they fit), on
 * a private workspace freed before the call returns.  Either output may be NULL; both are host
 * buffers, or device buffers when outputs_on_device = 1.  rep (may be NULL) as for ewos_solve,
 * with the times summed over the chunks.  Errors: EWOS_EINVAL (NULL toolbox, problem or A, no
 * output, a nonlinear problem, an unknown mode), and those of ewos_solve (EWOS_ENOMEM,
 * EWOS_ESINGULAR, EWOS_ETIMEOUT, EWOS_ECUDA); the outputs are complete only on EWOS_OK. */
ewos_status ewos_operators(ewos_toolbox* tb, const ewos_problem* pb, double* GL, double* HL,
                           int outputs_on_device, ewos_solve_report* rep);

/*
 * Request server (no counterpart in the paper; the serving loop around ewos_solve).  Solve
 * requests on device-resident toolboxes are queued in arrival order and admitted to worker
 * slots as slots and device memory free up (continuous batching); each slot is a host thread
 * with its own non-blocking CUDA stream and solve workspace, so requests in different slots run
 * concurrently on the GPU.  A request's right-hand sides are refined together in CUDA-graph
 * sweeps (mixed mode, as ewos_problem.batched = 1).  Memory: the budget is memory_fraction of
 * the device memory free at creation minus reserve_bytes (and at most budget_bytes when > 0); a
 * slot's workspace is charged at its estimated size; a request that does not fit waits for a
 * slot to finish, or fails with EWOS_ENOMEM when nothing is running and it still does not fit.
 * The caller keeps every toolbox alive until the requests on it have been waited for.  Calls
 * are thread safe.
 */
typedef struct ewos_server ewos_server;
typedef struct {
    int max_slots;            /* concurrent requests (<= 0 -> 4, at most 64)                 */
    double memory_fraction;   /* of the free device memory (<= 0 -> 0.8)                      */
    int64_t reserve_bytes;    /* kept free for the caller                                     */
    int64_t budget_bytes;     /* > 0: upper bound of the budget                               */
} ewos_server_opts;
typedef struct {
    uint64_t submitted, completed, failed;
    int queued, active, peak_active, slots;
    int64_t budget_bytes, charged_bytes;
} ewos_server_stats;
typedef struct {
    double queue_ms;          /* submission -> admission to a slot                            */
    double run_ms;            /* admission -> results on the host                             */
    double total_ms;
    int slot;
} ewos_request_timing;

ewos_status ewos_server_create(const ewos_server_opts* opts, ewos_server** out);
/* Copies the problem's host arrays (inputs_on_device must be 0; stream is ignored: the slot's
 * stream is used) and queues it; *ticket identifies the request. */
ewos_status ewos_server_submit(ewos_server* sv, ewos_toolbox* tb, const ewos_problem* pb, uint64_t* ticket);
/* Waits (timeout_s <= 0: without limit; on expiry EWOS_ETIMEOUT and the request stays queued)
 * for a request, copies u [nrhs][n] and s [nrhs][m] to the host buffers that are not NULL and
 * releases it; returns the solve's status. */
ewos_status ewos_server_wait(ewos_server* sv, uint64_t ticket, double timeout_s, double* u_out, double* s_out,
                             ewos_solve_report* rep, ewos_request_timing* timing);
ewos_status ewos_server_query(ewos_server* sv, ewos_server_stats* out);
/* Finishes the queued requests, stops the slots and frees their workspaces. */
void ewos_server_destroy(ewos_server* sv);

/* Test hooks (no counterpart in the paper): Philox4x32-10 blocks for count counters
 * (ctr [count][4], key [2], out [count][4], host uint32), and the d = 2 Green-density radius
 * R(u) (inverse of F(t) = t^2 - t^2 ln t^2, Prop. 2.6 (i.1)) in FP32 or FP64 for count
 * uniforms (host arrays of the chosen type).  Both run the device code of the walk kernel. */
ewos_status ewos_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t count);
ewos_status ewos_debug_green_radius(const void* u, void* R, int64_t count, int precision);
/* Test hook (no counterpart in the paper): C [M][N] = A^T B for host FP32 arrays A [K][M],
 * B [K][N], through the tensor-core (tcgen05) GEMMs of the mixed-precision solve: split = 0
 * plain TF32; split = 1 three TF32 products per step (hi*hi + hi*lo + lo*hi), accumulated in
 * chunks (the long-K product of the assembly); split = 3 the same with A and B scaled by powers
 * of two and split into FP16 halves (kind::f16); split = 2 and 4 are 1 and 3 with the symmetric
 * launch (only the tiles on and below the diagonal are computed, each also stored transposed: for
 * a symmetric A^T B, M = N).  EWOS_EINVAL for another split, and when the device has no
 * sm_100-family tensor cores. */
ewos_status ewos_debug_tc_gemm(const float* A, const float* B, float* C, int M, int N, int K, int split);
/* Test hook (no counterpart in the paper): the tensor-core assembly of the mixed-precision solve,
 * C [m][m] = Lambda = P^T Q with Q_i = M_i P_i (eq. linear_q), for host arrays P [D+1][n][m] (FP32),
 * M [n][D+1][D+1] (FP64; row-major blocks) and C (FP32); D = 2 or 3.  f16 != 0 takes the FP16
 * form (operands scaled by powers of two and split into FP16 halves), f16 = 0 the TF32 form
 * (three TF32 products); sym != 0 computes the tiles on and below the diagonal and mirrors them
 * (for symmetric M_i).  EWOS_EINVAL when the device has no sm_100-family tensor cores. */
ewos_status ewos_debug_tc_assemble(const float* P, const double* M, int n, int m, int D, float* C, int sym, int f16);
/* Test hook (no counterpart in the paper): the trailing update of the FP32 LU of the mixed-precision
 * solve on the tensor cores, C [M][N] -= A [M][K] B [K][N] for host FP32 row-major arrays (C read
 * and written in place).  f16 != 0: each row of A and each column of B scaled by a power of two
 * and split into FP16 halves, three kind::f16 products (the form of the LU's rank-512 updates);
 * f16 = 0: three TF32 products.  EWOS_EINVAL for M, N or K below 1, and when the device has no
 * sm_100-family tensor cores. */
ewos_status ewos_debug_tc_update(const float* A, const float* B, float* C, int M, int N, int K, int f16);

/* Test hooks for the failure paths (no counterpart in the paper).
 * ewos_debug_set_flow_wait_limit: the flag waits of the dataflow triangular solves (mixed mode)
 * give up after `polls` polls on the current device (polls < 0 restores the default, 2^22);
 * a solve whose waits run out returns EWOS_ETIMEOUT and the device stays usable.  The waits
 * poll plain flags in global memory: no copy is in flight when they give up.
 * ewos_debug_fail_allocations: the device allocation of the library that follows `after` more
 * successful ones fails once, as if the device were out of memory (the entry point returns
 * EWOS_ENOMEM); after < 0 cancels. */
ewos_status ewos_debug_set_flow_wait_limit(int64_t polls);
void ewos_debug_fail_allocations(int64_t after);

/* Number of kernels this library has launched in the process so far (all entry points). */
unsigned long long ewos_launch_count(void);

const char* ewos_status_string(ewos_status s);
const char* ewos_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* EWOS_API_H_ */

/*
 * tacta.h -- C ABI of the GB300 (sm_103a) Triangle Algorithm / Centering
 * Triangle Algorithm solvers (Lau & Kalantari, arXiv:2304.12168).
 *
 * The library computes approximate and minimum-norm solutions of A x = b and
 * of the normal equation AᵀA x = Aᵀb for an m x n real matrix A of any shape
 * and rank, stored dense row-major or CSR, in FP64 on one GPU.
 *
 * Entry points (all return a tacta_status; none aborts or prints):
 *   cta_solve  -- Algorithm 1.1 (CTA, H = A Aᵀ, Sec. 3.2) with the t-cycling
 *                 of Sec. 5.1: iterates of F_t (Eqs. F_t, eqcoeff, CTAGEN7,
 *                 CTAGEN7A).
 *   ta_solve   -- Algorithm 2.2 (TA with growing rho, Sec. 4.3): pivot from
 *                 Thm. prop0TA (Eqs. vr, eqlem2), step from Prop. prop1TA
 *                 (Eq. alph).
 *   ta_minnorm -- the hybrid of Sec. 5.2: CTA to tol_cta, then Algorithm 2.5
 *                 (bisection on rho, Sec. 4.4, lower bound of Cor. cor1) on
 *                 (A, b) when CTA's x solves A x = b, else on (AᵀA, Aᵀb)
 *                 applied through products with A and Aᵀ.
 * Plans (tacta_plan_*) hold the device copy of A and its transpose, so that
 * several right-hand sides reuse one setup.
 *
 * Conventions
 *   - Every array is caller-owned. The library copies A into its own device
 *     storage (plus Aᵀ) at plan creation; the caller's A may be freed after
 *     tacta_plan_create returns (one-shot calls keep nothing).
 *   - on_device = 1: every pointer argument of the call (A's arrays, b, x0,
 *     x_out, hist) is a CUDA device pointer of the current device;
 *     on_device = 0: all are host pointers and the library does the copies.
 *   - All GPU work is enqueued on opt->stream (a cudaStream_t; NULL = the
 *     legacy default stream). Every call synchronises that stream before it
 *     returns, so outputs are ready on return.
 *   - Tolerances are relative: the residual test is ||b - A x|| <= tol ||b||,
 *     the normal-equation test ||Aᵀ(b - A x)|| <= tol_normal ||Aᵀ b||.
 *   - Validation: sizes and options are checked on the host before any GPU
 *     work (m, n >= 1 and < 2^31; dense m*n <= 2^40; 0 <= nnz < 2^31; tol
 *     finite and > 0; t_max in 1..8; max_iter >= 0). The CSR structure
 *     (rowptr[0] = 0, non-decreasing, rowptr[m] = nnz, 0 <= colidx < n) is
 *     checked by a kernel right after A is copied to the device, before any
 *     kernel indexes with it; a violation returns TACTA_ERR_INVALID.
 *   - MAXITER, BREAKDOWN and WITNESS still fill x_out and info.
 *   - Errors (negative status) leave x_out unspecified; tacta_last_error()
 *     gives a message for the calling thread.
 */
#ifndef TACTA_H
#define TACTA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TACTA_OK = 0,            /* a stopping test of the algorithm was met          */
    TACTA_MAXITER = 1,       /* iteration cap reached first                        */
    TACTA_BREAKDOWN = 2,     /* step undefined: Hankel rank 0 or ||v - b'|| = 0    */
    TACTA_WITNESS = 3,       /* Alg. 2.1 witness (only from internal trips)        */
    TACTA_ERR_INVALID = -1,  /* bad argument (message in tacta_last_error)         */
    TACTA_ERR_NONFINITE = -2,/* NaN / Inf appeared in a reduction                  */
    TACTA_ERR_CUDA = -3,     /* a CUDA runtime call failed                         */
    TACTA_ERR_OOM = -4,      /* device allocation failed                           */
    TACTA_ERR_TIMEOUT = -5   /* a bounded device wait gave up                      */
} tacta_status;

/* why the iteration ended (tacta_info.reason) */
enum {
    TACTA_REASON_NONE = 0,
    TACTA_REASON_RESIDUAL = 1,   /* ||b - A x|| <= tol ||b|| (true residual)               */
    TACTA_REASON_NORMAL = 2,     /* ||Aᵀ r|| <= tol_normal ||Aᵀ b||: normal equation solved */
    TACTA_REASON_MAXITER = 3,
    TACTA_REASON_BREAKDOWN = 4,
    TACTA_REASON_WITNESS = 5,
    TACTA_REASON_GAP = 6,        /* Alg. 2.5: rho_upper - rho_lower <= tol ||x_eps||        */
    TACTA_REASON_ZERO_RHS = 7,   /* b = 0: x = 0                                            */
    TACTA_REASON_NONFINITE = 8,
    TACTA_REASON_TIMEOUT = 9,    /* a bounded wait inside a kernel gave up (TACTA_ERR_TIMEOUT) */
    TACTA_REASON_RHO_BOUND = 10, /* ta_solve: rho passed opt->rho_max                          */
    TACTA_REASON_ENHANCED = 11   /* CTA with opt->enhanced: the enhanced stop of Sec. 3.2 held   */
};

enum { TACTA_DENSE = 0, TACTA_CSR = 1 };

/* t-cycling (Sec. 5.1): ping-pong 1,2,..,t_max,..,2,1,2,..; sawtooth 1..t_max,1..; fixed t_max */
enum { TACTA_CYCLE_PINGPONG = 0, TACTA_CYCLE_SAWTOOTH = 1, TACTA_CYCLE_FIXED = 2 };

typedef struct {
    int64_t m, n;            /* rows, columns                                        */
    int64_t nnz;             /* CSR: stored entries (= rowptr[m]); dense: ignored     */
    int32_t format;          /* TACTA_DENSE (row-major m x n) or TACTA_CSR            */
    int32_t on_device;       /* 1: device pointers (all arrays of the call); 0: host  */
    const double* vals;      /* dense: m*n values, row-major; CSR: nnz values         */
    const int32_t* rowptr;   /* CSR: m+1 offsets                                      */
    const int32_t* colidx;   /* CSR: nnz column indices                               */
} tacta_matrix;

typedef struct {
    double tol;              /* relative residual tolerance (> 0)                              */
    double tol_normal;       /* relative normal-equation tolerance; < 0: same as tol;
                                0: stop only when Aᵀ r is exactly 0                            */
    double tol_cta;          /* ta_minnorm: tolerance of the CTA phase; <= 0: same as tol     */
    double pivot_tol;        /* truncation threshold of the scaled Hankel Cholesky; <= 0: 1e-12 */
    int32_t max_iter;        /* iteration cap (CTA: F_t steps; TA: loop trips)                 */
    int32_t t_max;           /* largest CTA order (1..8; the paper cycles up to 5)             */
    int32_t cycle;           /* TACTA_CYCLE_*                                                   */
    int32_t recompute_every; /* R: true residual b - A x every R iterations; 0: never          */
    int32_t use_graph;       /* 1: replay the iteration body as a captured CUDA graph          */
    int32_t poll_every;      /* host checks the device stop flag every this many iterations    */
    int32_t profile;         /* 1: time every product of the iteration with CUDA events on the
                                stream (forces use_graph = 0); results in tacta_info.spmv_*    */
    int32_t precision;       /* TACTA_PRECISION_FP64 (default) or TACTA_PRECISION_MIXED (CSR,
                                cta_solve / plan_cta / minnorm's CTA phase): FP32 chain products
                                and updates, FP64 centering solve, stop tests and refinement
                                b - A x every recompute_every steps; pivot_tol <= 0 then means 1e-6 */
    int32_t nonneg;          /* ta_solve only: 1 = TA for LP feasibility A x = b, x >= 0 (Sec. 6):
                                c is replaced by max(c, 0); WITNESS when ||max(c,0)|| <=
                                tol_normal ||Aᵀb|| while (b - b')ᵀb > 0 (Farkas certificate)   */
    int32_t enhanced;        /* CTA, FP64 path: 1 = the enhanced algorithm of Sec. 3.2. At a step of
                                order t >= 2 it also stops when, for the smallest j <= t-1, the j-th
                                first-order iterate r_j = F_1^j(r') has r_jᵀ H r_j <= tol_normal²
                                ||Aᵀb||², and returns x^ = x' + sum_{i<j} alpha_{1,1}(r_i) Aᵀ r_i
                                (Eq. widehatxB; reason ENHANCED). r_jᵀ H r_j is evaluated from the
                                step's moments phi_1..phi_{2j+1}, so the test is resolved for
                                tol_normal down to ~1e-7 (below that its rounding, ~1e-16 phi_1,
                                reaches the threshold)                                          */
    int32_t fused_chain;     /* CTA on CSR operands whose A and Aᵀ both take the run-staged product
                                (banded and stencil matrices): 1 (default) = the 2t products
                                z_i = Aᵀ u_{i-1}, u_i = A z_i of a step (Alg. 1.1) and their moments
                                run as one cooperative launch, the products separated by grid-wide
                                barriers, on the diagonal form of A and Aᵀ when their nonzeros lie
                                on at most 5 diagonals (col - row constant), else on the run-staged
                                CSR; 2 = the same launch, always on the run-staged CSR; 0 = one
                                launch per product. Same arithmetic per row; the moments' partial
                                sums are added in a different fixed order. With 1 and 2 the
                                launch is the whole F_t step: after the products every block
                                solves the auxiliary equation from the same moment partials and
                                updates its slice of x and r (one launch per step); 3 = the
                                products of option 1 in one launch, the auxiliary solve and the
                                update as two more launches                                       */
    int32_t wait_limit_log2; /* the fused chain's grid-wide waits (a block waiting for every block
                                to finish the previous product) give up after 2^this SM cycles
                                and end the call with TACTA_ERR_TIMEOUT; 0 = 31 (about a second).
                                Small values exist so that tests can make a wait run out; the
                                waits on the block's own copies keep the ~1 s limit          */
    double rho_max;          /* ta_solve: stop (reason RHO_BOUND) once rho exceeds this; <= 0: none */
    void* stream;            /* cudaStream_t (NULL: legacy default stream)                      */
} tacta_options;

enum { TACTA_PRECISION_FP64 = 0, TACTA_PRECISION_MIXED = 1 };

typedef struct {
    int32_t status;          /* same as the return value                               */
    int32_t reason;          /* TACTA_REASON_*                                         */
    int32_t iters;           /* CTA: F_t steps; TA: loop trips (all trips for minnorm) */
    int32_t matvecs;         /* products with A or Aᵀ made by the iteration            */
    double rel_res;          /* true ||b - A x|| / ||b|| at exit                       */
    double rel_normal_res;   /* true ||Aᵀ(b - A x)|| / ||Aᵀ b|| at exit                */
    double rho;              /* TA: final rho; minnorm: rho_upper                      */
    double rho_lower;        /* minnorm: the lower bound rho_lower (Cor. cor1)         */
    int32_t trips;           /* minnorm: bisection trips                               */
    int32_t cta_iters;       /* minnorm: CTA iterations of the first phase             */
    int32_t normal_system;   /* minnorm: 1 when TA ran on (AᵀA, Aᵀb)                    */
    int32_t hist_len;        /* entries written to hist                                */
    int64_t launches;        /* GPU kernels launched by the call                        */
    int32_t spmv_count;      /* profile = 1: units timed. Fused step (fused_chain 1, 2): one
                                unit per F_t step launch; otherwise one per product of the
                                iteration chain                                          */
    int32_t spmv_pad;
    double spmv_ms;          /* profile = 1: summed device time of those launches       */
    double spmv_bytes;       /* profile = 1: their algorithmic bytes. Per product: values,
                                indices, row offsets, input vector once, output vector
                                once. Per fused F_t step of order t: t such products with
                                A and t with Aᵀ in CSR, the chain's vectors and the update's
                                8 (t + 2)(m + n) (4-byte values and vectors on the FP32
                                chain)                                                   */
} tacta_info;

/* Fill *opt with the defaults: tol 1e-10, tol_normal -1, tol_cta 0, pivot_tol 1e-12,
   max_iter 1000, t_max 5, ping-pong cycle, R = 40, use_graph 1, poll_every 64, profile 0,
   precision FP64, nonneg 0, enhanced 0, fused_chain 1, wait_limit_log2 0 (2^31 cycles),
   rho_max 0 (none), NULL stream. */
void tacta_default_options(tacta_options* opt);

/*
 * cta_solve -- Algorithm 1.1 (CTA) with H = A Aᵀ.
 *   A       matrix (see tacta_matrix); b: m values; x0: n values or NULL (start at 0;
 *           from 0 the iterates stay in range(Aᵀ), Thm. thmone (4));
 *   opt     options (NULL: defaults); x_out: n values (written);
 *   hist    relative residual after each F_t step, hist[0] at the start
 *           (min(iters+1, hist_cap) values; NULL or hist_cap = 0: not written);
 *   info    outcome (may be NULL).
 */
tacta_status cta_solve(const tacta_matrix* A, const double* b, const double* x0,
                       const tacta_options* opt, double* x_out, double* hist,
                       int32_t hist_cap, tacta_info* info);

/* ta_solve -- Algorithm 2.2 (TA, rho = 0 grown on witnesses). Arguments as cta_solve;
   x0 (optional) is a warm start: b' = A x0 and rho = ||x0||. hist holds ||b - b'|| / ||b||. */
tacta_status ta_solve(const tacta_matrix* A, const double* b, const double* x0,
                      const tacta_options* opt, double* x_out, double* hist,
                      int32_t hist_cap, tacta_info* info);

/* ta_minnorm -- approximate minimum-norm solution (Def. minnormapp): CTA to tol_cta from 0,
   then Algorithm 2.5 at tol. x0 is ignored. hist holds the CTA phase's history.
   info->rho = rho_upper (>= ||x_out||), info->rho_lower = rho_lower (< ||x_*||). */
tacta_status ta_minnorm(const tacta_matrix* A, const double* b, const double* x0,
                        const tacta_options* opt, double* x_out, double* hist,
                        int32_t hist_cap, tacta_info* info);

/* Plans: device copy of A (+ Aᵀ, built on the GPU) and solver workspace, on the device
   that is current at creation. The plan must be used from that device only.
   Plan solves take the same arguments as the one-shot calls minus A; their vector
   pointers follow A's on_device flag given at creation. */
typedef struct tacta_plan_s* tacta_plan;

tacta_status tacta_plan_create(const tacta_matrix* A, const tacta_options* opt, tacta_plan* plan);
tacta_status tacta_plan_cta(tacta_plan plan, const double* b, const double* x0,
                            const tacta_options* opt, double* x_out, double* hist,
                            int32_t hist_cap, tacta_info* info);
tacta_status tacta_plan_ta(tacta_plan plan, const double* b, const double* x0,
                           const tacta_options* opt, double* x_out, double* hist,
                           int32_t hist_cap, tacta_info* info);
tacta_status tacta_plan_minnorm(tacta_plan plan, const double* b, const double* x0,
                                const tacta_options* opt, double* x_out, double* hist,
                                int32_t hist_cap, tacta_info* info);
void tacta_plan_destroy(tacta_plan plan);

/* tacta_plan_minnorm_bisect -- Algorithm 2.5 (Sec. 4.4) alone: bisection on rho from a given
   approximate solution x_eps of M x = rhs, M = A and rhs = b (normal = 0) or M = AᵀA and
   rhs = Aᵀb applied through products with A and Aᵀ (normal = 1).
   rho_hi = ||x_eps||, rho_lo = 0; while rho_hi - rho_lo > tol ||x_eps||: Alg. 2.1 at the
   midpoint rho, from the last witness (from x = 0 before the first); a trip that meets the
   residual test sets rho_hi = rho and its x becomes the answer, a witness sets
   rho_lo = (b - b')ᵀb / ||Mᵀ(b - b')|| (Cor. cor1), a normal-equation stop ends the call with
   that x. max_iter bounds the TA iterations of all trips together.
   b, x_eps, x_out follow the plan's on_device flag (m, n, n values). trip_log is a HOST
   array of 6 * log_cap doubles (NULL with log_cap = 0: not written): trip i writes
   {rho, the trip's stop reason (TACTA_REASON_*), rho_hi after the trip, rho_lo after the
   trip, the trip's TA iterations, 0}. info->trips = trips run (log rows beyond log_cap are
   dropped), info->rho = rho_hi, info->rho_lower = rho_lo, info->reason = GAP when the gap
   closed. Errors as the other plan calls. */
tacta_status tacta_plan_minnorm_bisect(tacta_plan plan, const double* b, const double* x_eps, int32_t normal,
                                       const tacta_options* opt, double* x_out, double* trip_log,
                                       int32_t log_cap, tacta_info* info);

/* tacta_plan_transpose -- a new plan for Aᵀ built from the device copy held by `plan`
   (used by adjoint solves: the backward of a solve with A solves with Aᵀ). The new plan's
   vector pointers follow the same on_device flag. */
tacta_status tacta_plan_transpose(tacta_plan plan, const tacta_options* opt, tacta_plan* out);

/* tacta_plan_matvec -- y = A x (transpose = 0) or y = Aᵀ x (transpose = 1) with the plan's
   product kernels; x and y follow the plan's on_device flag (lengths n / m, or m / n). */
tacta_status tacta_plan_matvec(tacta_plan plan, int32_t transpose, const double* x, double* y,
                               const tacta_options* opt);

/* tacta_plan_residual -- r = b - A x (transpose = 0) or r = b - Aᵀ x (transpose = 1), the
   residual of Sec. 2 formed by the plan's product kernel (its residual epilogue, FP64);
   x, b, r follow the plan's on_device flag (lengths n, m, m or m, n, n). r may not alias
   x or b. */
tacta_status tacta_plan_residual(tacta_plan plan, int32_t transpose, const double* x, const double* b, double* r,
                                 const tacta_options* opt);

/* tacta_plan_outer -- out[k] += alpha * u[row(k)] * v[col(k)] for every stored entry k of A
   (CSR: in the caller's nonzero order; dense: row-major m*n). With u = -lambda, v = x it
   forms the gradient dL/dA of x = A^{-1} b on A's pattern (Sec. 3 solves made
   differentiable; the paper has no counterpart). u: m values, v: n values, out: the
   caller's value array layout; all follow the plan's on_device flag. */
tacta_status tacta_plan_outer(tacta_plan plan, double alpha, const double* u, const double* v,
                              double* out, const tacta_options* opt);

/*
 * tacta_residual_static -- r = b - A x with ||r||² and rᵀb, allocating nothing.
 *   The paper has no counterpart: this entry serves callers that cannot allocate
 *   device memory when they need a residual -- code inside a framework whose
 *   caching allocator has reserved the device, and latency-bound loops that must
 *   not enter cudaMalloc / cudaFree (which may synchronize the device). Instead of
 *   plan workspace it uses one file-scope device array of 1 MiB per device
 *   (held by every GPU that loads the library until the process exits).
 *   A        dense or CSR, on_device = 1 (host arrays are rejected: copying them
 *            would need an allocation); A->m <= 16,773,120 (the scratch holds one
 *            pair of doubles per 256-row block); larger m -> TACTA_ERR_INVALID.
 *   x, b     device pointers, n and m values; r_out: device pointer, m values.
 *   norms_out  two doubles (host or device): ||r||², rᵀb.
 *   stream   cudaStream_t or NULL; the call synchronizes it before returning.
 *   Makes no cudaMalloc / cudaFree or other allocating call. Every call on a device
 *   shares the scratch array, which keeps the last call's contents; the ticket
 *   counter that must start at zero is cleared at the start of each call; calls
 *   whose work overlaps on the GPU race on the array. The first call on each
 *   device looks up the array's address (cudaGetSymbolAddress) with that device
 *   current; make that first call before any stream capture. The address stays
 *   cached for the process's life, so it is stale after a cudaDeviceReset of that
 *   device: do not call this entry point on a device after resetting it. Device
 *   indices >= 64 -> TACTA_ERR_INVALID.
 */
tacta_status tacta_residual_static(const tacta_matrix* A, const double* x, const double* b,
                                   double* r_out, double* norms_out, void* stream);

/*
 * Batched dense systems -- tacta_batch_*
 *   Many independent systems A_s x_s = b_s (s = 0 .. count-1), A_s dense m_s x n_s,
 *   each solved by CTA (Alg. 1.1 with H = A_s A_sᵀ and the t-cycling of Sec. 5.1)
 *   from x_s = 0, so that x_s stays in range(A_sᵀ) (Thm. thmone (4)) and a consistent
 *   rank-deficient system yields the minimum-norm solution. The systems run in one
 *   persistent launch of a single-block kernel (replayed as a CUDA graph when
 *   opt->use_graph is set): each thread block takes the next unsolved system from a
 *   queue, ordered longest first by the earlier solves' measured time per system (the
 *   first solve: largest m_s n_s first), so the slowest systems start at once and short
 *   ones fill the tail. From the second solve on, the longest systems can go to thread-
 *   block clusters of a second persistent launch that starts first
 *   (tacta_batch_set_wide). The paper treats one system at a time; batching is this
 *   library's extension.
 *
 *   Storage of the copy of A_s that the chain z_i = Aᵀ u_{i-1}, u_i = A z_i reads:
 *     TACTA_BATCH_FP64 -- FP64 chain; the iteration follows the FP64 path exactly.
 *     TACTA_BATCH_FP32 -- FP32 values and chain (FP32 accumulation).
 *     TACTA_BATCH_BF16 -- BF16 values, FP32 chain and accumulation (widened on CUDA
 *                         cores, or on the tensor cores: tacta_batch_config_tensor_cores).
 *   In every mode the moments, the auxiliary solve (Eq. eqcoeff) and the stop
 *   tests are FP64, and the residual b - A x is recomputed in FP64 from an FP64
 *   copy of A_s: every recompute_every steps, whenever the carried residual passes
 *   the tolerance (a pass counts only on the recomputed residual), and -- FP32 and
 *   BF16 -- once the carried residual has fallen by 1e-3 since the last recompute,
 *   where the FP32 correction is folded into the FP64 x (iterative refinement).
 *   A low-precision copy perturbs A_s by up to its unit roundoff (2^-24 FP32,
 *   2^-9 BF16): refinement still drives the FP64 residual to tol while
 *   cond(A_s) times that roundoff stays below one, and the solution's component
 *   outside range(A_sᵀ) is of that relative size.
 *
 *   Layout: the systems are packed back to back in system order -- A_s row-major
 *   at element sum_{j<s} m_j n_j of vals, b_s at sum_{j<s} m_j of b, x_s at
 *   sum_{j<s} n_j of x. 1 <= m_s, n_s <= 4096; the chain's vectors of the largest
 *   system must fit a block's shared memory ((t_max + 1)(m_max + n_max) values),
 *   else tacta_batch_cta returns TACTA_ERR_INVALID.
 */
typedef struct tacta_batch_s* tacta_batch;
enum { TACTA_BATCH_FP64 = 0, TACTA_BATCH_FP32 = 1, TACTA_BATCH_BF16 = 2 };

/* tacta_batch_create -- copy the count systems' matrices (vals, FP64, host or device per
   on_device; m and n are host arrays) to the device, with the storage copy and each
   system's chain scale. Uses opt->stream only. The caller's arrays may be freed after. */
tacta_status tacta_batch_create(int32_t count, const int32_t* m, const int32_t* n, const double* vals,
                                int32_t on_device, int32_t storage, const tacta_options* opt,
                                tacta_batch* out);

/* tacta_batch_cta -- solve every system. b: sum m_s values, x: sum n_s values (host or
   device, any: copies go through cudaMemcpyDefault). iters, rel_res (the recomputed FP64
   ||b_s - A_s x_s|| / ||b_s||) and reason (TACTA_REASON_*) receive count values each and
   may be NULL. Options used: tol, tol_normal, pivot_tol (0: 1e-12 FP64, 1e-6 otherwise),
   max_iter (per system), t_max, cycle, recompute_every, use_graph, stream. */
tacta_status tacta_batch_cta(tacta_batch batch, const double* b, double* x, int32_t* iters,
                             double* rel_res, int32_t* reason, const tacta_options* opt);

/* Launch configurations: threads per block and resident blocks per SM. The autotuner
   times every configuration that fits on (batch, b) with the given options (max_iter caps
   each system's steps; single blocks only), keeps the best for later solves and returns
   its index and score (ms): before any full solve the capped run's time; after one, the
   makespan of a full solve that the capped run predicts -- every system's one-block time
   taken as its time per step in the capped run times its step count in the last full
   solve, then the planner's simulated makespan with those times (tacta_batch_set_wide).
   set_config picks one (-1: the default). tacta_batch_config_tensor_cores(c) is 1 when configuration c runs
   the chain's products on the tensor cores (BF16 tiles, mma.sync m16n8k16 with FP32
   accumulation, the FP32 chain vectors carried exactly as three BF16 terms): it admits
   BF16 storage with n_s <= 1024 only (other batches: TACTA_ERR_INVALID from
   tacta_batch_cta, skipped by the autotuner). tacta_batch_config_stage_bytes(c) is the
   ring stage of the fused-pass configurations (the tile of rows of A_s that a pass takes
   at a time: 16, 32 or 48 KB on CUDA cores, 40 or 48 KB on the tensor cores; 0 for the
   others), so the autotuner searches tile sizes as well as launch shapes. */
int32_t tacta_batch_num_configs(void);
tacta_status tacta_batch_config_shape(int32_t config, int32_t* threads, int32_t* blocks_per_sm);
int32_t tacta_batch_config_tensor_cores(int32_t config);
int32_t tacta_batch_config_stage_bytes(int32_t config);
tacta_status tacta_batch_tune(tacta_batch batch, const double* b, const tacta_options* opt,
                              int32_t* best_config, double* best_ms);
tacta_status tacta_batch_set_config(tacta_batch batch, int32_t config);
/* tacta_batch_timeline -- when each system of the last completed tacta_batch_cta was
   taken by a thread block and when that block finished it: count values each, device
   clock (%globaltimer, nanoseconds; only differences are meaningful), host or device
   pointers. Systems the last solve did not reach hold their previous values (0 before
   the first solve). The batch's completion profile -- how many systems are done by a
   given time, how many blocks are still busy in the launch's tail -- follows from them.
   Synchronous. */
tacta_status tacta_batch_timeline(tacta_batch batch, int64_t* t_begin_ns, int64_t* t_end_ns);
/* tacta_batch_set_wide -- thread-block clusters for the longest systems. A batch takes
   its slowest system's time, and a system that needs the whole step budget keeps one
   block busy long after the others have finished. A cluster of C blocks (one per SM)
   solves such a system together: each block holds ceil(m_s / C) rows of A_s, the
   partial products Aᵀu are added across the cluster through distributed shared memory,
   the moments and norms are block partials added in rank order (every block takes the
   same FP64 decisions). The clusters start first and the single-block kernel takes the
   other systems on the remaining SMs and on each SM a cluster leaves.
     systems -1 (default): planned before each solve from the measured times of the
                earlier solves (none before the first): the share of least simulated
                makespan (tacta_batch_wide_plan). A system's time on a C-block cluster is
                modelled per step as the larger of its one-block time / C and the time to
                stream a block's rows when they exceed its shared memory, plus an overhead
                h0 + h1 C refitted after every clustered solve;
     systems 0: off;
     systems > 0: that many systems from the head of the queue order (longest first by
                the last solve; largest m_s n_s first before any), on clusters of
                `cluster` blocks (1..8; 0: the largest of 8, 4, 2, 1 whose vectors fit
                a block's shared memory), `clusters` clusters (0: one per system, at most
                as many as can be resident).
   A system a cluster solves runs the same iteration with its sums in another order:
   its bits may differ from a one-block solve, within the same tolerances. */
tacta_status tacta_batch_set_wide(tacta_batch batch, int32_t systems, int32_t cluster, int32_t clusters);
/* tacta_batch_wide_plan -- the clusters' share that the next tacta_batch_cta with these
   options would use (systems 0: none) and its predicted makespan in ms (0 while no
   solve has measured the systems' times). Any output may be NULL. */
tacta_status tacta_batch_wide_plan(tacta_batch batch, const tacta_options* opt, int32_t* systems, int32_t* cluster,
                                   int32_t* clusters, double* predicted_ms);
/* tacta_batch_simulate_makespan -- the planner's schedule model, on the host (no device
   needed): nw cluster jobs of times w take `clusters` clusters of `cluster` SMs, each job
   the next cluster to be free (longest first); nd one-block jobs of times d take per_sm
   blocks on every SM no cluster holds from time 0 and on a cluster's SMs from the time
   it has finished, each job the next block to be free (longest first; past the 512
   longest, the rest spread as a fluid over the blocks' free times). Returns the time
   the last job ends, in the unit of w and d; -1 on invalid arguments (a negative count,
   a negative or NaN time, clusters x cluster > sms, a NULL array with a nonzero count,
   cluster jobs without clusters). */
double tacta_batch_simulate_makespan(const double* w, int32_t nw, int32_t clusters, int32_t cluster, const double* d,
                                     int32_t nd, int32_t sms, int32_t per_sm);
/* tacta_batch_plan_search -- the planner that tacta_batch_cta runs before each solve,
   on the host (no device needed), given what the solve would take from the device.
     dur[count]       each system's one-block time (ns); all > 0, else "unknown": no plan
     steps[count]     its step count in the last full solve (NULL: 0)
     m, n[count]      its shape (the rows a block of a cluster holds, the row length)
     storage, t_max, cycle   as in tacta_batch_create / tacta_options
     sms, per_sm      the device's SMs and the launch configuration's blocks per SM
     max_clusters[5], a_cap[5]   for cluster sizes 16, 8, 4, 2, 1: how many clusters can
                      be resident (0: the size's vectors do not fit a block) and how many
                      elements of A a block stages in shared memory
     wide_mode, wide_cluster, wide_clusters   as in tacta_batch_set_wide
     h0               the cluster-time model's per-step overhead (ns; 12000 before any
                      clustered solve)
   A system's time on a C-block cluster is modelled per step as the larger of its
   one-block time / C and, when a block's ceil(m/C) rows exceed a_cap, the time to stream
   them (2 x the schedule's mean order passes at 40 GB/s), plus h0 + 500 ns x C. With the
   planner on (wide_mode -1) the plan is the one of least simulated makespan
   (tacta_batch_simulate_makespan) among: no clusters, and for C = 16, 8, 4, 2 the K = 1,
   2, ... (at most 96) longest systems with at least 4C rows and at least a quarter of the
   balanced time (sum dur / (sms per_sm)), on min(K, max_clusters) clusters; a plan must
   beat the best so far by 2%. Out: plan[3] = systems, cluster size, clusters (0, 0, 0:
   none) and order[count], the queue order (a permutation of 0 .. count-1): the
   clusters' systems first, longest in cluster time first, then the rest longest first
   (ties keep system order). Returns the simulated makespan in ms; 0 while the times are
   unknown; infinity for a forced plan with no cluster size that fits; -1 on invalid
   arguments. */
double tacta_batch_plan_search(int32_t count, const double* dur, const int32_t* steps, const int32_t* m,
                               const int32_t* n, int32_t storage, int32_t t_max, int32_t cycle, int32_t sms,
                               int32_t per_sm, const int32_t* max_clusters, const int64_t* a_cap, int32_t wide_mode,
                               int32_t wide_cluster, int32_t wide_clusters, double h0, int32_t* plan,
                               int32_t* order);
void tacta_batch_destroy(tacta_batch batch);
/* message of the last failed tacta_batch_* call on the calling thread */
const char* tacta_batch_last_error(void);

/* tacta_column_partition -- the column shards of a CTA solve spread over G GPUs (one
   process per GPU). With A = [A_1 ... A_G] split by columns, H = A Aᵀ = sum_g A_g A_gᵀ
   (Sec. 3 with H = A Aᵀ, Sec. 5), so every GPU keeps its slice x_g of x and the replicated
   m-vectors r and u_i: z_{i,g} = A_gᵀ u_{i-1} is local, and u_i = sum_g A_g z_{i,g} needs
   one sum over the GPUs per H-apply. That all-reduce carries m + 2 doubles per GPU:
   [0, m) the GPU's A_g z_{i,g}, [m] its ||z_{i,g}||² (the partial of phi_{2i-1}),
   [m + 1] zero (keeps the buffer a multiple of 16 bytes); phi_{2i} = ||u_i||² is then
   computed on every GPU from the replicated u_i, and the true residual b - sum_g A_g x_g
   takes one more all-reduce of the same layout (with ||x_g||²). This call only computes
   the split: the n columns of a CSR matrix (host arrays) into nparts contiguous ranges
   holding nearly equal numbers of stored entries, each range at least one column.
   col_begin: nparts + 1 values (col_begin[0] = 0, col_begin[nparts] = n); shard_nnz:
   nparts values. TACTA_ERR_INVALID on sizes outside m, n >= 1, 1 <= nparts <= n, on
   rowptr[0] != 0 or rowptr[m] != nnz, or a column index outside [0, n). Touches no GPU. */
tacta_status tacta_column_partition(int64_t m, int64_t n, int64_t nnz, const int32_t* rowptr,
                                    const int32_t* colidx, int32_t nparts, int64_t* col_begin,
                                    int64_t* shard_nnz);

/* tacta_aux_solve -- CTA's auxiliary equation of order t (Eq. eqcoeff),
     [phi_{i+j}]_{i,j=1..t} alpha = [phi_i]_{i=1..t},
   solved on the host by the code the kernels run on the device: Jacobi scaling by
   phi_{2i}^{-1/2}, square-root-free Cholesky in natural order truncated at the first
   pivot <= pivot_tol (the minimum-norm reading of a singular system: the leading block
   is solved, the trailing alphas are 0). phi: 2t + 1 doubles (phi[0] unused);
   alpha: t doubles. Returns the order of the block solved (0..t; 0 is a breakdown), or
   -1 when t is outside 1..8 or a pointer is NULL. Touches no GPU. */
int32_t tacta_aux_solve(const double* phi, int32_t t, double pivot_tol, double* alpha);

/* tacta_dia_tile_plan -- the per-tile plan of the diagonal form the fused chain and the
   single products use for banded operands (rows x cols, k <= 5 diagonals col - row =
   offsets[0..k-1], strictly ascending), computed on the host by the code the plan-time
   kernel runs: tile `tile` (rows [256 tile, 256 tile + 256) clipped to rows) stages the
   ranges x[row + offset_i] clipped to [0, cols), aligned outwards to 4 entries and merged
   when closer than 16, laid end to end; row r of the tile reads x[r + offset_i] at slot
   sbase[i] + (r - 256 tile). Writes runs (4 {first column, length} pairs, 8 int32, unused
   pairs {0, 0}) and sbase (8 int32) and returns 1 when the tile fits (at most 4 runs of at
   most 896 entries in total), 0 when it does not (outputs untouched), -1 on invalid
   arguments. Touches no GPU. */
int32_t tacta_dia_tile_plan(int64_t rows, int64_t cols, int32_t k, const int32_t* offsets, int32_t tile,
                            int32_t* runs, int32_t* sbase);

/* Description of the last error on the calling thread ("" if none). */
const char* tacta_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int32_t tacta_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TACTA_H */

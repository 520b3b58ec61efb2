// The CTA product chain of one F_t step as one persistent launch (banded operands, on
// their diagonal form or their run-staged CSR form: the two tile formats of rowtiles.cuh).
//
// Alg. 1.1 with H = AAᵀ builds, from u_0 = r, the chain z_i = Aᵀ u_{i-1}, u_i = A z_i
// (i = 1..t) and the moments phi_{2i-1} = ||z_i||², phi_{2i} = ||u_i||² (Eq. eqcoeff).
// Each product depends on the whole previous one, so as separate launches each of
// the 2t products pays a launch ramp (every block's first copies in flight, nothing to
// multiply) and a tail (the last blocks' reduction and ticket). Here one cooperative
// launch keeps every block resident for the whole chain:
//   * every block walks the same ring of stages through all 2t products;
//   * at the end of product p each block writes its partial of phi_{p+1} and arrives
//     on a grid-wide counter; product p+1 reads p's output vector, so its x runs are
//     copied only once all G blocks have arrived (p + 1) times;
//   * the matrix part of the first tiles of product p+1 (values and the format's
//     indexing data) does not depend on the counter: the producer
//     warp issues it into the free stages before waiting, so the copies of the next
//     product are in flight while the slowest blocks finish the current one;
//   * the fused step (STEP = true) also finishes the F_t step in the same launch: after
//     the last product every block waits for all G blocks, sums the moments from the
//     per-block partials in one fixed order (so every block holds the same bits), takes
//     the step decision and solves the auxiliary equation (Eq. eqcoeff) redundantly with
//     one warp, and then updates its slice of x and r (Eqs. CTAGEN7, CTAGEN7A); the
//     last block to finish (atomic ticket) adds the ||r||² partials and runs the stop
//     tests. One launch per F_t step instead of three;
//   * without STEP the moments are summed by the step's auxiliary kernel (fixed order,
//     deterministic) and the update runs as its own launch.
// Every wait is bounded (about a second); a block that gives up sets the TIMEOUT stop
// reason, which every other waiting block polls, so the launch always ends.
#include <algorithm>
#include <cstddef>
#include <type_traits>

#include "internal.h"
#include "aux_step.cuh"
#include "finish.cuh"
#include "mbarrier.cuh"
#include "rowtiles.cuh"

namespace tacta {

// stages of the ring and resident blocks per SM (the launch bounds). The FP32 chain runs
// three blocks per SM like the FP64 one: at four its fused step (the decision and update
// code in the same kernel) spilled under the 56-register budget (1000² stencil, mixed
// precision: 13,679 against 11,925 F_t/s; five stages at three blocks 13,082)
template <typename V> struct ChainShape;
template <> struct ChainShape<double> { static constexpr int S = kRwStages, MINB = 3; };
template <> struct ChainShape<float> { static constexpr int S = kRw32Stages, MINB = 3; };

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One thread: wait until the grid-wide counter reaches `target` (all blocks arrived
// after the previous product). Gives up when another block timed out (the TIMEOUT
// stop reason; no other reason is set while a block of the launch can still wait) or
// after ctl->wait_cycles SM cycles (2^31, about a second, unless the caller asked for
// less). The proxy fence orders the bulk copies (async proxy) that follow
// after the acquire of the other blocks' plain stores.
__device__ bool grid_wait(Ctl* ctl, uint32_t target) {
    const long long t0 = clock64();
    const long long limit = ctl->wait_cycles > 0 ? ctl->wait_cycles : (1LL << 31);
    while (ld_acquire_gpu(&ctl->chain_bar) < target) {
        if (*(volatile int32_t*)&ctl->status == TACTA_REASON_TIMEOUT) return false;
        if (clock64() - t0 > limit) return false;
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return true;
}

// The update of the fused step (Eqs. CTAGEN7, CTAGEN7A) over this thread's slice:
// x += sum_j ax_j z_j, r -= sum_j al_j u_j, and the thread's sum of r_i² (FP64 chain:
// al = ax = alpha; FP32 chain: al = alpha, ax = alpha * xscale on the correction dx).
// Every thread of every block takes 16-byte chunks in a grid-wide stride; each entry's
// FMAs run in j order (as the separate update kernels do). The chain vectors were written
// by other blocks in this launch, so they are read through L2 (ld.global.cg), not the
// read-only path.
template <int T, typename V>
__device__ __forceinline__ double step_update(const StepArgs<V>& sa, const ChainVecs<V>& vec, const double* alpha) {
    constexpr int W = 16 / (int)sizeof(V);
    using VW = typename std::conditional<sizeof(V) == 8, double2, float4>::type;
    V al[T], ax[T];
#pragma unroll
    for (int j = 0; j < T; ++j) {
        al[j] = (V)alpha[j];
        ax[j] = sizeof(V) == 8 ? (V)alpha[j] : (V)(alpha[j] * (double)sa.xscale);
    }
    // the eight consumer warps of every block (two per sub-partition: the update is FP64-bound)
    const int64_t nth = (int64_t)gridDim.x * kTileRows;
    const int64_t gt = (int64_t)blockIdx.x * kTileRows + threadIdx.x;
    // x (n entries)
    const int64_t nx = sa.n / W;
    for (int64_t c = gt; c < nx; c += nth) {
        VW zv[T];
#pragma unroll
        for (int j = 0; j < T; ++j) zv[j] = __ldcg(reinterpret_cast<const VW*>(vec.z[j]) + c);
        VW xv = __ldcg(reinterpret_cast<const VW*>(sa.x) + c);
        V* xe = reinterpret_cast<V*>(&xv);
#pragma unroll
        for (int e = 0; e < W; ++e) {
            V v = xe[e];
#pragma unroll
            for (int j = 0; j < T; ++j) v = fma(ax[j], reinterpret_cast<const V*>(&zv[j])[e], v);
            xe[e] = v;
        }
        reinterpret_cast<VW*>(sa.x)[c] = xv;
    }
    for (int64_t i = nx * W + gt; i < sa.n; i += nth) {
        V v = sa.x[i];
#pragma unroll
        for (int j = 0; j < T; ++j) v = fma(ax[j], __ldcg(vec.z[j] + i), v);
        sa.x[i] = v;
    }
    // r (m entries) and its squared norm
    V acc = V(0);
    const int64_t nr = sa.m / W;
    for (int64_t c = gt; c < nr; c += nth) {
        VW uv[T];
#pragma unroll
        for (int j = 0; j < T; ++j) uv[j] = __ldcg(reinterpret_cast<const VW*>(vec.u[j]) + c);
        VW rv = __ldcg(reinterpret_cast<const VW*>(sa.r) + c);
        V* re = reinterpret_cast<V*>(&rv);
#pragma unroll
        for (int e = 0; e < W; ++e) {
            V v = re[e];
#pragma unroll
            for (int j = 0; j < T; ++j) v = fma(-al[j], reinterpret_cast<const V*>(&uv[j])[e], v);
            re[e] = v;
            acc = fma(v, v, acc);
        }
        reinterpret_cast<VW*>(sa.r)[c] = rv;
    }
    for (int64_t i = nr * W + gt; i < sa.m; i += nth) {
        V v = sa.r[i];
#pragma unroll
        for (int j = 0; j < T; ++j) v = fma(-al[j], __ldcg(vec.u[j] + i), v);
        sa.r[i] = v;
        acc = fma(v, v, acc);
    }
    return (double)acc;
}

template <typename V>
__device__ __noinline__ double step_update_t(const StepArgs<V>& sa, const ChainVecs<V>& vec, const double* alpha,
                                             int t) {
    switch (t) {
    case 1: return step_update<1, V>(sa, vec, alpha);
    case 2: return step_update<2, V>(sa, vec, alpha);
    case 3: return step_update<3, V>(sa, vec, alpha);
    case 4: return step_update<4, V>(sa, vec, alpha);
    case 5: return step_update<5, V>(sa, vec, alpha);
    case 6: return step_update<6, V>(sa, vec, alpha);
    case 7: return step_update<7, V>(sa, vec, alpha);
    default: return step_update<8, V>(sa, vec, alpha);
    }
}

__device__ __forceinline__ double chain_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double sq_acc(double s, double a) { return fma(s, s, a); }
__device__ __forceinline__ float sq_acc(float s, float a) { return fmaf(s, s, a); }

// t of F_t step k under the cycle (the host's schedule; Sec. 5.1: ping-pong 1..t_max..1)
__device__ __forceinline__ int step_order(int64_t k, int t_max, int cycle) {
    if (cycle == TACTA_CYCLE_FIXED || t_max == 1) return t_max;
    if (cycle == TACTA_CYCLE_SAWTOOTH) return 1 + (int)(k % t_max);
    const int period = 2 * t_max - 2;
    const int j = (int)(k % period);
    return j < t_max ? j + 1 : 2 * t_max - 1 - j;
}

// The fields the steps of a launch change, from a block's copy of the control block to the
// control block itself, once at the end of the launch (block 0 only; every block keeps an
// identical copy, and nothing else reads these fields while the launch runs).
__device__ __forceinline__ void publish_steps(Ctl* c, const Ctl& sc) {
    c->k = sc.k;
    c->is_true = sc.is_true;
    c->need_true = sc.need_true;
    c->rn2 = sc.rn2;
    c->db = sc.db;
    c->ref_thr = sc.ref_thr;
    c->hist_len = sc.hist_len;
    c->rank = sc.rank;
    c->enh_stop = sc.enh_stop;
    c->matvecs = sc.matvecs;
    for (int k = 0; k < kTMax; ++k) c->alpha[k] = sc.alpha[k];
    for (int k = 0; k < 2 * kTMax + 2; ++k) c->phi[k] = sc.phi[k];
    if (sc.status != 0) c->status = sc.status;
}

// The stop tests of the last step (the finisher of the separate update kernel: step
// count, history, true-residual period, residual and cap tests): every block waits for
// every block's update, adds the ||r||² partials in one fixed order and runs them on its
// copy of the control block. All threads of the block call it; false if the wait gave up.
template <typename V>
__device__ bool resolve_pending(Ctl* ctl, Ctl& sc, const StepArgs<V>& sa, int G, uint32_t base, int warp, int lane,
                                int rot, volatile int& failed) {
    if (threadIdx.x == 0 && !grid_wait(ctl, base)) {
        failed = 1;
        atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
    }
    __syncthreads();
    if (failed) return false;
    if (warp == rot) {
        const double rn2 = warp_sum_partials(sa.upart + (size_t)(sc.k & 1) * G, G);
        if (lane == 0) finish(&sc, FinArgs{FIN_CTA_UPDATE, 0, blockIdx.x == 0 ? sa.hist : nullptr}, rn2, 0.0);
    }
    __syncthreads();
    return true;
}

template <typename V, class F, bool STEP>
__global__ void __launch_bounds__(kRwThreads, ChainShape<V>::MINB)
cta_chain(typename F::Ops ops, ChainVecs<V> vec, StepArgs<V> sa, int t_arg, float scale, Ctl* ctl, double* part) {
    constexpr int S = ChainShape<V>::S;
    constexpr bool kFp64 = sizeof(V) == 8;
    using Stage = typename F::Stage;
    using Meta = typename F::Meta;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Stage* st = reinterpret_cast<Stage*>(smem_raw);
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ double red[3][kTileRows];
    __shared__ volatile int failed;
    __shared__ int stopped;
    __shared__ int decision;     // fused step: the step decision (0: update)
    __shared__ Ctl sc;           // fused step: this block's copy of the control block
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    if (tid == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kRwConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
        stopped = ctl->status != 0;
        if (!STEP && !stopped && blockIdx.x == 0) ctl->matvecs += 2 * t_arg;
    }
    if (STEP) {   // every block keeps a copy: the step decisions are taken in every block alike
        const uint64_t* src = reinterpret_cast<const uint64_t*>(ctl);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&sc);
        for (int i = tid; i < (int)(sizeof(Ctl) / 8); i += kRwThreads) dst[i] = __ldcg(src + i);
    }
    __syncthreads();
    if (stopped) return;   // every block reads the status left by the previous kernels
    // Co-resident blocks (G = blocks per SM x SMs, filled SM by SM) use different warps for
    // the one-warp work, so their FP64 chains run on different sub-partitions.
    const int rot = (int)(blockIdx.x / (unsigned)max(1, G / ChainShape<V>::MINB)) & 3;
    int q = 0;               // position of the next tile in this block's sequence of tiles
    uint32_t base = 0;       // grid-wide arrivals before the current step
    int last_use[S];         // producer: the last use of each stage
    for (int k = 0; k < S; ++k) last_use[k] = -1;
    const int nsteps = STEP ? sa.nsteps : 1;
    // FP64 fused step: the stop tests of a step (its ||r||², the iteration count, the
    // true-residual period) are taken at the next step's grid-wide wait, so that the
    // update needs no wait of its own. pending: the last step's tests are still to be
    // taken; the next step runs its chain meanwhile and is dropped if they stop the solve
    // or ask for the true residual first. Steps whose tests do not depend on ||r||² being
    // small (the period, the cap, the enhanced stop) take them before their chain.
    bool pending = false;
    int step = 0;
    while (step < nsteps) {
        if (STEP && kFp64 && pending) {
            const int kk = sc.k + 1;
            if (sc.enh_stop || (sc.R > 0 && kk % sc.R == 0) || kk >= sc.max_iter) {
                if (!resolve_pending(ctl, sc, sa, G, base, warp, lane, rot, failed)) return;
                pending = false;
                if (sc.status != 0) break;
            }
        }
        if (STEP && !kFp64 && sc.need_true) break;   // FP32 chain: the refinement runs first
        ++step;
        const int t = STEP ? step_order(sc.k + (pending ? 1 : 0), sa.t_max, sa.cycle) : t_arg;
        const int P = 2 * t;
        // FP64 fused step after a step that asked for the true residual: product p = -1 is
        // r = b - A x (on A, from x), before the chain reads r
        const int p0 = (STEP && kFp64 && sc.need_true) ? -1 : 0;
        if (warp == kRwConsumers) {
            // ---- producer: lane 0 issues, the lanes prefetch tile metadata
            Meta pend[S];
            int pend_k[S];
            for (int p = p0; p < P && !__any_sync(0xffffffffu, failed != 0); ++p) {   // one decision per warp
                const int o = p < 0 ? 1 : (p & 1);   // 0: Aᵀ (z_i = Aᵀ u_{i-1}), 1: A (u_i = A z_i; r = b - A x)
                const V* x = p < 0 ? sa.x : (p == 0 ? vec.r : (o ? vec.z[p >> 1] : vec.u[(p >> 1) - 1]));
                const int nt = ops.ntiles[o];
                // x of product p exists once every block finished p - 1 (and the previous
                // step's update, for the first product of a later pass)
                bool gated = p > p0 || step > 1;
                const uint32_t target = base + (uint32_t)(p - p0) * (uint32_t)G;
                int np = 0;
                typename F::Prefetch pf;
                for (int j = 0;; ++j) {
                    if (blockIdx.x + j * G >= nt || __any_sync(0xffffffffu, failed != 0)) break;
                    const Meta tm = pf.get(j, ops, o, G, lane);
                    if (lane == 0) {
                        const int k = q % S, u = q / S;
                        if (u > 0 && !mbar_wait_bounded(&empty[k], (uint32_t)((u - 1) & 1))) {
                            failed = 1;
                            atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
                        } else {
                            F::issue_mat(tm, st + k, &full[k], ops, o);
                            last_use[k] = u;
                            if (gated) {
                                pend[np] = tm;
                                pend_k[np] = k;
                                ++np;
                            } else {
                                F::issue_x(tm, st + k, &full[k], x);
                            }
                        }
                        if (gated && np == S) {   // every stage holds a tile waiting for its x runs
                            if (!grid_wait(ctl, target) && !failed) {
                                failed = 1;
                                atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
                            }
                            // issued even after a failure (in-bounds reads) so that every armed
                            // stage completes and the block can drain its copies
                            for (int i = 0; i < np; ++i) F::issue_x(pend[i], st + pend_k[i], &full[pend_k[i]], x);
                            np = 0;
                            gated = false;
                        }
                    }
                    ++q;
                    __syncwarp();
                }
                if (lane == 0 && np > 0) {   // fewer of this block's tiles than stages
                    if (!grid_wait(ctl, target) && !failed) {
                        failed = 1;
                        atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
                    }
                    for (int i = 0; i < np; ++i) F::issue_x(pend[i], st + pend_k[i], &full[pend_k[i]], x);
                }
                __syncwarp();
            }
            if (failed && lane == 0) {
                // a wait gave up: let every copy already issued land before the block exits
                for (int k = 0; k < S; ++k)
                    if (last_use[k] >= 0) mbar_wait_bounded(&full[k], (uint32_t)(last_use[k] & 1));
            }
        } else {
            // ---- eight consumer warps: warp w multiplies rows [32 w, 32 w + 32) of each tile
            for (int p = p0; p < P; ++p) {
                const int o = p < 0 ? 1 : (p & 1);
                V* y = p < 0 ? sa.r : (o ? vec.u[p >> 1] : vec.z[p >> 1]);
                const int nt = ops.ntiles[o];
                V acc = V(0);
                double acc1 = 0.0;   // the true residual's rᵀb
                for (int j = 0; blockIdx.x + j * G < nt; ++j, ++q) {
                    const int k = q % S;
                    bool ok = !failed && mbar_wait_bounded(&full[k], (uint32_t)((q / S) & 1));
                    ok = __all_sync(0xffffffffu, ok);   // the warp takes one path
                    if (!ok) {
                        if (lane == 0 && !failed) {
                            failed = 1;
                            atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
                        }
                        continue;
                    }
                    int row;
                    bool active;
                    V sum = F::row_dot(st + k, ops, warp, lane, row, active);
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&empty[k]);   // this warp is done with stage k
                    if (active) {
                        if constexpr (kFp64) {
                            if (p < 0) {   // r = b - A x, with ||r||² and rᵀb
                                const double bv = __ldg(sa.b + row);
                                sum = bv - sum;
                                acc1 = fma(sum, bv, acc1);
                            }
                        } else {
                            sum *= (V)scale;   // FP32 chain scale: a power of two, exact
                        }
                        y[row] = sum;
                        acc = sq_acc(sum, acc);
                    }
                }
                // product p is done in this block: its partials (phi_{p+1}; the true
                // residual's ||r||² and rᵀb), then (all but the chain-only launch's last
                // product) the block's arrival on the grid-wide counter, after every
                // consumer's stores of y (named barrier of the 256 consumer threads)
                double* sh = p < 0 ? red[2] : red[p & 1];
                sh[tid] = (double)acc;
                if (p < 0) red[1][tid] = acc1;
                asm volatile("bar.sync 1, %0;" ::"n"(kTileRows) : "memory");
                if (warp == 0) {
                    double s = sh[lane];
#pragma unroll
                    for (int i = 1; i < kRwConsumers; ++i) s += sh[lane + 32 * i];
                    s = chain_warp_sum(s);
                    double s1 = 0.0;
                    if (p < 0) {
                        s1 = red[1][lane];
#pragma unroll
                        for (int i = 1; i < kRwConsumers; ++i) s1 += red[1][lane + 32 * i];
                        s1 = chain_warp_sum(s1);
                    }
                    if (lane == 0) {
                        if (p < 0) {
                            sa.rpart[blockIdx.x] = s;
                            sa.rpart[G + blockIdx.x] = s1;
                        } else {
                            part[(size_t)p * G + blockIdx.x] = s;
                        }
                        if (STEP || p + 1 < P) {   // the fused step also counts the last product
                            asm volatile("fence.proxy.async.global;" ::: "memory");
                            __threadfence();
                            atomicAdd(&ctl->chain_bar, 1u);
                        }
                    }
                }
            }
        }
        if constexpr (!STEP) {
            break;
        } else {
            // ---- the rest of the F_t step. Every copy of this block has landed (consumers
            // waited on every armed stage; a producer that gave up drained). Every block
            // sums the moments from all blocks' partials in one fixed order, so every block
            // holds the same bits, and takes the step decision itself (a warp solves the
            // auxiliary equation): no block waits on another's decision. Then the eight
            // consumer warps update the block's slice of x and r, and the next step starts
            // in the same launch.
            base += (uint32_t)(P - p0) * (uint32_t)G;
            __syncthreads();
            if (tid == 0 && !failed && !grid_wait(ctl, base)) {
                failed = 1;
                atomicExch(&ctl->status, (int32_t)TACTA_REASON_TIMEOUT);
            }
            __syncthreads();
            if (failed) return;
            const int pw = (rot + 1) & 3;   // the warp that adds the last step's ||r||² partials
            if (p0 < 0 && warp < 2) {   // the true residual's ||r||² and rᵀb
                const double s2 = warp_sum_partials(sa.rpart + (size_t)warp * G, G);
                if (lane == 0) sc.red[warp] = s2;
            }
            if (pending && warp == pw) {
                const double s2 = warp_sum_partials(sa.upart + (size_t)(sc.k & 1) * G, G);
                if (lane == 0) sc.red[2] = s2;
            }
            sum_moment_partials(&sc, t, part, G, nullptr, 2 + rot);
            if (warp == rot) {
                int st2 = 0;
                bool go_on = true;
                if (pending) {   // the last step's stop tests (the update kernel's finisher)
                    if (lane == 0) finish(&sc, FinArgs{FIN_CTA_UPDATE, 0, blockIdx.x == 0 ? sa.hist : nullptr},
                                          sc.red[2], 0.0);
                    __syncwarp();
                    if (sc.status != 0) {
                        go_on = false;
                        st2 = sc.status;
                    } else if (sc.need_true) {   // this chain ran on the recursive residual: dropped
                        go_on = false;
                        st2 = -1;
                    }
                }
                if (go_on && p0 < 0) {   // the true residual first (as the finisher of a separate residual kernel)
                    if (lane == 0) finish(&sc, FinArgs{FIN_TRUE_RES, 0, blockIdx.x == 0 ? sa.hist : nullptr},
                                          sc.red[0], sc.red[1]);
                    __syncwarp();
                    go_on = sc.status == 0;
                    st2 = sc.status;
                }
                if (go_on) {
                    for (int i = 1; i <= 2 * t; ++i)
                        if (!finite(sc.phi[i])) st2 = TACTA_REASON_NONFINITE;
                    if (st2 == 0 && sc.phi[1] <= __dmul_rn(sc.nrm_thr, sc.cs2)) st2 = TACTA_REASON_NORMAL;
                    if (st2 == 0 && sc.enhanced && t >= 2) {
                        if (lane == 0) enhanced_stop(&sc, t);   // sets sc.enh_stop, sc.alpha
                        __syncwarp();
                    }
                    if (st2 == 0 && !sc.enh_stop) {
                        const int rank = hankel_solve_warp(sc.phi, t, sc.pivot_tol, sc.alpha);
                        if (rank == 0) st2 = TACTA_REASON_BREAKDOWN;
                        if (lane == 0) sc.rank = rank;
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    decision = st2;
                    if (st2 > 0) sc.status = st2;
                    sc.matvecs += (p0 < 0 ? 1 : 0) + (st2 >= 0 && (st2 == 0 || go_on) ? P : 0);
                }
            }
            __syncthreads();
            pending = false;
            if (decision < 0) continue;  // the true residual goes first: the next pass starts with it
            if (decision != 0) break;    // the solve ends with this step
            const double acc = warp < kRwConsumers ? step_update_t<V>(sa, vec, sc.alpha, t) : 0.0;
            // ||r||²: the block's partial, and its arrival (the next step's first product
            // waits for every block's update through it)
            const double bs = block_sum_warp0<kRwThreads>(acc, &red[0][0]);
            if (tid == 0) {
                sa.upart[(size_t)(sc.k & 1) * G + blockIdx.x] = bs;
                asm volatile("fence.proxy.async.global;" ::: "memory");
                __threadfence();
                atomicAdd(&ctl->chain_bar, 1u);
            }
            base += (uint32_t)G;
            if constexpr (kFp64) {
                pending = true;
            } else {
                // FP32 chain: the stop tests now (a refinement ends the launch)
                if (!resolve_pending(ctl, sc, sa, G, base, warp, lane, rot, failed)) return;
                if (sc.status != 0 || sc.need_true) break;
            }
        }
    }
    if constexpr (STEP) {
        if (pending && !resolve_pending(ctl, sc, sa, G, base, warp, lane, rot, failed)) return;
        if (blockIdx.x == 0 && tid == 0) publish_steps(ctl, sc);
        // every block is past its last grid-wide wait once it takes its ticket: the last one
        // resets the counters for the next launch
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            if (atomicAdd(&ctl->counter, 1u) == (uint32_t)G - 1u) {
                ctl->counter = 0;
                ctl->chain_bar = 0;
            }
        }
    }
}

template <typename V, class F>
static size_t chain_smem() { return (size_t)ChainShape<V>::S * sizeof(typename F::Stage); }

// blocks of the cooperative launch: all resident, for both the chain-only and the fused
// step kernel (the smaller of their occupancies)
template <typename V, class F>
static int chain_grid_t(int sms, int max_tiles) {
    static const char attr_key = 0;
    if (!done_on_device(&attr_key)) {
        if (cudaFuncSetAttribute(cta_chain<V, F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)chain_smem<V, F>()) != cudaSuccess ||
            cudaFuncSetAttribute(cta_chain<V, F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)chain_smem<V, F>()) != cudaSuccess)
            return 0;
        mark_done_on_device(&attr_key);
    }
    int per_sm = 0, per_sm2 = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cta_chain<V, F, false>, kRwThreads,
                                                      chain_smem<V, F>()) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, cta_chain<V, F, true>, kRwThreads,
                                                      chain_smem<V, F>()) != cudaSuccess)
        return 0;
    return std::max(0, std::min(std::min(per_sm, per_sm2) * sms, max_tiles));
}

int cta_chain_grid(int sms, int max_tiles, bool fp32, bool dia) {
    int dev = 0, coop = 0;
    int g = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop) {
        if (dia) g = fp32 ? chain_grid_t<float, DiaFmt<float>>(sms, max_tiles)
                          : chain_grid_t<double, DiaFmt<double>>(sms, max_tiles);
        else g = fp32 ? chain_grid_t<float, RunFmt<float>>(sms, max_tiles)
                      : chain_grid_t<double, RunFmt<double>>(sms, max_tiles);
    }
    (void)cudaGetLastError();   // a refused query leaves no error for the next launch to report
    return g;
}

template <typename V, class F, bool STEP>
static cudaError_t launch_chain_t(const LaunchCtx& L, const typename F::Ops& ops, const ChainVecs<V>& v,
                                  const StepArgs<V>& sa, int t, float scale, double* part, int grid) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kRwThreads);
    cfg.dynamicSmemBytes = chain_smem<V, F>();
    cfg.stream = L.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;   // all blocks resident: they wait on one another
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, cta_chain<V, F, STEP>, ops, v, sa, t, scale, L.ctl, part);
    if (L.launches) ++*L.launches;
    return e;
}

// sa == nullptr: the chain alone (the auxiliary step and the update follow as their own
// launches); else the fused step
template <typename V, class F>
static cudaError_t launch_chain_any(const LaunchCtx& L, const typename F::Ops& ops, const ChainVecs<V>& v,
                                    const StepArgs<V>* sa, int t, float scale, double* part, int grid) {
    if (sa) return launch_chain_t<V, F, true>(L, ops, v, *sa, t, scale, part, grid);
    return launch_chain_t<V, F, false>(L, ops, v, StepArgs<V>{}, t, scale, part, grid);
}

cudaError_t launch_cta_chain(const LaunchCtx& L, const ChainOps<double>& ops, const ChainVecs<double>& v, int t,
                             double* part, int grid, const StepArgs<double>* sa) {
    return launch_chain_any<double, RunFmt<double>>(L, ops, v, sa, t, 1.0f, part, grid);
}

cudaError_t launch_cta_chain32(const LaunchCtx& L, const ChainOps<float>& ops, const ChainVecs<float>& v, int t,
                               float scale, double* part, int grid, const StepArgs<float>* sa) {
    return launch_chain_any<float, RunFmt<float>>(L, ops, v, sa, t, scale, part, grid);
}

cudaError_t launch_cta_chain_dia(const LaunchCtx& L, const ChainOpsDia<double>& ops, const ChainVecs<double>& v,
                                 int t, double* part, int grid, const StepArgs<double>* sa) {
    return launch_chain_any<double, DiaFmt<double>>(L, ops, v, sa, t, 1.0f, part, grid);
}

cudaError_t launch_cta_chain_dia32(const LaunchCtx& L, const ChainOpsDia<float>& ops, const ChainVecs<float>& v,
                                   int t, float scale, double* part, int grid, const StepArgs<float>* sa) {
    return launch_chain_any<float, DiaFmt<float>>(L, ops, v, sa, t, scale, part, grid);
}

}  // namespace tacta

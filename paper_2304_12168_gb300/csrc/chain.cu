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
//   * the moments are summed from the per-block partials by the step's auxiliary
//     kernel (fixed order, deterministic), not by a last block.
// Every wait is bounded (about a second); a block that gives up sets the TIMEOUT stop
// reason, which every other waiting block polls, so the launch always ends.
#include <algorithm>
#include <cstddef>

#include "internal.h"
#include "mbarrier.cuh"
#include "rowtiles.cuh"

namespace tacta {

template <typename V> struct ChainShape;
template <> struct ChainShape<double> { static constexpr int S = kRwStages, MINB = 3; };
template <> struct ChainShape<float> { static constexpr int S = kRw32Stages, MINB = kRw32BlocksPerSM; };

__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One thread: wait until the grid-wide counter reaches `target` (all blocks arrived
// after the previous product). Gives up when the solve stops (another block's timeout)
// or after ~2^31 cycles. The proxy fence orders the bulk copies (async proxy) that
// follow after the acquire of the other blocks' plain stores.
__device__ bool grid_wait(Ctl* ctl, uint32_t target) {
    const long long t0 = clock64();
    while (ld_acquire_gpu(&ctl->chain_bar) < target) {
        if (*(volatile int32_t*)&ctl->status != 0) return false;
        if (clock64() - t0 > (1LL << 31)) return false;
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return true;
}

__device__ __forceinline__ double chain_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double sq_acc(double s, double a) { return fma(s, s, a); }
__device__ __forceinline__ float sq_acc(float s, float a) { return fmaf(s, s, a); }

template <typename V, class F>
__global__ void __launch_bounds__(kRwThreads, ChainShape<V>::MINB)
cta_chain(typename F::Ops ops, ChainVecs<V> vec, int t, float scale, Ctl* ctl, double* part) {
    constexpr int S = ChainShape<V>::S;
    using Stage = typename F::Stage;
    using Meta = typename F::Meta;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Stage* st = reinterpret_cast<Stage*>(smem_raw);
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ double red[2][kTileRows];
    __shared__ volatile int failed;
    __shared__ int stopped;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x, P = 2 * t;
    if (tid == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kRwConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
        stopped = ctl->status != 0;
        if (!stopped && blockIdx.x == 0) ctl->matvecs += P;
    }
    __syncthreads();
    if (stopped) return;   // every block reads the status left by the previous kernels

    if (warp == kRwConsumers) {
        // ---- producer: lane 0 issues, the lanes prefetch tile metadata
        int last_use[S];
        for (int k = 0; k < S; ++k) last_use[k] = -1;
        Meta pend[S];
        int pend_k[S];
        int q = 0;   // position of the next tile in this block's sequence over all products
        for (int p = 0; p < P && !__any_sync(0xffffffffu, failed != 0); ++p) {   // one decision per warp
            const int o = p & 1;   // 0: Aᵀ (z_i = Aᵀ u_{i-1}), 1: A (u_i = A z_i)
            const V* x = p == 0 ? vec.r : (o ? vec.z[p >> 1] : vec.u[(p >> 1) - 1]);
            const int nt = ops.ntiles[o];
            bool gated = p > 0;    // x of product p exists once every block finished p - 1
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
                        if (!grid_wait(ctl, (uint32_t)p * (uint32_t)G) && !failed) {
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
                if (!grid_wait(ctl, (uint32_t)p * (uint32_t)G) && !failed) {
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
        int q = 0;
        for (int p = 0; p < P; ++p) {
            const int o = p & 1;
            V* y = o ? vec.u[p >> 1] : vec.z[p >> 1];
            const int nt = ops.ntiles[o];
            V acc = V(0);
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
                    if (sizeof(V) == 4) sum *= (V)scale;   // FP32 chain scale: a power of two, exact
                    y[row] = sum;
                    acc = sq_acc(sum, acc);
                }
            }
            // product p is done in this block: its partial of phi_{p+1}, then (all but the
            // last product) the block's arrival on the grid-wide counter, after every
            // consumer's stores of y (named barrier of the 256 consumer threads)
            double* sh = red[p & 1];
            sh[tid] = (double)acc;
            asm volatile("bar.sync 1, %0;" ::"n"(kTileRows) : "memory");
            if (warp == 0) {
                double s = sh[lane];
#pragma unroll
                for (int i = 1; i < kRwConsumers; ++i) s += sh[lane + 32 * i];
                s = chain_warp_sum(s);
                if (lane == 0) {
                    part[(size_t)p * G + blockIdx.x] = s;
                    if (p + 1 < P) {
                        asm volatile("fence.proxy.async.global;" ::: "memory");
                        __threadfence();
                        atomicAdd(&ctl->chain_bar, 1u);
                    }
                }
            }
        }
    }
}

template <typename V, class F>
static size_t chain_smem() { return (size_t)ChainShape<V>::S * sizeof(typename F::Stage); }

template <typename V, class F>
static int chain_grid_t(int sms, int max_tiles) {
    static const char attr_key = 0;
    if (!done_on_device(&attr_key)) {
        if (cudaFuncSetAttribute(cta_chain<V, F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)chain_smem<V, F>()) != cudaSuccess)
            return 0;
        mark_done_on_device(&attr_key);
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cta_chain<V, F>, kRwThreads, chain_smem<V, F>()) !=
        cudaSuccess)
        return 0;
    return std::max(0, std::min(per_sm * sms, max_tiles));
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

template <typename V, class F>
static cudaError_t launch_chain_t(const LaunchCtx& L, const typename F::Ops& ops, const ChainVecs<V>& v, int t,
                                  float scale, double* part, int grid) {
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
    const cudaError_t e = cudaLaunchKernelEx(&cfg, cta_chain<V, F>, ops, v, t, scale, L.ctl, part);
    if (L.launches) ++*L.launches;
    return e;
}

cudaError_t launch_cta_chain(const LaunchCtx& L, const ChainOps<double>& ops, const ChainVecs<double>& v, int t,
                             double* part, int grid) {
    return launch_chain_t<double, RunFmt<double>>(L, ops, v, t, 1.0f, part, grid);
}

cudaError_t launch_cta_chain32(const LaunchCtx& L, const ChainOps<float>& ops, const ChainVecs<float>& v, int t,
                               float scale, double* part, int grid) {
    return launch_chain_t<float, RunFmt<float>>(L, ops, v, t, scale, part, grid);
}

cudaError_t launch_cta_chain_dia(const LaunchCtx& L, const ChainOpsDia<double>& ops, const ChainVecs<double>& v,
                                 int t, double* part, int grid) {
    return launch_chain_t<double, DiaFmt<double>>(L, ops, v, t, 1.0f, part, grid);
}

cudaError_t launch_cta_chain_dia32(const LaunchCtx& L, const ChainOpsDia<float>& ops, const ChainVecs<float>& v,
                                   int t, float scale, double* part, int grid) {
    return launch_chain_t<float, DiaFmt<float>>(L, ops, v, t, scale, part, grid);
}

}  // namespace tacta

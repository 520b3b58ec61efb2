// CTA on a small dense A held on chip: one thread-block cluster, A and Aᵀ in the
// distributed shared memory of its blocks, whole F_t steps without a kernel boundary.
//
// Alg. 1.1 with H = A Aᵀ needs, per step of order t, the chain z_i = Aᵀ u_{i-1},
// u_i = A z_i (u_0 = r) and the moments phi_{2i-1} = ||z_i||², phi_{2i} = ||u_i||²
// (Eq. eqcoeff), then the auxiliary solve and the update of x and r (Eqs. CTAGEN7,
// CTAGEN7A). For A of a few hundred rows and columns (the 256 x 256 workload: 512 KB) a
// step is a few microseconds of arithmetic, so launches, not bytes, set its pace when every
// product is its own kernel. Here the C blocks of one cluster (C = 16, or 8 where 16 does
// not launch) split A by rows and Aᵀ by rows:
//   * block c keeps rows [c mr, c mr + mr) of A and rows [c nr, c nr + nr) of Aᵀ in its
//     shared memory, and the matching slices of x, r, b and of every z_i, u_i;
//   * a product first gathers its whole input vector from the blocks' slices through
//     distributed shared memory, then every block forms its own rows of the output, one
//     warp per row (lanes stride the row, then a fixed shuffle tree), and the squared norm
//     of its rows; a cluster barrier publishes the output slices and the block partials;
//   * every block adds the C partials in rank order, so all hold the same moments, solves
//     the auxiliary equation with one warp (the same solve as the banded fused step) and
//     updates its slices; the stop tests run on every block's copy of the control block.
// The true residual b - A x every R steps is one more product from the gathered x.
#include <cooperative_groups.h>

#include <algorithm>
#include <string>

#include "internal.h"
#include "aux_step.cuh"
#include "finish.cuh"
#include "hankel.cuh"

namespace cg = cooperative_groups;

namespace tacta {
namespace {

constexpr int kDcThreads = 256;             // eight warps per block
constexpr size_t kDcSmemMax = 220 * 1024;   // dynamic shared memory a block may use

__device__ __forceinline__ int dc_step_order(int64_t k, int t_max, int cycle) {
    if (cycle == TACTA_CYCLE_FIXED || t_max == 1) return t_max;
    if (cycle == TACTA_CYCLE_SAWTOOTH) return 1 + (int)(k % t_max);
    const int period = 2 * t_max - 2;
    const int j = (int)(k % period);
    return j < t_max ? j + 1 : 2 * t_max - 1 - j;
}

// shared-memory layout of every block (the same offsets in all blocks, so that a peer's
// slice is found at the same address in its shared memory)
struct DcLayout {
    int64_t mr, nr, L;            // rows per block of A and of Aᵀ; gather length max(m, n)
    int64_t a, at, g, xo, ro, bo, z, u, part;   // offsets in doubles
    int64_t total;
    __host__ __device__ DcLayout(int64_t m, int64_t n, int C) {
        mr = (m + C - 1) / C;
        nr = (n + C - 1) / C;
        L = m > n ? m : n;
        a = 0;
        at = a + mr * n;
        g = at + nr * m;
        xo = g + L;
        ro = xo + nr;
        bo = ro + mr;
        z = bo + mr;
        u = z + (int64_t)kTMax * nr;
        part = u + (int64_t)kTMax * mr;
        total = part + 8;         // two sets of up to 3 block partials (+ padding)
    }
};

// g[0, len) = the vector whose slice of `chunk` entries block j keeps at offset `off` of
// its shared memory (all threads of the block)
__device__ __forceinline__ void dc_gather(cg::cluster_group& cl, double* sm, int64_t off, int64_t chunk, int64_t len,
                                          double* g) {
    for (int64_t j = threadIdx.x; j < len; j += kDcThreads) {
        const unsigned owner = (unsigned)(j / chunk);
        const double* peer = cl.map_shared_rank(sm + off, owner);
        g[j] = peer[j - (int64_t)owner * chunk];
    }
    __syncthreads();
}

// y[i] = sum_j M[i][j] g[j] for the block's `rows` rows of M (row-major, length len), with
// the rows' sum of squares (and, with b, y = b - M g and its dot with b) in acc / acc1 of
// thread 0 after the block reduction. One warp per row: lanes stride the row, then a fixed
// shuffle tree, so every run gives the same bits.
__device__ void dc_rows(const double* M, int64_t rows, int64_t len, const double* g, double* y, const double* b,
                        double* red, double& acc, double& acc1) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = kDcThreads / 32;
    double a0 = 0.0, a1 = 0.0;
    // rows i and i + NW together: two independent FMA chains hide the FP64 latency
    for (int64_t i = warp; i < rows; i += 2 * NW) {
        const bool two = i + NW < rows;
        const double* row0 = M + i * len;
        const double* row1 = M + (two ? i + NW : i) * len;
        double s[2] = {0.0, 0.0};
        for (int64_t j = lane; j < len; j += 32) {
            const double gj = g[j];
            s[0] = fma(row0[j], gj, s[0]);
            s[1] = fma(row1[j], gj, s[1]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s[0] += __shfl_xor_sync(0xffffffffu, s[0], o);
            s[1] += __shfl_xor_sync(0xffffffffu, s[1], o);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !two) break;
            const int64_t ri = i + h * NW;
            double v = s[h];
            if (b) {
                const double bv = b[ri];
                v = bv - v;
                a1 = fma(v, bv, a1);
            }
            if (lane == 0) y[ri] = v;
            a0 = fma(v, v, a0);
        }
    }
    // per-warp values are the same in every lane; warp 0 adds the eight in a fixed tree
    if (lane == 0) {
        red[warp] = a0;
        red[8 + warp] = a1;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double s0 = lane < NW ? red[lane] : 0.0, s1 = lane < NW ? red[8 + lane] : 0.0;
#pragma unroll
        for (int o = NW / 2; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        if (threadIdx.x == 0) {
            acc = s0;
            acc1 = s1;
        }
    }
}

// The cluster-wide sums of `k` <= 2 block partials published at part[0, k) of every block
// (after the cluster barrier that follows their writes), into out on thread 0: the same
// bits in every block.
// The remote loads run in parallel (thread j of warp 0 fetches block j's partials), the
// additions in a fixed tree.
__device__ __forceinline__ void dc_sum(cg::cluster_group& cl, const double* part, int k, double* out) {
    if (threadIdx.x < 32) {
        const unsigned j = threadIdx.x;
        double v0 = 0.0, v1 = 0.0;
        if (j < cl.num_blocks()) {
            const double* pp = cl.map_shared_rank(part, j);
            v0 = pp[0];
            if (k > 1) v1 = pp[1];
        }
        // a fixed butterfly (lanes beyond the cluster hold exact zeros): lane 0's sum has the
        // same bits in every block
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v0 += __shfl_xor_sync(0xffffffffu, v0, o);
            v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        }
        if (threadIdx.x == 0) {
            out[0] = v0;
            if (k > 1) out[1] = v1;
        }
    }
}

// Every step's decision on this block's copy sc of the control block (warp 0; the same bits
// in every block): finite moments, the normal-equation test, the enhanced stop, the
// auxiliary solve. Returns the stop reason (0: update).
__device__ int dc_decide(Ctl& sc, int t) {
    const int lane = threadIdx.x & 31;
    int st = 0;
    for (int i = 1; i <= 2 * t; ++i)
        if (!finite(sc.phi[i])) st = TACTA_REASON_NONFINITE;
    if (st == 0 && sc.phi[1] <= __dmul_rn(sc.nrm_thr, sc.cs2)) st = TACTA_REASON_NORMAL;
    if (st == 0 && sc.enhanced && t >= 2) {
        if (lane == 0) enhanced_stop(&sc, t);   // sets sc.enh_stop, sc.alpha
        __syncwarp();
    }
    if (st == 0 && !sc.enh_stop) {
        const int rank = hankel_solve_warp(sc.phi, t, sc.pivot_tol, sc.alpha);
        if (rank == 0) st = TACTA_REASON_BREAKDOWN;
        __syncwarp();
        if (lane == 0) sc.rank = rank;
    }
    return st;
}

__global__ void __launch_bounds__(kDcThreads, 1) cta_dense_cluster(DenseClusterArgs a, Ctl* ctl) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), c = (int)cl.block_rank();
    extern __shared__ __align__(16) double sm[];
    __shared__ Ctl sc;
    __shared__ double red[16];
    __shared__ double red2[kDcThreads];
    __shared__ double sums[4];
    __shared__ int decision;
    const int tid = threadIdx.x, warp = tid >> 5;
    const DcLayout Ly(a.m, a.n, C);
    const int64_t ra0 = (int64_t)c * Ly.mr, rt0 = (int64_t)c * Ly.nr;
    int64_t ma = (a.m < ra0 + Ly.mr ? a.m : ra0 + Ly.mr) - ra0;   // own rows of A
    int64_t na = (a.n < rt0 + Ly.nr ? a.n : rt0 + Ly.nr) - rt0;   // own rows of Aᵀ
    ma = ma > 0 ? ma : 0;
    na = na > 0 ? na : 0;
    double* A_ = sm + Ly.a;
    double* At_ = sm + Ly.at;
    double* g = sm + Ly.g;
    double* xo = sm + Ly.xo;
    double* ro = sm + Ly.ro;
    double* bo = sm + Ly.bo;
    double* z = sm + Ly.z;
    double* u = sm + Ly.u;
    double* part = sm + Ly.part;
    for (int64_t i = tid; i < ma * a.n; i += kDcThreads) A_[i] = __ldg(a.A + ra0 * a.n + i);
    for (int64_t i = tid; i < na * a.m; i += kDcThreads) At_[i] = __ldg(a.At + rt0 * a.m + i);
    for (int64_t i = tid; i < na; i += kDcThreads) xo[i] = a.x[rt0 + i];
    for (int64_t i = tid; i < ma; i += kDcThreads) {
        ro[i] = a.r[ra0 + i];
        bo[i] = __ldg(a.b + ra0 + i);
    }
    {
        const uint64_t* src = reinterpret_cast<const uint64_t*>(ctl);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&sc);
        for (int i = tid; i < (int)(sizeof(Ctl) / 8); i += kDcThreads) dst[i] = __ldcg(src + i);
    }
    cl.sync();
    double acc = 0.0, acc1 = 0.0;
    int par = 0;   // which of the two partial sets the next cluster sum uses
    // one product's cluster step: publish this block's partials, barrier, sum them all
    auto cluster_sum = [&](int k, double* out) {
        double* pp = part + par * 4;
        if (tid == 0) {
            pp[0] = acc;
            pp[1] = acc1;
        }
        cl.sync();
        dc_sum(cl, pp, k, out);
        __syncthreads();
        par ^= 1;
    };
    for (int step = 0; step < a.nsteps && sc.status == 0; ++step) {
        const int t = dc_step_order(sc.k, a.t_max, a.cycle);
        if (sc.need_true) {   // the true residual r = b - A x (the finisher of a residual kernel)
            dc_gather(cl, sm, Ly.xo, Ly.nr, a.n, g);
            dc_rows(A_, ma, a.n, g, ro, bo, red, acc, acc1);
            cluster_sum(2, sums);
            if (tid == 0) {
                sc.matvecs += 1;
                finish(&sc, FinArgs{FIN_TRUE_RES, 0, c == 0 ? a.hist : nullptr}, sums[0], sums[1]);
            }
            __syncthreads();
            if (sc.status != 0) break;
        }
        for (int i = 1; i <= t; ++i) {
            // z_i = Aᵀ u_{i-1} (u_0 = r), phi_{2i-1} = ||z_i||²
            dc_gather(cl, sm, i == 1 ? Ly.ro : Ly.u + (int64_t)(i - 2) * Ly.mr, Ly.mr, a.m, g);
            dc_rows(At_, na, a.m, g, z + (int64_t)(i - 1) * Ly.nr, nullptr, red, acc, acc1);
            cluster_sum(1, &sc.phi[2 * i - 1]);
            // u_i = A z_i, phi_{2i} = ||u_i||²
            dc_gather(cl, sm, Ly.z + (int64_t)(i - 1) * Ly.nr, Ly.nr, a.n, g);
            dc_rows(A_, ma, a.n, g, u + (int64_t)(i - 1) * Ly.mr, nullptr, red, acc, acc1);
            cluster_sum(1, &sc.phi[2 * i]);
        }
        if (warp == 0) {
            const int st = dc_decide(sc, t);
            if (tid == 0) {
                decision = st;
                sc.matvecs += 2 * t;
                if (st != 0) sc.status = st;
            }
        }
        __syncthreads();
        if (decision != 0) break;
        // x += sum alpha_j z_j, r -= sum alpha_j u_j on this block's slices, ||r||²
        double a0 = 0.0;
        for (int64_t i = tid; i < na; i += kDcThreads) {
            double v = xo[i];
            for (int j = 0; j < t; ++j) v = fma(sc.alpha[j], z[(int64_t)j * Ly.nr + i], v);
            xo[i] = v;
        }
        for (int64_t i = tid; i < ma; i += kDcThreads) {
            double v = ro[i];
            for (int j = 0; j < t; ++j) v = fma(-sc.alpha[j], u[(int64_t)j * Ly.mr + i], v);
            ro[i] = v;
            a0 = fma(v, v, a0);
        }
        acc = block_sum_warp0<kDcThreads>(a0, red2);
        acc1 = 0.0;
        cluster_sum(1, sums);
        if (tid == 0) finish(&sc, FinArgs{FIN_CTA_UPDATE, 0, c == 0 ? a.hist : nullptr}, sums[0], 0.0);
        __syncthreads();
    }
    for (int64_t i = tid; i < na; i += kDcThreads) a.x[rt0 + i] = xo[i];
    for (int64_t i = tid; i < ma; i += kDcThreads) a.r[ra0 + i] = ro[i];
    if (c == 0 && tid == 0) {   // the fields the steps changed
        ctl->k = sc.k;
        ctl->is_true = sc.is_true;
        ctl->need_true = sc.need_true;
        ctl->rn2 = sc.rn2;
        ctl->db = sc.db;
        ctl->ref_thr = sc.ref_thr;
        ctl->hist_len = sc.hist_len;
        ctl->rank = sc.rank;
        ctl->enh_stop = sc.enh_stop;
        ctl->matvecs = sc.matvecs;
        for (int k = 0; k < kTMax; ++k) ctl->alpha[k] = sc.alpha[k];
        for (int k = 0; k < 2 * kTMax + 2; ++k) ctl->phi[k] = sc.phi[k];
        if (sc.status != 0) ctl->status = sc.status;
    }
    cl.sync();   // no block leaves while a peer may still read its shared memory
}

}  // namespace
}  // namespace tacta

namespace tacta {

// bytes of dynamic shared memory a block of a C-block cluster needs for m x n
static size_t dc_smem(int64_t m, int64_t n, int C) {
    const DcLayout ly(m, n, C);
    return (size_t)ly.total * sizeof(double);
}

static cudaError_t dc_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* at, int64_t m, int64_t n, int C,
                             cudaStream_t s) {
    cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kDcThreads);
    cfg.dynamicSmemBytes = dc_smem(m, n, C);
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaSuccess;
}

int dense_cluster_size(int64_t m, int64_t n) {
    if (m < 1 || n < 1) return 0;
    for (int C : {16, 8}) {
        if (m < C || n < C) continue;
        const size_t smem = dc_smem(m, n, C);
        if (smem > kDcSmemMax) continue;
        if (cudaFuncSetAttribute(cta_dense_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            (C > 8 && cudaFuncSetAttribute(cta_dense_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                          cudaSuccess)) {
            (void)cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg;
        cudaLaunchAttribute at[1];
        dc_config(cfg, at, m, n, C, nullptr);
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, cta_dense_cluster, &cfg) == cudaSuccess && clusters > 0)
            return C;
        (void)cudaGetLastError();
    }
    return 0;
}

cudaError_t launch_cta_dense_cluster(const LaunchCtx& L, const DenseClusterArgs& a, int C) {
    const size_t smem = dc_smem(a.m, a.n, C);
    cudaError_t e = cudaFuncSetAttribute(cta_dense_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(cta_dense_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    dc_config(cfg, at, a.m, a.n, C, L.stream);
    e = cudaLaunchKernelEx(&cfg, cta_dense_cluster, a, L.ctl);
    if (L.launches) ++*L.launches;
    return e;
}

}  // namespace tacta

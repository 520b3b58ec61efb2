// Batched dense CTA: many independent systems A_s x_s = b_s in one persistent launch
// (the longest systems, from the second solve on, in a cluster kernel launched first:
// see batch_cta_w and plan_batch).
//
// Each block takes the next unsolved system from a queue (longest first by the previous
// solve's measured time per system; largest first on the first solve) and runs
// CTA (Alg. 1.1 with H = A_s A_sᵀ, Eqs. CTAGEN7/CTAGEN7A, auxiliary equation
// Eq. eqcoeff) on it to its own stop, then takes the next one. The chain
// z_i = Aᵀ u_{i-1}, u_i = A z_i runs in the storage precision's arithmetic (FP64,
// or FP32 for FP32 and BF16 copies of A) on a copy of A_s staged in shared memory
// when it fits (read through L2 otherwise); the moments, the centering solve and
// every stop test are FP64. With an FP32 chain the correction dx accumulates in
// FP32 and is folded into the FP64 x at each refinement, where the residual
// b - A x is recomputed in FP64 from the FP64 A_s: every R steps, once the inner
// solve has reduced the residual by kRefineEta, and whenever the recursive
// residual passes the tolerance (verify-on-pass). The chain is scaled by a power of
// two s >= ||A_s||_2 (z_i by s^-(2i-1), u_i by s^-2i): the scaled auxiliary system
// gives beta_j = s^(2j) alpha_j, and x += s^-1 sum beta_j z_j, r -= sum beta_j u_j
// (exact in binary arithmetic).
//
// The paper solves one system at a time; batching is this library's extension.
#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <queue>
#include <string>
#include <type_traits>
#include <vector>

#include "hankel.cuh"
#include "internal.h"
#include "mbarrier.cuh"

namespace cg = cooperative_groups;

namespace tacta {
namespace {

// ------------------------------------------------------------------ storage types

template <class TA> struct Elem;
template <> struct Elem<double> { using TC = double; static constexpr int V = 2; };
template <> struct Elem<float> { using TC = float; static constexpr int V = 4; };
template <> struct Elem<__nv_bfloat16> { using TC = float; static constexpr int V = 8; };

// V consecutive elements from a 16-byte aligned address, widened to the chain type
__device__ __forceinline__ void load16(const double* p, double (&o)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x;
    o[1] = v.y;
}
__device__ __forceinline__ void load16(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load16(const __nv_bfloat16* p, float (&o)[8]) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {   // bf16 -> fp32 is a 16-bit shift (exact)
        o[2 * i] = __uint_as_float(w[i] << 16);
        o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
}

__device__ __forceinline__ bool finite_d(double v) {
    return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;   // exponent not all ones
}

template <class TA> __device__ __forceinline__ TA to_store(double v);
template <> __device__ __forceinline__ double to_store<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_store<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

struct SysDesc {
    int32_t m, n, ld;      // rows, columns, padded row length of the low-precision copy
    int32_t pad_;
    int64_t a_lo;          // offset (elements) of A_s in the low-precision copy
    int64_t a64;           // offset of A_s in the FP64 copy (row-major m x n)
    int64_t b_off, x_off;  // offsets of b_s and x_s
    double s, inv_s;       // chain scale (power of two) and its inverse
};

struct BatchParams {
    double tol2, tol_n2, pivot_tol, eta2;
    int32_t max_iter, R, t_max, cycle;
    int32_t m_cap, n_cap;  // vector capacities (multiples of 8: every vector starts 16-byte aligned)
    int32_t stage_bytes;   // streamed kernel: bytes of a ring stage (the autotuner's tile size)
    int32_t nc_cap;        // cluster kernel: capacity of a block's column slice (multiple of 8)
    int64_t a_cap;         // elements of A a block can stage in shared memory
    int64_t area_bytes;    // streamed kernel: bytes of the A area (ring, or A when resident)
};

struct BatchOut {
    int32_t* iters;
    int32_t* reason;
    double* rel_res;
    int64_t* t_beg;        // per system: device clock (ns) when a block took it and when it finished
    int64_t* t_end;
};

__device__ __forceinline__ int64_t clock_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (int64_t)t;
}

__device__ __forceinline__ int schedule_dev(int k, int t_max, int cycle) {
    if (cycle == TACTA_CYCLE_FIXED || t_max == 1) return t_max;
    if (cycle == TACTA_CYCLE_SAWTOOTH) return 1 + k % t_max;
    const int period = 2 * t_max - 2;
    const int j = k % period;
    return j < t_max ? j + 1 : 2 * t_max - 1 - j;
}

// Sums of squares of chain values. An FP64 chain sums in FP64. An FP32 chain sums in
// FP32 pairs hi + lo: each square is split exactly (p = fl(v v), e = fma(v, v, -p)) and
// added by Knuth's TwoSum, whose error term goes to lo, so the pair carries about
// 2^-44 relative accuracy while every operation stays on the FP32 pipe (this GPU issues
// FP64 at a small fraction of the FP32 rate). The _rn intrinsics keep the compiler from
// contracting the split's multiply-add pairs.
template <class TC> struct SqAcc;
template <> struct SqAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s = fma(v, v, s); }
    __device__ __forceinline__ void merge(const SqAcc& o) { s += o.s; }
    __device__ __forceinline__ SqAcc shfl_xor(int o) const {
        SqAcc r;
        r.s = __shfl_xor_sync(0xffffffffu, s, o);
        return r;
    }
    __device__ __forceinline__ void put(double* slot) const { *slot = s; }
    __device__ __forceinline__ static SqAcc get(const double* slot) {
        SqAcc r;
        r.s = *slot;
        return r;
    }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct SqAcc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add_pair(float p, float e) {
        const float sm = __fadd_rn(hi, p);
        const float bv = __fsub_rn(sm, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sm, bv)), __fsub_rn(p, bv));
        hi = sm;
        lo = __fadd_rn(lo, __fadd_rn(err, e));
    }
    __device__ __forceinline__ void add(float v) {
        const float p = __fmul_rn(v, v);
        add_pair(p, __fmaf_rn(v, v, -p));
    }
    __device__ __forceinline__ void merge(const SqAcc& o) { add_pair(o.hi, o.lo); }
    __device__ __forceinline__ SqAcc shfl_xor(int o) const {
        SqAcc r;
        r.hi = __shfl_xor_sync(0xffffffffu, hi, o);
        r.lo = __shfl_xor_sync(0xffffffffu, lo, o);
        return r;
    }
    __device__ __forceinline__ void put(double* slot) const {
        *reinterpret_cast<float2*>(slot) = make_float2(hi, lo);
    }
    __device__ __forceinline__ static SqAcc get(const double* slot) {
        const float2 v = *reinterpret_cast<const float2*>(slot);
        SqAcc r;
        r.hi = v.x;
        r.lo = v.y;
        return r;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <class TC>
__device__ __forceinline__ SqAcc<TC> warp_sum_sq(SqAcc<TC> a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a.merge(a.shfl_xor(o));
    return a;
}

// block-wide sums of two accumulators (red: 2 NT/32 + 2 slots); thread 0 adds the warps'
// sums in warp order and every thread gets the FP64 totals
template <int NT, class TC>
__device__ __forceinline__ double2 block_sum_sq(SqAcc<TC> a, SqAcc<TC> b, double* red) {
    a = warp_sum_sq(a);
    b = warp_sum_sq(b);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();                       // red is free (previous readers are done)
    if (lane == 0) { a.put(red + 2 * w); b.put(red + 2 * w + 1); }
    __syncthreads();
    if (threadIdx.x == 0) {
        SqAcc<TC> ta = SqAcc<TC>::get(red), tb = SqAcc<TC>::get(red + 1);
        for (int i = 1; i < NT / 32; ++i) {
            ta.merge(SqAcc<TC>::get(red + 2 * i));
            tb.merge(SqAcc<TC>::get(red + 2 * i + 1));
        }
        red[2 * (NT / 32)] = ta.value();
        red[2 * (NT / 32) + 1] = tb.value();
    }
    __syncthreads();
    return make_double2(red[2 * (NT / 32)], red[2 * (NT / 32) + 1]);
}

// block-wide sums of two FP64 values; every thread gets the result
template <int NT>
__device__ __forceinline__ double2 block_sum2(double a, double b, double* red) {
    SqAcc<double> sa, sb;
    sa.s = a;
    sb.s = b;
    return block_sum_sq<NT, double>(sa, sb, red);
}

// out = (Aᵀ u) * scale, out and the sum of its squares
template <class TA, int NT>
__device__ SqAcc<typename Elem<TA>::TC> prod_t(const TA* A, int m, int n, int ld, const typename Elem<TA>::TC* u,
                         typename Elem<TA>::TC* out, typename Elem<TA>::TC* part, double scale) {
    using TC = typename Elem<TA>::TC;
    constexpr int V = Elem<TA>::V;
    const int CG = (n + V - 1) / V;
    const int RG = CG >= NT ? 1 : NT / CG;
    const TC sc = (TC)scale;
    SqAcc<TC> sq;
    for (int w = threadIdx.x; w < CG * RG; w += NT) {
        const int cg = w % CG, rg = w / CG;
        TC acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0;
        // four rows' loads in flight per thread (A is read through L2 when it is not staged)
        int i = rg;
        for (; i + 3 * RG < m; i += 4 * RG) {
            TC a0[V], a1[V], a2[V], a3[V];
            const TA* p = A + (int64_t)i * ld + cg * V;
            load16(p, a0);
            load16(p + (int64_t)RG * ld, a1);
            load16(p + (int64_t)2 * RG * ld, a2);
            load16(p + (int64_t)3 * RG * ld, a3);
            const TC u0 = u[i], u1 = u[i + RG], u2 = u[i + 2 * RG], u3 = u[i + 3 * RG];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                acc[v] = fma(a0[v], u0, acc[v]);
                acc[v] = fma(a1[v], u1, acc[v]);
                acc[v] = fma(a2[v], u2, acc[v]);
                acc[v] = fma(a3[v], u3, acc[v]);
            }
        }
        for (; i < m; i += RG) {
            TC a[V];
            load16(A + (int64_t)i * ld + cg * V, a);
            const TC ui = u[i];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = fma(a[v], ui, acc[v]);
        }
        if (RG == 1) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int c = cg * V + v;
                if (c < n) {
                    const TC z = acc[v] * sc;
                    out[c] = z;
                    sq.add(z);
                }
            }
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) part[rg * CG * V + cg * V + v] = acc[v];
        }
    }
    if (RG > 1) {
        __syncthreads();
        for (int c = threadIdx.x; c < n; c += NT) {
            TC acc = 0;
            for (int rg = 0; rg < RG; ++rg) acc += part[rg * CG * V + c];
            const TC z = acc * sc;
            out[c] = z;
            sq.add(z);
        }
    }
    return sq;
}

// out = (A z) * scale: LPR lanes per row (a power of two >= the row's vectors, <= 32)
template <class TA, int NT>
__device__ SqAcc<typename Elem<TA>::TC> prod_n(const TA* A, int m, int n, int ld, const typename Elem<TA>::TC* z,
                         typename Elem<TA>::TC* out, double scale) {
    using TC = typename Elem<TA>::TC;
    constexpr int V = Elem<TA>::V;
    const int CG = (n + V - 1) / V;
    int lpr = 1;
    while (lpr < CG && lpr < 32) lpr <<= 1;
    const int rpw = 32 / lpr;                       // rows per warp pass
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane / lpr, sl = lane % lpr;
    const TC sc = (TC)scale;
    SqAcc<TC> sq;
    for (int base = warp * rpw; base < m; base += (NT / 32) * rpw) {
        const int row = base + sub;
        TC acc = 0;
        if (row < m) {
            const TA* p = A + (int64_t)row * ld;
            int c = sl;
            for (; c + 3 * lpr < CG; c += 4 * lpr) {   // four loads in flight per lane
                TC a0[V], a1[V], a2[V], a3[V];
                load16(p + c * V, a0);
                load16(p + (c + lpr) * V, a1);
                load16(p + (c + 2 * lpr) * V, a2);
                load16(p + (c + 3 * lpr) * V, a3);
#pragma unroll
                for (int v = 0; v < V; ++v) acc = fma(a0[v], z[c * V + v], acc);
#pragma unroll
                for (int v = 0; v < V; ++v) acc = fma(a1[v], z[(c + lpr) * V + v], acc);
#pragma unroll
                for (int v = 0; v < V; ++v) acc = fma(a2[v], z[(c + 2 * lpr) * V + v], acc);
#pragma unroll
                for (int v = 0; v < V; ++v) acc = fma(a3[v], z[(c + 3 * lpr) * V + v], acc);
            }
            for (; c < CG; c += lpr) {
                TC a[V];
                load16(p + c * V, a);
#pragma unroll
                for (int v = 0; v < V; ++v) acc = fma(a[v], z[c * V + v], acc);
            }
        }
        for (int o = lpr >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (row < m && sl == 0) {
            const TC y = acc * sc;
            out[row] = y;
            sq.add(y);
        }
    }
    return sq;
}

// r = b - A64 x in FP64 (A64 row-major m x n); returns ||r||² and rᵀb
template <class TC, int NT>
__device__ double2 residual64(const double* __restrict__ A64, int m, int n, const double* __restrict__ b,
                              const double* x, TC* r) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sq = 0.0, rb = 0.0;
    for (int row = warp; row < m; row += NT / 32) {
        double acc = 0.0;
        const double* a = A64 + (int64_t)row * n;
        int c = lane;
        for (; c + 96 < n; c += 128) {
            const double a0 = __ldg(a + c), a1 = __ldg(a + c + 32), a2 = __ldg(a + c + 64), a3 = __ldg(a + c + 96);
            acc = fma(a0, __ldcg(x + c), acc);
            acc = fma(a1, __ldcg(x + c + 32), acc);
            acc = fma(a2, __ldcg(x + c + 64), acc);
            acc = fma(a3, __ldcg(x + c + 96), acc);
        }
        for (; c < n; c += 32) acc = fma(__ldg(a + c), __ldcg(x + c), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const double v = b[row] - acc;
            r[row] = (TC)v;
            sq = fma(v, v, sq);
            rb = fma(v, b[row], rb);
        }
    }
    return make_double2(sq, rb);
}

struct Shared {           // block-wide scalars (static shared memory)
    double red[2 * 16 + 2];
    double phi[2 * kTMax + 2];
    double beta[kTMax];
    double coef[2 * kTMax];   // the update's coefficients in the chain type (beta_j, beta_j / s)
    int32_t sys;
    int32_t rank;
    int32_t stop;
};

template <class TA, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
batch_cta(const SysDesc* __restrict__ sys, const int32_t* __restrict__ order, int count,
          const TA* __restrict__ alo, const double* __restrict__ a64, const double* __restrict__ bvec,
          double* __restrict__ xvec, BatchOut out, int32_t* queue, BatchParams P) {
    using TC = typename Elem<TA>::TC;
    __shared__ Shared S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* As = reinterpret_cast<TA*>(smem_raw);
    TC* vec = reinterpret_cast<TC*>(smem_raw + ((P.a_cap * (int64_t)sizeof(TA) + 15) & ~(int64_t)15));
    TC* r = vec;                                     // m_cap
    TC* u = r + P.m_cap;                             // t_max x m_cap
    TC* z = u + (int64_t)P.t_max * P.m_cap;          // t_max x n_cap
    TC* dx = z + (int64_t)P.t_max * P.n_cap;         // n_cap
    TC* part = dx + P.n_cap;                         // NT * V
    const int tid = threadIdx.x;

    for (;;) {
        if (tid == 0) S.sys = atomicAdd(queue, 1);
        __syncthreads();
        const int q = S.sys;
        if (q >= count) break;
        if (tid == 0) out.t_beg[order[q]] = clock_ns();
        const SysDesc d = sys[order[q]];
        const int m = d.m, n = d.n, ld = d.ld;
        const double* b = bvec + d.b_off;
        double* x = xvec + d.x_off;
        const double* A64 = a64 + d.a64;
        // stage A_s in shared memory when it fits (16-byte copies)
        const TA* A = alo + d.a_lo;
        const int64_t a_elems = (int64_t)m * ld;
        if (a_elems <= P.a_cap) {
            const int64_t nv = a_elems * (int64_t)sizeof(TA) / 16;
            const uint4* src = reinterpret_cast<const uint4*>(A);
            uint4* dst = reinterpret_cast<uint4*>(As);
            for (int64_t i = tid; i < nv; i += NT) dst[i] = __ldg(src + i);
            A = As;
        }
        // x = 0, dx = 0 (with the padding the products read), r = b
        for (int c = tid; c < n; c += NT) __stcg(x + c, 0.0);
        for (int c = tid; c < P.n_cap; c += NT) dx[c] = 0;
        for (int i = 0; i < P.t_max; ++i)
            for (int c = tid; c < P.n_cap; c += NT) z[(int64_t)i * P.n_cap + c] = 0;
        double bb = 0.0;
        for (int i = tid; i < m; i += NT) {
            r[i] = (TC)b[i];
            bb = fma(b[i], b[i], bb);
        }
        const double bn2 = block_sum2<NT>(bb, 0.0, S.red).x;   // also orders the writes above
        double nrm_thr = 0.0;
        if (P.tol_n2 > 0.0 && bn2 > 0.0) {
            const SqAcc<TC> mt = prod_t<TA, NT>(A, m, n, ld, r, z, part, 1.0);
            nrm_thr = P.tol_n2 * block_sum_sq<NT>(mt, SqAcc<TC>{}, S.red).x;
            for (int c = tid; c < n; c += NT) z[c] = 0;
        }
        double rn2 = bn2;
        bool is_true = true, need_true = false;
        int k = 0, reason = 0;
        const double res_thr = P.tol2 * bn2;
        double ref_thr = P.eta2 * bn2;
        if (bn2 == 0.0) reason = TACTA_REASON_ZERO_RHS;
        while (reason == 0) {
            if (!finite_d(rn2)) { reason = TACTA_REASON_NONFINITE; break; }
            if (rn2 <= res_thr) {
                if (is_true) { reason = TACTA_REASON_RESIDUAL; break; }
                need_true = true;
            }
            if (need_true) {   // refinement: fold dx into x, FP64 residual
                for (int c = tid; c < n; c += NT) {
                    __stcg(x + c, __ldcg(x + c) + (double)dx[c]);
                    dx[c] = 0;
                }
                __syncthreads();
                const double2 rr = residual64<TC, NT>(A64, m, n, b, x, r);
                rn2 = block_sum2<NT>(rr.x, 0.0, S.red).x;
                is_true = true;
                need_true = false;
                ref_thr = P.eta2 * rn2;
                continue;
            }
            if (k >= P.max_iter) { reason = TACTA_REASON_MAXITER; break; }
            const int t = schedule_dev(k, P.t_max, P.cycle);
            // the chain u_0 = r, z_i = Aᵀ u_{i-1} / s, u_i = A z_i / s
            const TC* uprev = r;
            for (int i = 1; i <= t; ++i) {
                TC* zi = z + (int64_t)(i - 1) * P.n_cap;
                TC* ui = u + (int64_t)(i - 1) * P.m_cap;
                const SqAcc<TC> p1 = prod_t<TA, NT>(A, m, n, ld, uprev, zi, part, d.inv_s);
                __syncthreads();   // zi complete before the product with A reads it
                const SqAcc<TC> p2 = prod_n<TA, NT>(A, m, n, ld, zi, ui, d.inv_s);
                const double2 ph = block_sum_sq<NT>(p1, p2, S.red);   // also completes ui
                if (tid == 0) {
                    S.phi[2 * i - 1] = ph.x;
                    S.phi[2 * i] = ph.y;
                }
                uprev = ui;
            }
            if (tid < 32) {   // the auxiliary solve by one warp (bit for bit the serial solve)
                __syncwarp();
                int st = 0;
                for (int i = 1; i <= 2 * t; ++i)
                    if (!finite_d(S.phi[i])) st = TACTA_REASON_NONFINITE;
                // normal-equation test on the unscaled phi_1 = s² phi~_1
                if (st == 0 && S.phi[1] * d.s * d.s <= nrm_thr) st = TACTA_REASON_NORMAL;
                if (st == 0) {
                    const int rank = hankel_solve_warp(S.phi, t, P.pivot_tol, S.beta);
                    if (rank == 0) st = TACTA_REASON_BREAKDOWN;
                    __syncwarp();
                    if (tid < t) {   // the update's coefficients, converted once
                        TC* cf = reinterpret_cast<TC*>(S.coef);
                        cf[tid] = (TC)S.beta[tid];
                        cf[kTMax + tid] = (TC)(S.beta[tid] * d.inv_s);
                    }
                }
                if (tid == 0) S.stop = st;
            }
            __syncthreads();
            if (S.stop) { reason = S.stop; break; }
            // dx += s^-1 sum beta_j z_j ; r -= sum beta_j u_j ; ||r||²
            TC bz[kTMax], bu[kTMax];
            for (int j = 0; j < t; ++j) {
                bu[j] = reinterpret_cast<const TC*>(S.coef)[j];
                bz[j] = reinterpret_cast<const TC*>(S.coef)[kTMax + j];
            }
            for (int c = tid; c < n; c += NT) {
                TC v = dx[c];
                for (int j = 0; j < t; ++j) v = fma(bz[j], z[(int64_t)j * P.n_cap + c], v);
                dx[c] = v;
            }
            SqAcc<TC> sq;
            for (int i = tid; i < m; i += NT) {
                TC v = r[i];
                for (int j = 0; j < t; ++j) v = fma(-bu[j], u[(int64_t)j * P.m_cap + i], v);
                r[i] = v;
                sq.add(v);
            }
            rn2 = block_sum_sq<NT>(sq, SqAcc<TC>{}, S.red).x;
            ++k;
            is_true = false;
            if (P.R > 0 && k % P.R == 0) need_true = true;
            else if (P.eta2 > 0.0 && rn2 <= ref_thr) need_true = true;
        }
        // exit: fold the correction and report the true residual
        double rel = 0.0;
        if (reason != TACTA_REASON_ZERO_RHS) {
            for (int c = tid; c < n; c += NT) {
                __stcg(x + c, __ldcg(x + c) + (double)dx[c]);
                dx[c] = 0;
            }
            __syncthreads();
            const double2 rr = residual64<TC, NT>(A64, m, n, b, x, r);
            rel = sqrt(block_sum2<NT>(rr.x, 0.0, S.red).x / bn2);
        }
        if (tid == 0) {
            out.iters[order[q]] = k;
            out.reason[order[q]] = reason;
            out.rel_res[order[q]] = rel;
            out.t_end[order[q]] = clock_ns();
        }
        __syncthreads();   // the next system may reuse every buffer
    }
    // launched after the cluster kernel (programmatic dependent launch): finish no
    // earlier than it, so that the stream's next operation sees every system solved
    // (returns at once when there is no such dependency)
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------------ streamed, fused kernel
//
// Same iteration as batch_cta, with the products reorganised around the reads of A:
//  * one pass over A serves both products of a chain step: for each row, the warp that
//    owns it forms u_i[row] = A[row,:] z_i / s (lanes hold the row's values in registers,
//    a shuffle reduction gives the dot product) and at once adds A[row,:]ᵀ u_i[row] / s
//    to its lanes' register accumulators of z_{i+1}; a step of order t costs t + 1
//    passes (z_1 = Aᵀ r, then u_i with z_{i+1}, the last pass u_t only) instead of 2t;
//  * A reaches shared memory by 1-D bulk copies (cp.async.bulk) of 32 KB row chunks: one
//    producer warp keeps a three-chunk ring full ("full"/"empty" mbarriers, bounded
//    waits), so tens of kilobytes are in flight per SM whatever the registers allow;
//    when A_s fits the area it is copied once and every pass reads it in place.
// Inside an iteration the consumer warps synchronise among themselves (named barrier
// 1), never with the producer, which may be waiting for a stage; the whole block meets
// only at iteration boundaries, after the producer has issued the iteration's chunks.
// Requires ceil(n / V) <= 32 JV for every system (the accumulators live in registers).

constexpr int kChunkBytes = 32 * 1024;   // default ring stage of the CUDA-core passes
constexpr int kRing = 3;

template <int NT>
__device__ __forceinline__ void consumers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

// the sums of the consumer threads' two accumulators (all NT must call; red: 2 NT/32
// slots), added in warp order by consumer thread 0, the only thread that receives them;
// a_lane0: only lane 0 of each warp holds a nonzero a (no shuffles needed for it)
template <int NT, class TC>
__device__ __forceinline__ double2 consumer_sum2(SqAcc<TC> a, bool a_lane0, SqAcc<TC> b, double* red) {
    if (!a_lane0) a = warp_sum_sq(a);
    b = warp_sum_sq(b);
    const int w = threadIdx.x >> 5;
    consumers_sync<NT>();
    if ((threadIdx.x & 31) == 0) { a.put(red + 2 * w); b.put(red + 2 * w + 1); }
    consumers_sync<NT>();
    double2 r = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        SqAcc<TC> ta = SqAcc<TC>::get(red), tb = SqAcc<TC>::get(red + 1);
        for (int i = 1; i < NT / 32; ++i) {
            ta.merge(SqAcc<TC>::get(red + 2 * i));
            tb.merge(SqAcc<TC>::get(red + 2 * i + 1));
        }
        r = make_double2(ta.value(), tb.value());
    }
    return r;
}

struct Ring {
    unsigned char* area;   // kRing stages of `stage` bytes
    uint64_t* full;
    uint64_t* empty;
    int stage;
};

// chain-vector values at V consecutive columns (16-byte aligned shared memory)
__device__ __forceinline__ void loadc(const double* p, double (&o)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x;
    o[1] = v.y;
}
__device__ __forceinline__ void loadc(const float* p, float (&o)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void loadc(const float* p, float (&o)[8]) {
    const float4 v = *reinterpret_cast<const float4*>(p), w = *reinterpret_cast<const float4*>(p + 4);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    o[4] = w.x; o[5] = w.y; o[6] = w.z; o[7] = w.w;
}

// One pass over A (consumer warps). DOT: uo = A zin * sc (returns ||uo||² in sq_u);
// else the row weights come from uin. AXPY: zo = Aᵀ u * sc (returns ||zo||² in sq_z).
// The sums of squares are valid in consumer thread 0 only.
// resident: A_s is in shared memory at Ares; else chunk q of the sequence sits in ring
// stage q % kRing. Returns false if a wait gave up.
// Each lane keeps its columns of zin in registers for the whole pass, and each warp
// takes two rows at a time (rows rr and rr + NW of the chunk), so that two dot products
// and their shuffle reductions are in flight together; slices of the register row past
// the row's end are skipped by warp-uniform branches.
template <class TA, int NW, int JV, bool DOT, bool AXPY>
__device__ bool fused_pass(const TA* Ares, bool resident, const Ring& ring, uint32_t& qseq, int m, int n, int ld,
                           int R, int nch, int n_cap, const typename Elem<TA>::TC* zin,
                           const typename Elem<TA>::TC* uin, typename Elem<TA>::TC* uo,
                           typename Elem<TA>::TC* zo, typename Elem<TA>::TC* part, double sc, double* red,
                           double& sq_u, double& sq_z) {
    using TC = typename Elem<TA>::TC;
    constexpr int V = Elem<TA>::V, NT = NW * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int CG = ld / V, CGn = (n + V - 1) / V;   // vectors per stored row; per row of A
    const TC tsc = (TC)sc;
    TC zr[JV][V];
    TC acc[JV][V];
#pragma unroll
    for (int j = 0; j < JV; ++j) {
        const int cv = lane + 32 * j;
        if (DOT && cv < CGn) {   // zin is zero from n up to its capacity, a multiple of 8
            loadc(zin + cv * V, zr[j]);
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) zr[j][v] = 0;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) acc[j][v] = 0;
    }
    SqAcc<TC> su;
    bool ok = true;
    for (int c = 0; c < nch; ++c) {
        const TA* chunk;
        int k = 0;
        if (resident) {
            chunk = Ares + (int64_t)c * R * ld;
        } else {
            k = (int)(qseq % kRing);
            if (ok) ok = mbar_wait_bounded(&ring.full[k], (qseq / kRing) & 1u);
            chunk = reinterpret_cast<const TA*>(ring.area + (size_t)k * ring.stage);
        }
        const int row0 = c * R, rows = min(R, m - row0);
        if (ok) {
            for (int rr = warp; rr < rows; rr += 2 * NW) {
                const int r1 = rr + NW;
                const bool two = r1 < rows;
                TC a0[JV][V], a1[JV][V];
#pragma unroll
                for (int j = 0; j < JV; ++j) {
                    const int cv = lane + 32 * j;
                    if (32 * j >= CG) {   // warp-uniform: this slice of the row is past its end
#pragma unroll
                        for (int v = 0; v < V; ++v) a0[j][v] = a1[j][v] = 0;
                        continue;
                    }
                    if (cv < CG) {
                        load16(chunk + (int64_t)rr * ld + cv * V, a0[j]);
                    } else {
#pragma unroll
                        for (int v = 0; v < V; ++v) a0[j][v] = 0;
                    }
                    if (two && cv < CG) {
                        load16(chunk + (int64_t)r1 * ld + cv * V, a1[j]);
                    } else {
#pragma unroll
                        for (int v = 0; v < V; ++v) a1[j][v] = 0;
                    }
                }
                TC u0, u1;
                if (DOT) {
                    TC d0 = 0, d1 = 0, e0 = 0, e1 = 0;   // two partial sums per row
#pragma unroll
                    for (int j = 0; j < JV; ++j) {
                        if (32 * j >= CG) break;   // warp-uniform
#pragma unroll
                        for (int v = 0; v < V; v += 2) {
                            d0 = fma(a0[j][v], zr[j][v], d0);
                            e0 = fma(a0[j][v + 1], zr[j][v + 1], e0);
                            d1 = fma(a1[j][v], zr[j][v], d1);
                            e1 = fma(a1[j][v + 1], zr[j][v + 1], e1);
                        }
                    }
                    d0 += e0;
                    d1 += e1;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        d0 += __shfl_xor_sync(0xffffffffu, d0, o);
                        d1 += __shfl_xor_sync(0xffffffffu, d1, o);
                    }
                    u0 = d0 * tsc;
                    u1 = two ? d1 * tsc : (TC)0;
                    if (lane == 0) {
                        uo[row0 + rr] = u0;
                        su.add(u0);
                        if (two) {
                            uo[row0 + r1] = u1;
                            su.add(u1);
                        }
                    }
                } else {
                    u0 = uin[row0 + rr];
                    u1 = two ? uin[row0 + r1] : (TC)0;
                }
                if (AXPY) {
#pragma unroll
                    for (int j = 0; j < JV; ++j) {
                        if (32 * j >= CG) break;   // warp-uniform
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[j][v] = fma(a1[j][v], u1, fma(a0[j][v], u0, acc[j][v]));
                    }
                }
            }
        }
        if (!resident) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&ring.empty[k]);   // this warp is done with the stage
            ++qseq;
        }
    }
    SqAcc<TC> sz;
    if (AXPY) {
        // zo = (sum over warps of the accumulators) * sc, in warp order (deterministic)
#pragma unroll
        for (int j = 0; j < JV; ++j) {
            const int cv = lane + 32 * j;
            if (cv < CGn) {
#pragma unroll
                for (int v = 0; v < V; ++v) part[(int64_t)warp * n_cap + cv * V + v] = acc[j][v];
            }
        }
        consumers_sync<NT>();
        for (int col = threadIdx.x; col < n; col += NT) {
            TC t = 0;
            for (int w = 0; w < NW; ++w) t += part[(int64_t)w * n_cap + col];
            t *= tsc;
            zo[col] = t;
            sz.add(t);
        }
    }
    // (the row sums of squares sit in lane 0 of each warp)
    const double2 sq = consumer_sum2<NT>(su, true, sz, red);
    sq_u = sq.x;
    sq_z = sq.y;
    return ok;
}

// ------------------------------------------------------------------ BF16 tensor-core pass
//
// The same pass with the products on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation). A 16 x 16 tile of A_s serves both products:
//  * u = A z: the tile is the MMA's A operand (ldmatrix from the staged rows) and z the
//    B operand, carried exactly as three BF16 terms z = z_hi + z_lo + z_lo2 in B's
//    columns 0..2 (an FP32 value has 24 significant bits, a BF16 term 8), so the
//    FP32 chain loses nothing to the BF16 operand;
//  * z' = Aᵀ u: the tile transposed in registers (movmatrix) is the A operand of a
//    second MMA whose B operand is u split the same way, accumulated over the rows.
// Work split: the row's 16-column tiles are divided among WG column groups of warps
// (WG a power of two, at most 8 tiles per group); the NW / WG warps of a group take
// SB consecutive 16-row blocks each per round. A round: every warp loads its tiles and
// forms its part of A z for its rows; the parts meet in shared memory (exch, double
// buffered by round parity); after one consumer barrier every warp sums them in group
// order and applies the transposed tiles it still holds in registers to the finished u.
// The stored row length ld is 8 (mod 16) elements, so the eight rows an ldmatrix reads
// fall in distinct bank groups.

constexpr int kMmaStageBytes = 40 * 1024;   // default ring stage of the tensor-core passes

struct MmaGeo {
    int KT;      // 16-column tiles of a row
    int WG;      // column groups of warps
    int KG;      // tiles per group (<= the pass's template bound)
    int KGT;     // template bound: 1, 2, 4 or 8
    int NL;      // warps per group (row lanes)
    int SB;      // row blocks per warp and round (8 / KGT)
    int R;       // rows per chunk (multiple of 16)
};

__host__ __device__ inline MmaGeo mma_geo(int n, int ld, int NW, int stage) {
    MmaGeo g{};
    g.KT = (n + 15) / 16;
    if (g.KT <= 8) {
        g.WG = 1;
        g.KGT = g.KT <= 1 ? 1 : g.KT <= 2 ? 2 : g.KT <= 4 ? 4 : 8;
    } else {
        g.WG = 2;
        while (g.WG * 8 < g.KT) g.WG *= 2;
        g.KGT = 8;
    }
    g.KG = (g.KT + g.WG - 1) / g.WG;
    g.NL = NW / g.WG;
    g.SB = 8 / g.KGT;
    const int row_bytes = ld * 2;
    const int round_rows = 16 * g.NL * g.SB;
    if (round_rows * row_bytes <= stage) {
        g.R = (stage / (round_rows * row_bytes)) * round_rows;
    } else {
        g.R = (stage / (16 * row_bytes)) * 16;
    }
    return g;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&a)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

__device__ __forceinline__ uint32_t movmatrix_t(uint32_t a) {
    uint32_t d;
    asm("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(d) : "r"(a));
    return d;
}

// term s (0, 1, 2) of the split v = hi + lo + lo2 into BF16 values, as raw bits; 0 for s > 2
__device__ __forceinline__ uint32_t split_term(float v, int s) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r1 = __fsub_rn(v, __bfloat162float(h));            // exact
    const __nv_bfloat16 l = __float2bfloat16_rn(r1);
    const __nv_bfloat16 l2 = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(l)));
    const __nv_bfloat16 t = s == 0 ? h : s == 1 ? l : l2;
    return s > 2 ? 0u : (uint32_t)__bfloat16_as_ushort(t);
}

__device__ __forceinline__ uint32_t pack2(uint32_t lo, uint32_t hi) { return lo | (hi << 16); }

// Same contract as fused_pass, for BF16 storage; KGT = G.KGT.
template <int NW, int KGT, bool DOT, bool AXPY>
__device__ bool mma_pass(const __nv_bfloat16* Ares, bool resident, const Ring& ring, uint32_t& qseq, int m, int n,
                         int ld, const MmaGeo& G, int nch, int n_cap, const float* zin, const float* uin, float* uo,
                         float* zo, float* part, float* exch, double sc, double* red, double& sq_u, double& sq_z) {
    constexpr int NT = NW * 32, SB = 8 / KGT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = warp % G.WG, l = warp / G.WG;
    const int sp = lane >> 2, q4 = lane & 3;      // B column (split term) / C row, and pair index
    const int RR = 16 * G.NL * SB;                // rows of a round
    const float tsc = (float)sc;
    // B fragments of z for this warp's tiles: rows (columns of A) 2 q4 + {0, 1} and + 8
    uint32_t bz[KGT][2];
#pragma unroll
    for (int kk = 0; kk < KGT; ++kk) {
        const int c0 = (g * G.KG + kk) * 16 + 2 * q4;
        const bool tile = DOT && kk < G.KG;
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int c = c0 + (e & 1) + (e >> 1) * 8;
            v[e] = tile && c < n ? zin[c] : 0.0f;
        }
        bz[kk][0] = pack2(split_term(v[0], sp), split_term(v[1], sp));
        bz[kk][1] = pack2(split_term(v[2], sp), split_term(v[3], sp));
    }
    float acc[KGT][4];
#pragma unroll
    for (int kk = 0; kk < KGT; ++kk)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[kk][e] = 0.0f;
    SqAcc<float> su;
    bool ok = true;
    int buf = 0;
    // this lane's ldmatrix row and column offsets within a 16 x 16 tile
    const int lrow = (lane & 7) + ((lane >> 3) & 1) * 8, lcol = (lane >> 4) * 8;
    for (int c = 0; c < nch; ++c) {
        const __nv_bfloat16* chunk;
        int k = 0;
        if (resident) {
            chunk = Ares + (int64_t)c * G.R * ld;
        } else {
            k = (int)(qseq % kRing);
            if (ok) ok = mbar_wait_bounded(&ring.full[k], (qseq / kRing) & 1u);
            chunk = reinterpret_cast<const __nv_bfloat16*>(ring.area + (size_t)k * ring.stage);
        }
        const int row0 = c * G.R, rows = min(G.R, m - row0);
        const int RBc = (rows + 15) / 16;
        // every warp runs every round (the rounds hold consumer barriers), loading nothing
        // once a wait has given up
        const int rounds = (RBc + G.NL * SB - 1) / (G.NL * SB);
        const uint32_t cbase = smem_addr(chunk);
        for (int rd = 0; rd < rounds; ++rd) {
            uint32_t af[SB][KGT][4];
            float cd[SB][4], ce[SB][4];   // A z over the even and the odd tiles (two MMA chains)
#pragma unroll
            for (int sb = 0; sb < SB; ++sb) {
                const int rb = (rd * G.NL + l) * SB + sb;
                const bool lo_ok = rb * 16 + sp < rows, hi_ok = rb * 16 + sp + 8 < rows;
#pragma unroll
                for (int e = 0; e < 4; ++e) cd[sb][e] = ce[sb][e] = 0.0f;
#pragma unroll
                for (int kk = 0; kk < KGT; ++kk) {
                    const int kt = g * G.KG + kk;
                    if (ok && rb < RBc && kk < G.KG && kt < G.KT) {
                        ldmatrix_x4(af[sb][kk],
                                    cbase + (uint32_t)(((rb * 16 + lrow) * ld + kt * 16 + lcol) * 2));
                        if (!lo_ok) { af[sb][kk][0] = 0u; af[sb][kk][2] = 0u; }   // rows past the chunk
                        if (!hi_ok) { af[sb][kk][1] = 0u; af[sb][kk][3] = 0u; }
                        if (DOT) mma_bf16((kk & 1) ? ce[sb] : cd[sb], af[sb][kk], bz[kk][0], bz[kk][1]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) af[sb][kk][e] = 0u;
                    }
                }
            }
            if (!resident && rd == rounds - 1) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&ring.empty[k]);   // the chunk's tiles are in registers
            }
            float* ex = exch + (size_t)buf * G.WG * RR;
            if (DOT) {
                // this group's part of A z for each row: (hi + lo) + lo2 columns of C
#pragma unroll
                for (int sb = 0; sb < SB; ++sb) {
                    float v0 = (cd[sb][0] + ce[sb][0]) + (cd[sb][1] + ce[sb][1]);
                    float v1 = (cd[sb][2] + ce[sb][2]) + (cd[sb][3] + ce[sb][3]);
                    v0 += __shfl_down_sync(0xffffffffu, v0, 1);
                    v1 += __shfl_down_sync(0xffffffffu, v1, 1);
                    if (q4 == 0) {
                        ex[g * RR + (l * SB + sb) * 16 + sp] = v0;
                        ex[g * RR + (l * SB + sb) * 16 + sp + 8] = v1;
                    }
                }
                consumers_sync<NT>();
            }
#pragma unroll
            for (int sb = 0; sb < SB; ++sb) {
                const int rb = (rd * G.NL + l) * SB + sb;
                if (rb >= RBc) continue;
                // u at rows 2 q4 + {0, 1} and + 8 of the block (the B fragment's K rows)
                float uv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int kr = 2 * q4 + (e & 1) + (e >> 1) * 8;
                    const int row = rb * 16 + kr;
                    float u = 0.0f;
                    if (row < rows) {
                        if (DOT) {
                            const int idx = (l * SB + sb) * 16 + kr;
                            for (int gg = 0; gg < G.WG; ++gg) u += ex[gg * RR + idx];
                            u *= tsc;
                            if (g == 0 && sp == 0) {
                                uo[row0 + row] = u;
                                su.add(u);
                            }
                        } else {
                            u = uin[row0 + row];
                        }
                    }
                    uv[e] = u;
                }
                if (AXPY) {
                    const uint32_t b0 = pack2(split_term(uv[0], sp), split_term(uv[1], sp));
                    const uint32_t b1 = pack2(split_term(uv[2], sp), split_term(uv[3], sp));
#pragma unroll
                    for (int kk = 0; kk < KGT; ++kk) {
                        const int kt = g * G.KG + kk;
                        if (kk < G.KG && kt < G.KT) {
                            const uint32_t at[4] = {movmatrix_t(af[sb][kk][0]), movmatrix_t(af[sb][kk][2]),
                                                    movmatrix_t(af[sb][kk][1]), movmatrix_t(af[sb][kk][3])};
                            mma_bf16(acc[kk], at, b0, b1);
                        }
                    }
                }
            }
            buf ^= 1;
        }
        if (!resident) ++qseq;
    }
    SqAcc<float> sz;
    if (AXPY) {
        // this warp's columns: (hi + lo) + lo2 columns of the accumulators, per row lane
#pragma unroll
        for (int kk = 0; kk < KGT; ++kk) {
            float v0 = acc[kk][0] + acc[kk][1], v1 = acc[kk][2] + acc[kk][3];
            v0 += __shfl_down_sync(0xffffffffu, v0, 1);
            v1 += __shfl_down_sync(0xffffffffu, v1, 1);
            const int kt = g * G.KG + kk;
            if (q4 == 0 && kk < G.KG && kt < G.KT) {
                const int col = kt * 16 + sp;
                if (col < n) part[(int64_t)l * n_cap + col] = v0;
                if (col + 8 < n) part[(int64_t)l * n_cap + col + 8] = v1;
            }
        }
        consumers_sync<NT>();
        for (int col = threadIdx.x; col < n; col += NT) {
            float t = 0.0f;
            for (int w = 0; w < G.NL; ++w) t += part[(int64_t)w * n_cap + col];
            t *= tsc;
            zo[col] = t;
            sz.add(t);
        }
    }
    const double2 sq = consumer_sum2<NT>(su, false, sz, red);
    sq_u = sq.x;
    sq_z = sq.y;
    return ok;
}

// the three kinds of pass of a chain step, on CUDA cores or (BF16, MMA) on the tensor cores
template <class TA, int NW, int JV, bool MMA, bool DOT, bool AXPY>
__device__ __forceinline__ bool chain_pass(const TA* Ares, bool resident, const Ring& ring, uint32_t& qseq, int m,
                                           int n, int ld, int R, const MmaGeo& G, int nch, int n_cap,
                                           const typename Elem<TA>::TC* zin, const typename Elem<TA>::TC* uin,
                                           typename Elem<TA>::TC* uo, typename Elem<TA>::TC* zo,
                                           typename Elem<TA>::TC* part, float* exch, double sc, double* red,
                                           double& sq_u, double& sq_z) {
    if constexpr (MMA) {
        switch (G.KGT) {
        case 1:
            return mma_pass<NW, 1, DOT, AXPY>(Ares, resident, ring, qseq, m, n, ld, G, nch, n_cap, zin, uin, uo, zo,
                                              part, exch, sc, red, sq_u, sq_z);
        case 2:
            return mma_pass<NW, 2, DOT, AXPY>(Ares, resident, ring, qseq, m, n, ld, G, nch, n_cap, zin, uin, uo, zo,
                                              part, exch, sc, red, sq_u, sq_z);
        case 4:
            return mma_pass<NW, 4, DOT, AXPY>(Ares, resident, ring, qseq, m, n, ld, G, nch, n_cap, zin, uin, uo, zo,
                                              part, exch, sc, red, sq_u, sq_z);
        default:
            return mma_pass<NW, 8, DOT, AXPY>(Ares, resident, ring, qseq, m, n, ld, G, nch, n_cap, zin, uin, uo, zo,
                                              part, exch, sc, red, sq_u, sq_z);
        }
    } else {
        return fused_pass<TA, NW, JV, DOT, AXPY>(Ares, resident, ring, qseq, m, n, ld, R, nch, n_cap, zin, uin, uo,
                                                 zo, part, sc, red, sq_u, sq_z);
    }
}

template <class TA, int NW, int JV, bool MMA>
__global__ void __launch_bounds__((NW + 1) * 32, 1)
batch_cta_s(const SysDesc* __restrict__ sys, const int32_t* __restrict__ order, int count,
            const TA* __restrict__ alo, const double* __restrict__ a64, const double* __restrict__ bvec,
            double* __restrict__ xvec, BatchOut out, int32_t* queue, BatchParams P, int32_t* fail_flag) {
    using TC = typename Elem<TA>::TC;
    constexpr int NT = NW * 32;              // consumer threads
    constexpr int NB = NT + 32;              // with the producer warp
    __shared__ Shared S;
    __shared__ double cred[2 * NW];
    __shared__ __align__(8) uint64_t full[kRing], empty[kRing], loaded;
    __shared__ int fail_s;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TC* vec = reinterpret_cast<TC*>(smem_raw + P.area_bytes);
    TC* r = vec;                                     // m_cap
    TC* u = r + P.m_cap;                             // t_max x m_cap
    TC* z = u + (int64_t)P.t_max * P.m_cap;          // t_max x n_cap
    TC* dx = z + (int64_t)P.t_max * P.n_cap;         // n_cap
    TC* part = dx + P.n_cap;                         // NW x n_cap
    float* exch = reinterpret_cast<float*>(part + (int64_t)NW * P.n_cap);   // MMA: 2 x 16 NW x 8
    const int kStage = P.stage_bytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool producer = warp == NW;
    const Ring ring{smem_raw, full, empty, P.stage_bytes};
    if (tid == 0) {
        for (int k = 0; k < kRing; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], NW);
        }
        mbar_init(&loaded, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_s = 0;
    }
    __syncthreads();
    uint32_t qseq = 0, loaded_phase = 0;
    for (;;) {
        if (tid == 0) S.sys = atomicAdd(queue, 1);
        __syncthreads();
        const int q = S.sys;
        if (q >= count) break;
        if (tid == 0) out.t_beg[order[q]] = clock_ns();
        if (fail_s) {   // this block stops; the system it took is reported as timed out
            if (tid == 0) {
                out.reason[order[q]] = TACTA_REASON_TIMEOUT;
                out.t_end[order[q]] = clock_ns();
            }
            break;
        }
        const SysDesc d = sys[order[q]];
        const int m = d.m, n = d.n, ld = d.ld;
        const double* b = bvec + d.b_off;
        double* x = xvec + d.x_off;
        const double* A64 = a64 + d.a64;
        const TA* Ag = alo + d.a_lo;
        const int64_t row_bytes = (int64_t)ld * (int64_t)sizeof(TA);
        const MmaGeo G = MMA ? mma_geo(n, ld, NW, kStage) : MmaGeo{};
        // CUDA-core chunks: a multiple of the 2 NW rows the consumer warps take per round
        // when the stage holds that many, so that no warp takes an extra round per chunk
        const int64_t fit = max((int64_t)1, (int64_t)kStage / row_bytes);
        const int R = MMA ? G.R : (int)(fit >= 2 * NW ? fit / (2 * NW) * (2 * NW) : fit);
        const int nch = (m + R - 1) / R;
        // (the tensor-core pass reads whole 16-row blocks)
        const bool resident = (int64_t)(MMA ? (m + 15) / 16 * 16 : m) * row_bytes <= P.area_bytes;
        const TA* Ares = reinterpret_cast<const TA*>(smem_raw);
        if (resident) {   // one copy of A_s into the area
            if (tid == NT) {
                const uint32_t bytes = (uint32_t)((int64_t)m * row_bytes);
                mbar_expect_tx(&loaded, bytes);
                bulk_g2s(smem_raw, Ag, bytes, &loaded);
            }
        }
        for (int c = tid; c < n; c += NB) __stcg(x + c, 0.0);
        for (int c = tid; c < P.n_cap; c += NB) dx[c] = 0;
        for (int i = 0; i < P.t_max; ++i)
            for (int c = tid; c < P.n_cap; c += NB) z[(int64_t)i * P.n_cap + c] = 0;
        double bb = 0.0;
        for (int i = tid; i < m; i += NB) {
            r[i] = (TC)b[i];
            bb = fma(b[i], b[i], bb);
        }
        if (resident) {
            if (!mbar_wait_bounded(&loaded, loaded_phase)) fail_s = 1;
            loaded_phase ^= 1u;
        }
        const double bn2 = block_sum2<NB>(bb, 0.0, S.red).x;
        double nrm_thr = 0.0;
        if (P.tol_n2 > 0.0 && bn2 > 0.0) {   // ||Aᵀb||² (from global memory, the slow path)
            const SqAcc<TC> mt = prod_t<TA, NB>(Ag, m, n, ld, r, z, part, 1.0);
            nrm_thr = P.tol_n2 * block_sum_sq<NB>(mt, SqAcc<TC>{}, S.red).x;
            for (int c = tid; c < n; c += NB) z[c] = 0;
        }
        double rn2 = bn2;
        bool is_true = true, need_true = false;
        int k = 0, reason = 0;
        const double res_thr = P.tol2 * bn2;
        double ref_thr = P.eta2 * bn2;
        if (bn2 == 0.0) reason = TACTA_REASON_ZERO_RHS;
        __syncthreads();
        if (fail_s) reason = TACTA_REASON_TIMEOUT;
        while (reason == 0) {
            if (!finite_d(rn2)) { reason = TACTA_REASON_NONFINITE; break; }
            if (rn2 <= res_thr) {
                if (is_true) { reason = TACTA_REASON_RESIDUAL; break; }
                need_true = true;
            }
            if (need_true) {
                for (int c = tid; c < n; c += NB) {
                    __stcg(x + c, __ldcg(x + c) + (double)dx[c]);
                    dx[c] = 0;
                }
                __syncthreads();
                const double2 rr = residual64<TC, NB>(A64, m, n, b, x, r);
                rn2 = block_sum2<NB>(rr.x, 0.0, S.red).x;
                is_true = true;
                need_true = false;
                ref_thr = P.eta2 * rn2;
                continue;
            }
            if (k >= P.max_iter) { reason = TACTA_REASON_MAXITER; break; }
            const int t = schedule_dev(k, P.t_max, P.cycle);
            if (producer) {
                if (!resident && lane == 0) {
                    // the iteration's t + 1 passes, chunk by chunk, into the ring
                    for (int pass = 0; pass <= t && !fail_s; ++pass) {
                        for (int c = 0; c < nch; ++c) {
                            const int kk = (int)(qseq % kRing);
                            const uint32_t use = qseq / kRing;
                            if (use > 0 && !mbar_wait_bounded(&empty[kk], (use - 1) & 1u)) {
                                fail_s = 1;
                                break;
                            }
                            const int row0 = c * R, rows = min(R, m - row0);
                            const uint32_t bytes = (uint32_t)((int64_t)rows * row_bytes);
                            mbar_expect_tx(&full[kk], bytes);
                            bulk_g2s(smem_raw + (size_t)kk * kStage, Ag + (int64_t)row0 * ld, bytes, &full[kk]);
                            ++qseq;
                        }
                    }
                }
                if (!resident) qseq = __shfl_sync(0xffffffffu, qseq, 0);
            } else {
                // z_1 = Aᵀ r / s ; then u_i = A z_i / s with z_{i+1} = Aᵀ u_i / s ; u_t alone
                double pu = 0.0, pz = 0.0;
                bool ok = chain_pass<TA, NW, JV, MMA, false, true>(Ares, resident, ring, qseq, m, n, ld, R, G, nch,
                                                                  P.n_cap, nullptr, r, nullptr, z, part, exch,
                                                                  d.inv_s, cred, pu, pz);
                if (tid == 0) S.phi[1] = pz;
                for (int i = 1; i <= t && ok; ++i) {
                    TC* zi = z + (int64_t)(i - 1) * P.n_cap;
                    TC* ui = u + (int64_t)(i - 1) * P.m_cap;
                    consumers_sync<NT>();   // z_i complete
                    if (i < t) {
                        ok = chain_pass<TA, NW, JV, MMA, true, true>(Ares, resident, ring, qseq, m, n, ld, R, G, nch,
                                                                    P.n_cap, zi, nullptr, ui, zi + P.n_cap, part,
                                                                    exch, d.inv_s, cred, pu, pz);
                        if (tid == 0) { S.phi[2 * i] = pu; S.phi[2 * i + 1] = pz; }
                    } else {
                        ok = chain_pass<TA, NW, JV, MMA, true, false>(Ares, resident, ring, qseq, m, n, ld, R, G,
                                                                     nch, P.n_cap, zi, nullptr, ui, nullptr, part,
                                                                     exch, d.inv_s, cred, pu, pz);
                        if (tid == 0) S.phi[2 * i] = pu;
                    }
                }
                if (!ok) fail_s = 1;
                if (warp == 0) {   // the auxiliary solve by one warp (bit for bit the serial solve)
                    __syncwarp();
                    int st = 0;
                    for (int i = 1; i <= 2 * t; ++i)
                        if (!finite_d(S.phi[i])) st = TACTA_REASON_NONFINITE;
                    if (st == 0 && S.phi[1] * d.s * d.s <= nrm_thr) st = TACTA_REASON_NORMAL;
                    if (st == 0) {
                        const int rank = hankel_solve_warp(S.phi, t, P.pivot_tol, S.beta);
                        if (rank == 0) st = TACTA_REASON_BREAKDOWN;
                        __syncwarp();
                        if (lane < t) {   // the update's coefficients, converted once
                            TC* cf = reinterpret_cast<TC*>(S.coef);
                            cf[lane] = (TC)S.beta[lane];
                            cf[kTMax + lane] = (TC)(S.beta[lane] * d.inv_s);
                        }
                    }
                    if (lane == 0) S.stop = st;
                }
            }
            __syncthreads();
            if (fail_s) { reason = TACTA_REASON_TIMEOUT; break; }
            if (S.stop) { reason = S.stop; break; }
            TC bz[kTMax], bu[kTMax];
            for (int j = 0; j < t; ++j) {
                bu[j] = reinterpret_cast<const TC*>(S.coef)[j];
                bz[j] = reinterpret_cast<const TC*>(S.coef)[kTMax + j];
            }
            for (int c = tid; c < n; c += NB) {
                TC v = dx[c];
                for (int j = 0; j < t; ++j) v = fma(bz[j], z[(int64_t)j * P.n_cap + c], v);
                dx[c] = v;
            }
            SqAcc<TC> sq;
            for (int i = tid; i < m; i += NB) {
                TC v = r[i];
                for (int j = 0; j < t; ++j) v = fma(-bu[j], u[(int64_t)j * P.m_cap + i], v);
                r[i] = v;
                sq.add(v);
            }
            rn2 = block_sum_sq<NB>(sq, SqAcc<TC>{}, S.red).x;
            ++k;
            is_true = false;
            if (P.R > 0 && k % P.R == 0) need_true = true;
            else if (P.eta2 > 0.0 && rn2 <= ref_thr) need_true = true;
        }
        double rel = 0.0;
        if (reason != TACTA_REASON_ZERO_RHS) {
            for (int c = tid; c < n; c += NB) {
                __stcg(x + c, __ldcg(x + c) + (double)dx[c]);
                dx[c] = 0;
            }
            __syncthreads();
            const double2 rr = residual64<TC, NB>(A64, m, n, b, x, r);
            rel = sqrt(block_sum2<NB>(rr.x, 0.0, S.red).x / bn2);
        }
        if (tid == 0) {
            out.iters[order[q]] = k;
            out.reason[order[q]] = reason;
            out.rel_res[order[q]] = rel;
            out.t_end[order[q]] = clock_ns();
        }
        __syncthreads();
    }
    if (fail_s && tid == NT) {
        // a wait gave up: let the chunks still in flight land before the block exits
        atomicExch(fail_flag, 1);
        const uint32_t first = qseq > (uint32_t)kRing ? qseq - (uint32_t)kRing : 0u;
        for (uint32_t qq = first; qq < qseq; ++qq) mbar_wait_bounded(&full[qq % kRing], (qq / kRing) & 1u);
        mbar_wait_bounded(&loaded, loaded_phase ^ 1u);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");   // as in batch_cta
}

// ------------------------------------------------------------------ cluster kernel for the longest systems
//
// A batch takes its slowest system's time: a system that needs the whole step budget
// runs for seconds on one block long after every other block has finished. Here the
// C blocks of a thread-block cluster (C = 2 .. 16, one block per SM) solve one such
// system together, with the same iteration as batch_cta:
//   * block c keeps rows [c mb, c mb + mb) of A_s (mb = ceil(m / C)), staged in its
//     shared memory when they fit, and the same rows of r and of every u_i;
//   * z_i = Aᵀ u_{i-1} / s: every block forms the partial product over its rows and a
//     cluster barrier publishes the partials. An FP32 chain: every block adds all C
//     partials of every column in rank order through distributed shared memory (the
//     same bits in all blocks; the partials are double-buffered, one barrier per
//     product). An FP64 chain (where every FP64 addition costs the SM's slow FP64 pipe):
//     block c adds the C partials of its columns [c nc, c nc + nc) only, in rank order,
//     and writes the sums into every block's copy of z_i; a second barrier completes it;
//   * u_i = A z_i / s: each block its own rows, from its copy of z_i (a block keeps the
//     whole current z_i and its own columns of every z_j of the step, for the update:
//     with the rest of the vectors this leaves most of the shared memory to its rows);
//   * the moments, ||r||² and the FP64 residual's norm are block partials (warp sums,
//     then the warps' sums in a fixed butterfly) that the blocks publish and add in rank
//     order, so every block holds the same FP64 values and takes the same auxiliary solve
//     and stop tests: every branch that encloses a cluster barrier depends on those
//     shared values only;
//   * x is updated in column slices; the FP64 residual b - A x reads the whole x from
//     global memory after a fence and a cluster barrier.
// Every block signals the dependent launch (the single-block kernel that takes the
// other systems) as soon as it starts, so that the clusters are placed first and that
// kernel's blocks fill the remaining SMs, and each SM a cluster leaves.
constexpr int kWideNT = 512;
constexpr int kWideMaxC = 16;

struct WideShared {
    double slot[2][2 * kTMax + 2];   // this block's published partial sums (two sets)
    double sum[2 * kTMax + 2];       // the cluster's sums of the last published set
    double wred[2 * kTMax][kWideNT / 32];   // per value: the warps' partial sums
    int32_t q;                       // the system the cluster took (rank 0 writes every block's copy)
};

template <class TA>
__global__ void __launch_bounds__(kWideNT, 1)
batch_cta_w(const SysDesc* __restrict__ sys, const int32_t* __restrict__ order, int count,
            const TA* __restrict__ alo, const double* __restrict__ a64, const double* __restrict__ bvec,
            double* __restrict__ xvec, BatchOut out, int32_t* queue, BatchParams P) {
    using TC = typename Elem<TA>::TC;
    constexpr int NT = kWideNT;
    constexpr int NW = NT / 32;
    constexpr bool kScatter = std::is_same_v<TC, double>;   // reduce-scatter, then all-gather
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), cr = (int)cl.block_rank();
    __shared__ Shared S;
    __shared__ WideShared W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* As = reinterpret_cast<TA*>(smem_raw);
    TC* vec = reinterpret_cast<TC*>(smem_raw + ((P.a_cap * (int64_t)sizeof(TA) + 15) & ~(int64_t)15));
    constexpr int kZpBufs = kScatter ? 1 : 2;
    TC* r = vec;                                     // m_cap (the block's rows)
    TC* u = r + P.m_cap;                             // t_max x m_cap
    TC* zf = u + (int64_t)P.t_max * P.m_cap;         // n_cap: the whole current z_i
    TC* zs = zf + P.n_cap;                           // t_max x nc_cap: the block's columns of every z_j
    TC* zp = zs + (int64_t)P.t_max * P.nc_cap;       // kZpBufs x n_cap: the published partial products
    TC* dx = zp + kZpBufs * (int64_t)P.n_cap;        // nc_cap: the block's columns
    TC* part = dx + P.nc_cap;                        // NT x V
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int par = 0;      // partial-product buffer of the next product (FP32 chain: two)
    int spar = 0;     // slot set of the next cluster sum

    // a block sum in two steps: the warp's sum at wred[j][warp] (no barrier) ...
    auto warp_part = [&](SqAcc<TC> a, int j) {
        a = warp_sum_sq(a);
        if (lane == 0) a.put(&W.wred[j][warp]);
    };
    // ... and, after a block barrier, values 0 .. k-1 added over the warps by a fixed
    // butterfly (warp j: value j) and published in this block's slot set spar
    auto publish = [&](int k) {
        for (int j = warp; j < k; j += NW) {
            SqAcc<TC> a = lane < NW ? SqAcc<TC>::get(&W.wred[j][lane]) : SqAcc<TC>{};
            a = warp_sum_sq(a);
            if (lane == 0) W.slot[spar][j] = a.value();
        }
    };
    // W.sum[0, k) = the cluster's sums of the k values every block published in its slot
    // set spar: warp j adds value j over the blocks by a fixed butterfly (lanes beyond the
    // cluster hold exact zeros), so every block gets the same bits
    auto cluster_sums = [&](int k) {
        cl.sync();
        for (int j = warp; j < k; j += NW) {
            double v = 0.0;
            if (lane < C) v = cl.map_shared_rank(&W.slot[spar][0], lane)[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) W.sum[j] = v;
        }
        __syncthreads();
        spar ^= 1;
    };
    // one block total (thread 0's value) published and summed over the cluster
    auto cluster_total = [&](double v) -> double {
        if (tid == 0) W.slot[spar][0] = v;
        cluster_sums(1);
        return W.sum[0];
    };
    // zf = (Aᵀ v) * scale, whole, in every block, from the blocks' partial products over
    // their rows, and the block's columns [c0, c1) also into slice (unless null); returns
    // their sum of squares
    auto full_t = [&](const TA* A, int mo, int n, int ld, const TC* v, TC* slice, double scale, int c0,
                      int c1) -> SqAcc<TC> {
        TC* mine = zp + (int64_t)par * P.n_cap;
        prod_t<TA, NT>(A, mo, n, ld, v, mine, part, 1.0);
        cl.sync();                                   // every block's partial is complete
        const TC sc = (TC)scale;
        SqAcc<TC> sq;
        if constexpr (kScatter) {
            for (int c = c0 + tid; c < c1; c += NT) {
                TC acc = 0;
#pragma unroll 4
                for (int j = 0; j < C; ++j) acc += *cl.map_shared_rank(mine + c, j);
                const TC zv = acc * sc;
#pragma unroll 4
                for (int j = 0; j < C; ++j) *cl.map_shared_rank(zf + c, j) = zv;
                if (slice) slice[c - c0] = zv;
                sq.add(zv);
            }
            cl.sync();                               // every block holds the whole zf
        } else {
            for (int c = tid; c < n; c += NT) {
                TC acc = 0;
#pragma unroll 4
                for (int j = 0; j < C; ++j) acc += *cl.map_shared_rank(mine + c, j);
                const TC zv = acc * sc;
                zf[c] = zv;
                if (c >= c0 && c < c1) {
                    if (slice) slice[c - c0] = zv;
                    sq.add(zv);
                }
            }
            __syncthreads();                         // zf complete before it is read
        }
        if constexpr (!kScatter) par ^= 1;
        return sq;
    };

    for (;;) {
        if (cr == 0 && tid == 0) {
            const int q = atomicAdd(queue, 1);
            for (int j = 0; j < C; ++j) *cl.map_shared_rank(&W.q, j) = q;
        }
        cl.sync();
        const int q = W.q;
        if (q >= count) break;
        const int s_id = order[q];
        if (cr == 0 && tid == 0) out.t_beg[s_id] = clock_ns();
        const SysDesc d = sys[s_id];
        const int m = d.m, n = d.n, ld = d.ld;
        const int mb = (m + C - 1) / C, r0 = min(m, cr * mb), mo = min(m, r0 + mb) - r0;
        const int nc = (n + C - 1) / C, c0 = min(n, cr * nc), c1 = min(n, c0 + nc);
        const double* b = bvec + d.b_off + r0;
        double* x = xvec + d.x_off;
        const double* A64 = a64 + d.a64 + (int64_t)r0 * n;
        const TA* A = alo + d.a_lo + (int64_t)r0 * ld;
        const int64_t a_elems = (int64_t)mo * ld;
        if (a_elems <= P.a_cap) {   // this block's rows in shared memory (16-byte copies)
            const int64_t nv = a_elems * (int64_t)sizeof(TA) / 16;
            const uint4* src = reinterpret_cast<const uint4*>(A);
            uint4* dst = reinterpret_cast<uint4*>(As);
            for (int64_t i = tid; i < nv; i += NT) dst[i] = __ldg(src + i);
            A = As;
        }
        for (int c = c0 + tid; c < c1; c += NT) __stcg(x + c, 0.0);
        for (int c = tid; c < P.nc_cap; c += NT) dx[c] = 0;
        for (int c = tid; c < P.n_cap; c += NT) zf[c] = 0;   // (prod_n reads the padding)
        double bb = 0.0;
        for (int i = tid; i < mo; i += NT) {
            r[i] = (TC)b[i];
            bb = fma(b[i], b[i], bb);
        }
        __threadfence();            // x = 0 is in global memory before a block reads it
        const double bn2 = cluster_total(block_sum2<NT>(bb, 0.0, S.red).x);
        double nrm_thr = 0.0;
        if (P.tol_n2 > 0.0 && bn2 > 0.0) {   // ||Aᵀ b||²
            const SqAcc<TC> mt = full_t(A, mo, n, ld, r, nullptr, 1.0, c0, c1);
            nrm_thr = P.tol_n2 * cluster_total(block_sum_sq<NT>(mt, SqAcc<TC>{}, S.red).x);
            for (int c = tid; c < n; c += NT) zf[c] = 0;
        }
        // fold dx into the block's columns of x, then r = b - A x in FP64 over the block's
        // rows (the whole x from global memory); returns the cluster's ||r||²
        auto true_residual = [&]() -> double {
            for (int c = c0 + tid; c < c1; c += NT) {
                __stcg(x + c, __ldcg(x + c) + (double)dx[c - c0]);
                dx[c - c0] = 0;
            }
            __threadfence();
            cl.sync();
            const double2 rr = residual64<TC, NT>(A64, mo, n, b, x, r);
            return cluster_total(block_sum2<NT>(rr.x, 0.0, S.red).x);
        };
        double rn2 = bn2;
        bool is_true = true, need_true = false;
        int k = 0, reason = 0;
        const double res_thr = P.tol2 * bn2;
        double ref_thr = P.eta2 * bn2;
        if (bn2 == 0.0) reason = TACTA_REASON_ZERO_RHS;
        while (reason == 0) {
            if (!finite_d(rn2)) { reason = TACTA_REASON_NONFINITE; break; }
            if (rn2 <= res_thr) {
                if (is_true) { reason = TACTA_REASON_RESIDUAL; break; }
                need_true = true;
            }
            if (need_true) {
                rn2 = true_residual();
                is_true = true;
                need_true = false;
                ref_thr = P.eta2 * rn2;
                continue;
            }
            if (k >= P.max_iter) { reason = TACTA_REASON_MAXITER; break; }
            const int t = schedule_dev(k, P.t_max, P.cycle);
            // the chain u_0 = r, z_i = Aᵀ u_{i-1} / s, u_i = A z_i / s
            const TC* uprev = r;
            for (int i = 1; i <= t; ++i) {
                TC* ui = u + (int64_t)(i - 1) * P.m_cap;
                warp_part(full_t(A, mo, n, ld, uprev, zs + (int64_t)(i - 1) * P.nc_cap, d.inv_s, c0, c1), 2 * i - 2);
                warp_part(prod_n<TA, NT>(A, mo, n, ld, zf, ui, d.inv_s), 2 * i - 1);
                __syncthreads();   // ui complete before the next product reads it
                uprev = ui;
            }
            publish(2 * t);
            cluster_sums(2 * t);
            if (tid < 32) {   // the auxiliary solve by one warp of every block (the same bits)
                if (tid < 2 * t) S.phi[tid + 1] = W.sum[tid];
                __syncwarp();
                int st = 0;
                for (int i = 1; i <= 2 * t; ++i)
                    if (!finite_d(S.phi[i])) st = TACTA_REASON_NONFINITE;
                if (st == 0 && S.phi[1] * d.s * d.s <= nrm_thr) st = TACTA_REASON_NORMAL;
                if (st == 0) {
                    const int rank = hankel_solve_warp(S.phi, t, P.pivot_tol, S.beta);
                    if (rank == 0) st = TACTA_REASON_BREAKDOWN;
                    __syncwarp();
                    if (tid < t) {
                        TC* cf = reinterpret_cast<TC*>(S.coef);
                        cf[tid] = (TC)S.beta[tid];
                        cf[kTMax + tid] = (TC)(S.beta[tid] * d.inv_s);
                    }
                }
                if (tid == 0) S.stop = st;
            }
            __syncthreads();
            if (S.stop) { reason = S.stop; break; }
            // dx += s^-1 sum beta_j z_j on the block's columns; r -= sum beta_j u_j on its rows
            TC bz[kTMax], bu[kTMax];
            for (int j = 0; j < t; ++j) {
                bu[j] = reinterpret_cast<const TC*>(S.coef)[j];
                bz[j] = reinterpret_cast<const TC*>(S.coef)[kTMax + j];
            }
            for (int c = tid; c < c1 - c0; c += NT) {
                TC v = dx[c];
                for (int j = 0; j < t; ++j) v = fma(bz[j], zs[(int64_t)j * P.nc_cap + c], v);
                dx[c] = v;
            }
            SqAcc<TC> sq;
            for (int i = tid; i < mo; i += NT) {
                TC v = r[i];
                for (int j = 0; j < t; ++j) v = fma(-bu[j], u[(int64_t)j * P.m_cap + i], v);
                r[i] = v;
                sq.add(v);
            }
            warp_part(sq, 0);
            __syncthreads();
            publish(1);
            cluster_sums(1);
            rn2 = W.sum[0];
            ++k;
            is_true = false;
            if (P.R > 0 && k % P.R == 0) need_true = true;
            else if (P.eta2 > 0.0 && rn2 <= ref_thr) need_true = true;
        }
        double rel = 0.0;
        if (reason != TACTA_REASON_ZERO_RHS) rel = sqrt(true_residual() / bn2);
        if (cr == 0 && tid == 0) {
            out.iters[s_id] = k;
            out.reason[s_id] = reason;
            out.rel_res[s_id] = rel;
            out.t_end[s_id] = clock_ns();
        }
        __syncthreads();   // the next system may reuse every buffer
    }
    cl.sync();   // no block leaves while a peer may still read its shared memory
}

// ------------------------------------------------------------------ setup kernels

// low-precision copy with padded rows; one block per system
template <class TA>
__global__ void pack_lo(const SysDesc* __restrict__ sys, const double* __restrict__ a64, TA* __restrict__ alo) {
    const SysDesc d = sys[blockIdx.x];
    const int64_t total = (int64_t)d.m * d.ld;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = (int)(e / d.ld), c = (int)(e % d.ld);
        const double v = c < d.n ? a64[d.a64 + (int64_t)i * d.n + c] : 0.0;
        alo[d.a_lo + e] = to_store<TA>(v);
    }
}

// chain scale: the smallest power of two >= sqrt(||A||_1 ||A||_inf) >= ||A||_2
__global__ void chain_scale(SysDesc* sys, const double* __restrict__ a64) {
    SysDesc& d = sys[blockIdx.x];
    __shared__ double red[2][32];
    double rmax = 0.0, cmax = 0.0;
    for (int i = threadIdx.x; i < d.m; i += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < d.n; ++c) s += fabs(a64[d.a64 + (int64_t)i * d.n + c]);
        rmax = fmax(rmax, s);
    }
    for (int c = threadIdx.x; c < d.n; c += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < d.m; ++i) s += fabs(a64[d.a64 + (int64_t)i * d.n + c]);
        cmax = fmax(cmax, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = rmax; red[1][threadIdx.x >> 5] = cmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { rmax = fmax(rmax, red[0][w]); cmax = fmax(cmax, red[1][w]); }
        rmax = fmax(rmax, red[0][0]);
        cmax = fmax(cmax, red[1][0]);
        const double bound = sqrt(rmax * cmax);
        int e = 0;
        if (bound > 0.0 && bound <= DBL_MAX) { (void)frexp(bound, &e); }
        d.s = ldexp(1.0, e);          // 2^e > bound (frexp: bound = f 2^e, f in [0.5, 1))
        d.inv_s = ldexp(1.0, -e);
    }
}

// ------------------------------------------------------------------ launch configurations

struct Config {
    int nt;            // threads per block (the streamed kernel: consumers, plus one producer warp)
    int per_sm;        // resident blocks per SM
    bool streamed;     // batch_cta_s (fused passes, bulk-copy ring) instead of batch_cta
    bool mma;          // batch_cta_s with the BF16 tensor-core passes (BF16 storage only)
    int stage_kb;      // streamed: KB per ring stage (the tile of rows a pass takes at a time)
};
constexpr Config kConfigs[] = {{128, 2, false, false, 0}, {128, 4, false, false, 0}, {256, 1, false, false, 0},
                               {256, 2, false, false, 0}, {512, 1, false, false, 0}, {256, 1, true, false, 32},
                               {256, 1, true, true, 40},  {256, 1, true, false, 16}, {256, 1, true, false, 48},
                               {256, 1, true, true, 48}};
constexpr int kDefaultConfig = 3;
constexpr int kStreamNW = 8;
// vectors of a row each lane holds in registers (FP64 2, FP32 4, BF16 8 values each):
// rows of up to 512, 1024 and 1024 columns
template <class TA> constexpr int stream_jv() { return std::is_same_v<TA, __nv_bfloat16> ? 4 : 8; }
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);

// A system's time on a C-block cluster, modelled per step as the larger of its one-block
// time / C and -- when a block's rows do not fit its shared memory -- the time to stream
// them (2 t_mean passes at kWideRowBw per SM), plus h0 + h1 C: the per-step work that
// does not shrink with C (the auxiliary solve, the cluster barriers and exchanges, the
// update) and a part that grows with the blocks to exchange with. h0 is learned from
// the clustered solves (this value before any); h1 and the bandwidth are fixed. (Fitted
// on 4096-system batches: FP64 h(8) = 17, h(16) = 21 us per step, FP32 14 / 18, BF16
// 17 / 20; FP32 rows streamed at ~40 GB/s per SM next to the single-block kernel.)
constexpr double kWideH0 = 12000.0;   // ns per step
constexpr double kWideH1 = 500.0;     // ns per step and block of the cluster
constexpr double kWideRowBw = 40.0;   // bytes per ns and SM

// the cluster kernel's share of a solve
struct WidePlan {
    int32_t systems = 0;    // the first `systems` entries of the queue order
    int32_t cluster = 0;    // blocks per cluster
    int32_t clusters = 0;   // clusters launched
    bool operator==(const WidePlan& o) const {
        return systems == o.systems && cluster == o.cluster && clusters == o.clusters;
    }
};

template <class TA>
size_t vec_bytes(const BatchParams& P, int nt) {
    using TC = typename Elem<TA>::TC;
    const int64_t v = (int64_t)P.m_cap * (1 + P.t_max) + (int64_t)P.n_cap * (1 + P.t_max) + (int64_t)nt * Elem<TA>::V;
    return (size_t)v * sizeof(TC);
}

// dynamic shared memory a block may ask for (the static Shared block and slack aside)
constexpr int64_t kBatchSmemMax = 232448 - 2048;
// the same for the cluster kernel (its static block also holds the warps' partial sums)
constexpr int64_t kWideSmemMax = 232448 - 4096;
static_assert(sizeof(Shared) + sizeof(WideShared) + 256 <= 4096, "the cluster kernel's static shared memory");

template <class TA>
void set_attrs(cudaError_t& attr) {
    auto set = [&](const void* f) {
        if (attr == cudaSuccess)
            attr = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmemMax);
    };
    set((const void*)batch_cta_s<TA, kStreamNW, stream_jv<TA>(), false>);
    if constexpr (std::is_same_v<TA, __nv_bfloat16>)
        set((const void*)batch_cta_s<TA, kStreamNW, stream_jv<TA>(), true>);
    set((const void*)batch_cta<TA, 128, 2>);
    set((const void*)batch_cta<TA, 128, 4>);
    set((const void*)batch_cta<TA, 256, 1>);
    set((const void*)batch_cta<TA, 256, 2>);
    set((const void*)batch_cta<TA, 512, 1>);
    if (attr == cudaSuccess)
        attr = cudaFuncSetAttribute((const void*)batch_cta_w<TA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kWideSmemMax);
    if (attr == cudaSuccess)   // clusters of 16 blocks
        attr = cudaFuncSetAttribute((const void*)batch_cta_w<TA>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

cudaError_t prepare_kernels() {
    static const char done_key = 0;   // the attributes are per device
    if (done_on_device(&done_key)) return cudaSuccess;
    cudaError_t attr = cudaSuccess;
    set_attrs<double>(attr);
    set_attrs<float>(attr);
    set_attrs<__nv_bfloat16>(attr);
    if (attr == cudaSuccess) mark_done_on_device(&done_key);
    return attr;
}

// a launch, optionally as a programmatic dependent of the previous kernel in the stream
template <class... KArgs, class... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), int grid, int threads, size_t smem, cudaStream_t s, bool pdl,
                     Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    if (pdl) {
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <class TA>
cudaError_t launch_cfg(int cfg, cudaStream_t s, int grid, size_t smem, bool pdl, const SysDesc* sys,
                       const int32_t* order, int count, const void* alo, const double* a64, const double* b,
                       double* x, BatchOut o, int32_t* queue, const BatchParams& P, int32_t* fail_flag) {
    const TA* a = reinterpret_cast<const TA*>(alo);
    const int stream_threads = kStreamNW * 32 + 32;
    switch (cfg) {
    case 5:
    case 7:
    case 8:
        return launch_k(batch_cta_s<TA, kStreamNW, stream_jv<TA>(), false>, grid, stream_threads, smem, s, pdl, sys,
                        order, count, a, a64, b, x, o, queue, P, fail_flag);
    case 6:
    case 9:
        if constexpr (std::is_same_v<TA, __nv_bfloat16>) {
            return launch_k(batch_cta_s<TA, kStreamNW, stream_jv<TA>(), true>, grid, stream_threads, smem, s, pdl,
                            sys, order, count, a, a64, b, x, o, queue, P, fail_flag);
        } else {
            return cudaErrorInvalidConfiguration;   // make_params admits it for BF16 storage only
        }
    case 0: return launch_k(batch_cta<TA, 128, 2>, grid, 128, smem, s, pdl, sys, order, count, a, a64, b, x, o, queue, P);
    case 1: return launch_k(batch_cta<TA, 128, 4>, grid, 128, smem, s, pdl, sys, order, count, a, a64, b, x, o, queue, P);
    case 2: return launch_k(batch_cta<TA, 256, 1>, grid, 256, smem, s, pdl, sys, order, count, a, a64, b, x, o, queue, P);
    case 3: return launch_k(batch_cta<TA, 256, 2>, grid, 256, smem, s, pdl, sys, order, count, a, a64, b, x, o, queue, P);
    default:
        return launch_k(batch_cta<TA, 512, 1>, grid, 512, smem, s, pdl, sys, order, count, a, a64, b, x, o, queue, P);
    }
}

// the cluster kernel: `clusters` clusters of C blocks over the first `count` entries of order
template <class TA>
cudaError_t launch_wide(int C, int clusters, size_t smem, cudaStream_t s, const SysDesc* sys, const int32_t* order,
                        int count, const void* alo, const double* a64, const double* b, double* x, BatchOut o,
                        int32_t* queue, const BatchParams& P) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(C * clusters));
    cfg.blockDim = dim3(kWideNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, batch_cta_w<TA>, sys, order, count, reinterpret_cast<const TA*>(alo), a64, b, x,
                              o, queue, P);
}

// clusters of C blocks of the cluster kernel that can be resident at once (0: none)
template <class TA>
int wide_max_clusters(int C, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kWideNT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, batch_cta_w<TA>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace
}  // namespace tacta

// ================================================================== C ABI

using namespace tacta;

struct tacta_batch_s {
    int device = 0, sms = 0;
    int32_t count = 0;
    int32_t storage = TACTA_BATCH_FP32;
    int32_t m_max = 0, n_max = 0;
    int64_t a64_len = 0, alo_len = 0, b_len = 0, x_len = 0;
    SysDesc* sys = nullptr;
    int32_t* order = nullptr;
    double* a64 = nullptr;
    void* alo = nullptr;
    double* b = nullptr;
    double* x = nullptr;
    int32_t* iters = nullptr;
    int32_t* reason = nullptr;
    double* rel = nullptr;
    int32_t* queue = nullptr;
    int64_t* stamps = nullptr;     // 2 x count: per-system begin and end clocks of the last solve
    std::vector<int32_t> last_iters;   // host: every system's step count in the last full solve
    std::vector<int32_t> ord;          // host copy of the queue order
    std::vector<int32_t> m_of, n_of;   // per system: rows, columns
    std::vector<double> dur;           // per system: predicted time (ns) on one block of the configuration
    std::vector<char> dur_meas;        // per system: dur was measured on one block (not derived)
    double wide_h0 = -1.0;            // learned per-step overhead of a cluster (ns; < 0: none yet)
    int32_t wide_mode = -1;            // cluster kernel: -1 planned, 0 off, > 0 that many systems
    int32_t wide_cluster = 0, wide_clusters = 0;   // asked for with wide_mode > 0 (0: chosen)
    WidePlan plan;                     // the cluster kernel's share of the next solve
    WidePlan graph_plan;
    int config = -1;               // index into kConfigs (-1: default)
    cudaGraphExec_t graph = nullptr;
    int graph_key = -1;
    BatchParams graph_params{};
};

namespace {

thread_local std::string g_batch_err;

void free_batch(tacta_batch_s* B) {
    if (!B) return;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    cudaFree(B->sys); cudaFree(B->order); cudaFree(B->a64); cudaFree(B->alo); cudaFree(B->b); cudaFree(B->x);
    cudaFree(B->iters); cudaFree(B->reason); cudaFree(B->rel); cudaFree(B->queue);
    cudaFree(B->stamps);
    delete B;
}

size_t elem_size(int storage) {
    return storage == TACTA_BATCH_FP64 ? 8 : storage == TACTA_BATCH_FP32 ? 4 : 2;
}

template <class TA>
int chain_size() { return (int)sizeof(typename Elem<TA>::TC); }

// launch parameters of configuration cfg; false when it cannot run this batch
// the iteration's parameters, shared by every kernel
BatchParams base_params(const tacta_batch_s* B, const tacta_options& o) {
    BatchParams P{};
    P.tol2 = o.tol * o.tol;
    P.tol_n2 = o.tol_normal > 0.0 ? o.tol_normal * o.tol_normal : 0.0;
    P.pivot_tol = o.pivot_tol > 0.0 ? o.pivot_tol : (B->storage == TACTA_BATCH_FP64 ? 1e-12 : 1e-6);
    P.eta2 = B->storage == TACTA_BATCH_FP64 ? 0.0 : kRefineEta2;
    P.max_iter = o.max_iter;
    P.R = o.recompute_every;
    P.t_max = o.t_max;
    P.cycle = o.cycle;
    return P;
}

bool make_params(const tacta_batch_s* B, const tacta_options& o, int cfg, BatchParams* out, size_t* smem_out) {
    const Config C = kConfigs[cfg];
    BatchParams P = base_params(B, o);
    P.m_cap = (B->m_max + 7) & ~7;
    P.n_cap = (B->n_max + 7) & ~7;
    const int V = B->storage == TACTA_BATCH_FP64 ? 2 : B->storage == TACTA_BATCH_FP32 ? 4 : 8;
    const int tc = B->storage == TACTA_BATCH_FP64 ? 8 : 4;
    // shared memory per block: what per_sm blocks can share of the SM's 228 KB
    // (1 KB per block reserved, the static shared block and slack)
    const int64_t per_block = std::min<int64_t>(kBatchSmemMax, (228 * 1024) / C.per_sm - 1024 - 2048);
    const int64_t chain = ((int64_t)P.m_cap + P.n_cap) * (1 + P.t_max);
    if (!C.streamed) {
        const int64_t vb = (chain + (int64_t)C.nt * V) * tc;
        const int64_t a_bytes = std::max<int64_t>(0, per_block - vb - 16);
        P.a_cap = (a_bytes / 16) * 16 / (int64_t)elem_size(B->storage);
        P.area_bytes = 0;
        *smem_out = (size_t)(((P.a_cap * (int64_t)elem_size(B->storage) + 15) & ~15) + vb);
    } else {
        if (C.mma && (B->storage != TACTA_BATCH_BF16 || B->n_max > 1024)) return false;
        const int jv = B->storage == TACTA_BATCH_FP64 ? stream_jv<double>() : B->storage == TACTA_BATCH_FP32
                                                                              ? stream_jv<float>()
                                                                              : stream_jv<__nv_bfloat16>();
        if (P.n_cap / V > 32 * jv) return false;                 // row slices must fit the registers
        const int64_t part = std::max<int64_t>((int64_t)kStreamNW * P.n_cap, (int64_t)(C.nt + 32) * V);
        const int64_t exch = C.mma ? 2 * 16 * kStreamNW * 8 : 0;
        const int64_t vb = (chain + part + exch) * tc;
        const int64_t area = ((per_block - vb) / 16) * 16;
        const int64_t stage = (int64_t)C.stage_kb * 1024;
        if (area < (int64_t)kRing * stage) return false;
        P.stage_bytes = (int32_t)stage;
        P.area_bytes = area;
        P.a_cap = 0;
        *smem_out = (size_t)(area + vb);
    }
    if ((int64_t)*smem_out > kBatchSmemMax) return false;
    *out = P;
    return true;
}

// launch parameters of the cluster kernel with C-block clusters; false when the largest
// system's vectors do not fit a block's shared memory
bool wide_params(const tacta_batch_s* B, const tacta_options& o, int C, BatchParams* out, size_t* smem_out) {
    if (C < 1 || C > kWideMaxC) return false;
    BatchParams P = base_params(B, o);
    P.m_cap = ((B->m_max + C - 1) / C + 7) & ~7;   // a block's rows
    P.n_cap = (B->n_max + 7) & ~7;
    P.nc_cap = ((B->n_max + C - 1) / C + 7) & ~7;  // a block's columns
    const int V = B->storage == TACTA_BATCH_FP64 ? 2 : B->storage == TACTA_BATCH_FP32 ? 4 : 8;
    const int tc = B->storage == TACTA_BATCH_FP64 ? 8 : 4;
    const int64_t es = (int64_t)elem_size(B->storage);
    const int zp_bufs = B->storage == TACTA_BATCH_FP64 ? 1 : 2;   // the kernel's kZpBufs
    const int64_t vb = ((int64_t)P.m_cap * (1 + P.t_max) + (int64_t)P.n_cap * (1 + zp_bufs) +
                        (int64_t)P.nc_cap * (1 + P.t_max) + (int64_t)kWideNT * V) * tc;
    const int64_t a_bytes = kWideSmemMax - vb - 16;
    if (a_bytes < 0) return false;
    P.a_cap = (a_bytes / 16) * 16 / es;
    *smem_out = (size_t)(((P.a_cap * es + 15) & ~15) + vb);
    if ((int64_t)*smem_out > kWideSmemMax) return false;
    *out = P;
    return true;
}

int wide_max_clusters_for(const tacta_batch_s* B, int C, size_t smem) {
    switch (B->storage) {
    case TACTA_BATCH_FP64: return wide_max_clusters<double>(C, smem);
    case TACTA_BATCH_FP32: return wide_max_clusters<float>(C, smem);
    default: return wide_max_clusters<__nv_bfloat16>(C, smem);
    }
}

// One solve: the queue reset, then (plan.systems > 0) the cluster kernel on the first
// plan.systems entries of the queue order, and the single-block kernel of configuration
// cfg on the rest -- a programmatic dependent launch, so that its blocks start once every
// cluster is placed and take the remaining SMs, and each SM a cluster leaves.
cudaError_t launch_batch(tacta_batch_s* B, cudaStream_t s, const tacta_options& o, int cfg, const WidePlan& plan) {
    const Config C = kConfigs[cfg];
    size_t smem = 0;
    BatchParams P{};
    if (!make_params(B, o, cfg, &P, &smem)) return cudaErrorInvalidConfiguration;
    const int K = std::min(std::max(plan.systems, 0), B->count);
    const int rest = B->count - K;
    const int grid = std::max(1, std::min(rest, B->sms * C.per_sm));
    BatchOut out{B->iters, B->reason, B->rel, B->stamps, B->stamps + B->count};
    // queue heads of the two kernels and the timeout flag
    cudaError_t e = cudaMemsetAsync(B->queue, 0, 4 * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if (K > 0) {
        BatchParams Pw{};
        size_t smw = 0;
        if (!wide_params(B, o, plan.cluster, &Pw, &smw) || plan.clusters < 1) return cudaErrorInvalidConfiguration;
        switch (B->storage) {
        case TACTA_BATCH_FP64:
            e = launch_wide<double>(plan.cluster, plan.clusters, smw, s, B->sys, B->order, K, B->alo, B->a64, B->b,
                                    B->x, out, B->queue + 2, Pw);
            break;
        case TACTA_BATCH_FP32:
            e = launch_wide<float>(plan.cluster, plan.clusters, smw, s, B->sys, B->order, K, B->alo, B->a64, B->b,
                                   B->x, out, B->queue + 2, Pw);
            break;
        default:
            e = launch_wide<__nv_bfloat16>(plan.cluster, plan.clusters, smw, s, B->sys, B->order, K, B->alo, B->a64,
                                           B->b, B->x, out, B->queue + 2, Pw);
            break;
        }
        if (e != cudaSuccess) return e;
    }
    if (rest == 0) return cudaSuccess;
    const bool pdl = K > 0;
    switch (B->storage) {
    case TACTA_BATCH_FP64:
        return launch_cfg<double>(cfg, s, grid, smem, pdl, B->sys, B->order + K, rest, B->alo, B->a64, B->b, B->x,
                                  out, B->queue, P, B->queue + 1);
    case TACTA_BATCH_FP32:
        return launch_cfg<float>(cfg, s, grid, smem, pdl, B->sys, B->order + K, rest, B->alo, B->a64, B->b, B->x,
                                 out, B->queue, P, B->queue + 1);
    default:
        return launch_cfg<__nv_bfloat16>(cfg, s, grid, smem, pdl, B->sys, B->order + K, rest, B->alo, B->a64, B->b,
                                         B->x, out, B->queue, P, B->queue + 1);
    }
}

// Predicted makespan (ns) of a solve, by list scheduling: the clusters take the wide
// systems (one-cluster times w, descending) each as soon as it is free; the single-block
// kernel's blocks (per_sm per SM) start at once on the SMs no cluster holds, and on a
// cluster's C SMs when it has finished, and take the other systems (one-block times d,
// descending) each as soon as one is free. Past the first kExact of d the short systems
// are spread as a fluid over the blocks' free times (water filling).
double simulate_makespan(const std::vector<double>& w, int clusters, int C, const std::vector<double>& d, int sms,
                         int per_sm) {
    constexpr size_t kExact = 512;
    std::priority_queue<double, std::vector<double>, std::greater<double>> cq, bq;
    double end = 0.0;
    if (!w.empty() && clusters < 1) return INFINITY;
    for (int i = 0; i < clusters; ++i) cq.push(0.0);
    for (double v : w) {
        const double t = cq.top();
        cq.pop();
        cq.push(t + v);
        end = std::max(end, t + v);
    }
    for (int i = 0; i < std::max(0, sms - clusters * C) * per_sm; ++i) bq.push(0.0);
    while (!cq.empty()) {
        for (int i = 0; i < C * per_sm; ++i) bq.push(cq.top());
        cq.pop();
    }
    if (bq.empty()) return d.empty() ? end : INFINITY;
    double fluid = 0.0;
    for (size_t i = 0; i < d.size(); ++i) {
        if (i >= kExact) { fluid += d[i]; continue; }
        const double t = bq.top();
        bq.pop();
        bq.push(t + d[i]);
        end = std::max(end, t + d[i]);
    }
    if (fluid > 0.0) {
        std::vector<double> f;
        while (!bq.empty()) { f.push_back(bq.top()); bq.pop(); }   // ascending
        double level = f[0], below = 0.0;   // below: fluid needed to raise f[0..i) to f[i]
        size_t i = 1;
        for (; i < f.size(); ++i) {
            const double need = below + (f[i] - f[i - 1]) * (double)i;
            if (need >= fluid) break;
            below = need;
        }
        level = f[i - 1] + (fluid - below) / (double)i;
        end = std::max(end, level);
    }
    return end;
}

// the mean order t of the step-order schedule (one period)
double mean_order(int t_max, int cycle) {
    if (cycle == TACTA_CYCLE_FIXED || t_max == 1) return t_max;
    if (cycle == TACTA_CYCLE_SAWTOOTH) return 0.5 * (t_max + 1);
    const int period = 2 * t_max - 2;
    double sum = 0.0;
    for (int j = 0; j < period; ++j) sum += j < t_max ? j + 1 : 2 * t_max - 1 - j;
    return sum / period;
}

// the cluster-time model above for a system of m rows and n columns on C blocks (a_cap:
// the elements of A a block stages; one-block time dur, steps, mean order tm, overhead h0)
double cluster_time_model(int storage, int32_t m, int32_t n, int C, int64_t a_cap, double dur, double steps,
                          double tm, double h0) {
    const int64_t ld = storage == TACTA_BATCH_BF16 ? ((n + 15) & ~15) + 8 : (n + 7) & ~7;
    const int64_t rows = (m + C - 1) / C;
    const double stream = rows * ld <= a_cap ? 0.0 : 2.0 * tm * rows * ld * elem_size(storage) / kWideRowBw;
    return std::max(dur / C, steps * stream) + steps * (h0 + kWideH1 * C);
}

// cluster sizes the planner considers, largest first (1: forced plans only)
constexpr int kPlanSizes[] = {16, 8, 4, 2, 1};
constexpr int kNumPlanSizes = 5;

// What plan_search needs to know; host data only.
struct PlanInput {
    int count = 0;
    const double* dur = nullptr;      // one-block time per system (ns; all > 0, else unknown)
    const int32_t* steps = nullptr;   // step count per system in the last full solve (or null)
    const int32_t* m = nullptr;
    const int32_t* n = nullptr;
    const int32_t* ord = nullptr;     // the current queue order
    int storage = TACTA_BATCH_FP32, t_max = 5, cycle = TACTA_CYCLE_PINGPONG;
    int sms = 1, per_sm = 1;
    int wide_mode = -1, wide_cluster = 0, wide_clusters = 0;
    double h0 = kWideH0;
    int32_t max_clusters[kNumPlanSizes] = {};   // per kPlanSizes: resident clusters (0: the vectors do not fit)
    int64_t a_cap[kNumPlanSizes] = {};          // per kPlanSizes: elements of A a block stages
};

// The queue order and the cluster kernel's share of the next solve. The order is longest
// first by dur. With the planner on (wide_mode -1) and the times known, the plan is the
// one of least simulated makespan among: no clusters, and, for C = 16, 8, 4, 2 (where the
// vectors fit), the K = 1, 2, ... (at most 96) longest systems with at least 4 C rows and
// at least a quarter of the balanced time (sum dur / blocks), on min(K, resident
// clusters) clusters, a system's cluster time by cluster_time_model; a plan must beat the
// best so far by 2%. The clusters' systems come first in the order, longest in cluster
// time first. wide_mode > 0 forces that many systems from the head of the order onto
// clusters (of wide_cluster blocks, or the largest C that fits; wide_clusters of them, or
// as many as are resident). Returns the simulated makespan in ms (0 when the times are
// unknown; infinite when a forced plan has no cluster size that fits).
double plan_search(const PlanInput& in, WidePlan* plan_out, std::vector<int32_t>* ord_out) {
    const int count = in.count;
    const double* dur = in.dur;
    std::vector<int32_t> ord(in.ord, in.ord + count);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t c) { return dur[a] > dur[c]; });
    const bool known = count > 0 && std::all_of(dur, dur + count, [](double v) { return v > 0.0; });
    const int per_sm = in.per_sm;
    const double tm = mean_order(in.t_max, in.cycle);
    int64_t a_cap_c = 0;   // of the cluster size being scored
    auto cluster_time = [&](int32_t q, int C) {
        const double steps = in.steps ? (double)in.steps[q] : 0.0;
        return cluster_time_model(in.storage, in.m[q], in.n[q], C, a_cap_c, dur[q], steps, tm, in.h0);
    };
    *plan_out = WidePlan{};
    *ord_out = ord;
    if (in.wide_mode == 0 || count == 0) {
        if (!known) return 0.0;
        std::vector<double> d;
        for (int32_t s_ : ord) d.push_back(dur[s_]);
        return simulate_makespan({}, 0, 1, d, in.sms, per_sm) * 1e-6;
    }
    auto fits = [&](int i, int* maxc) {
        if (in.max_clusters[i] <= 0) return false;
        a_cap_c = in.a_cap[i];
        *maxc = in.max_clusters[i];
        return true;
    };
    if (in.wide_mode > 0) {   // forced
        WidePlan p{};
        p.systems = std::min(in.wide_mode, count);
        int maxc = 0;
        for (int i = 0; i < kNumPlanSizes; ++i) {
            if (in.wide_cluster > 0 && kPlanSizes[i] != in.wide_cluster) continue;
            if (fits(i, &maxc)) { p.cluster = kPlanSizes[i]; break; }
        }
        if (p.cluster == 0) return known ? INFINITY : 0.0;   // launch_batch refuses it
        p.clusters = std::min(p.systems, maxc);
        if (in.wide_clusters > 0) p.clusters = std::min(p.clusters, in.wide_clusters);
        *plan_out = p;
        if (!known) return 0.0;
        // the clusters take their systems longest (in cluster time) first
        std::stable_sort(ord.begin(), ord.begin() + p.systems, [&](int32_t a, int32_t c) {
            return cluster_time(a, p.cluster) > cluster_time(c, p.cluster);
        });
        *ord_out = ord;
        std::vector<double> w, d;
        for (int j = 0; j < count; ++j) {
            if (j < p.systems) w.push_back(cluster_time(ord[j], p.cluster));
            else d.push_back(dur[ord[j]]);
        }
        return simulate_makespan(w, p.clusters, p.cluster, d, in.sms, per_sm) * 1e-6;
    }
    if (!known) return 0.0;
    std::vector<double> all;
    double total = 0.0;
    for (int32_t s_ : ord) { all.push_back(dur[s_]); total += dur[s_]; }
    double best = simulate_makespan({}, 0, 1, all, in.sms, per_sm);
    std::vector<int32_t> best_wide;
    int64_t best_a_cap = 0;
    const double balanced = total / ((double)in.sms * per_sm);
    for (int i = 0; i < kNumPlanSizes; ++i) {
        const int C = kPlanSizes[i];
        int maxc = 0;
        if (C == 1 || !fits(i, &maxc)) continue;
        std::vector<int32_t> elig;   // positions in ord
        for (int j = 0; j < count && elig.size() < 96; ++j)
            if (in.m[ord[j]] >= 4 * C && dur[ord[j]] >= 0.25 * balanced) elig.push_back(j);
        std::vector<char> wide((size_t)count, 0);
        for (size_t K = 1; K <= elig.size(); ++K) {
            wide[elig[K - 1]] = 1;
            std::vector<double> w, d;
            for (int j = 0; j < count; ++j) {
                if (wide[j]) w.push_back(cluster_time(ord[j], C));
                else d.push_back(dur[ord[j]]);
            }
            std::sort(w.begin(), w.end(), std::greater<double>());
            const int cl = std::min((int)K, maxc);
            const double ms = simulate_makespan(w, cl, C, d, in.sms, per_sm);
            if (ms < 0.98 * best) {
                best = ms;
                plan_out->systems = (int32_t)K;
                plan_out->cluster = C;
                plan_out->clusters = cl;
                best_wide.assign(elig.begin(), elig.begin() + K);
                best_a_cap = a_cap_c;
            }
        }
    }
    if (plan_out->systems > 0) {   // the wide systems first, then the rest, each longest first
        std::vector<char> wide((size_t)count, 0);
        std::vector<int32_t> o2;
        for (int32_t j : best_wide) { wide[j] = 1; o2.push_back(ord[j]); }
        const int Cb = plan_out->cluster;
        a_cap_c = best_a_cap;
        std::stable_sort(o2.begin(), o2.end(), [&](int32_t a, int32_t c) {
            return cluster_time(a, Cb) > cluster_time(c, Cb);
        });
        for (int j = 0; j < count; ++j)
            if (!wide[j]) o2.push_back(ord[j]);
        *ord_out = o2;
    }
    return best * 1e-6;
}

// plan_search on this batch: the device's facts (which cluster sizes' vectors fit a
// block, how many such clusters can be resident, how much of A a block stages) gathered
// here, the launch configuration's blocks per SM, the learned overhead h0
double plan_batch(const tacta_batch_s* B, const tacta_options& o, int cfg, const std::vector<double>& dur,
                  WidePlan* plan_out, std::vector<int32_t>* ord_out) {
    PlanInput in;
    in.count = B->count;
    in.dur = dur.data();
    in.steps = B->last_iters.size() == (size_t)B->count ? B->last_iters.data() : nullptr;
    in.m = B->m_of.data();
    in.n = B->n_of.data();
    in.ord = B->ord.data();
    in.storage = B->storage;
    in.t_max = o.t_max;
    in.cycle = o.cycle;
    in.sms = B->sms;
    in.per_sm = kConfigs[cfg].per_sm;
    in.wide_mode = B->wide_mode;
    in.wide_cluster = B->wide_cluster;
    in.wide_clusters = B->wide_clusters;
    in.h0 = B->wide_h0 >= 0.0 ? B->wide_h0 : kWideH0;
    const bool known = B->count > 0 && std::all_of(dur.begin(), dur.end(), [](double v) { return v > 0.0; });
    if (B->wide_mode != 0 && (known || B->wide_mode > 0)) {   // (the device queries only when used)
        for (int i = 0; i < kNumPlanSizes; ++i) {
            BatchParams Pw{};
            size_t smw = 0;
            if (!wide_params(B, o, kPlanSizes[i], &Pw, &smw)) continue;
            in.a_cap[i] = Pw.a_cap;
            in.max_clusters[i] = wide_max_clusters_for(B, kPlanSizes[i], smw);
        }
    }
    return plan_search(in, plan_out, ord_out);
}

bool batch_opts_ok(const tacta_options& o) {
    if (!(std::isfinite(o.tol) && o.tol > 0.0)) { g_batch_err = "tol must be finite and > 0"; return false; }
    if (!std::isfinite(o.tol_normal)) { g_batch_err = "tol_normal must be finite"; return false; }
    if (o.t_max < 1 || o.t_max > kTMax) { g_batch_err = "t_max must be in 1..8"; return false; }
    if (o.max_iter < 0) { g_batch_err = "max_iter must be >= 0"; return false; }
    if (o.recompute_every < 0) { g_batch_err = "recompute_every must be >= 0"; return false; }
    if (o.cycle < 0 || o.cycle > 2) { g_batch_err = "unknown cycle"; return false; }
    return true;
}

tacta_options resolve_opts(const tacta_options* opt) {
    tacta_options o;
    tacta_default_options(&o);
    if (opt) o = *opt;
    if (o.tol_normal < 0.0) o.tol_normal = 0.0;
    return o;
}

}  // namespace

#define BTRY(expr)                                                                     \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            g_batch_err = std::string(#expr) + ": " + cudaGetErrorString(e_);          \
            return e_ == cudaErrorMemoryAllocation ? TACTA_ERR_OOM : TACTA_ERR_CUDA;   \
        }                                                                              \
    } while (0)

extern "C" const char* tacta_batch_last_error(void) { return g_batch_err.c_str(); }

extern "C" tacta_status tacta_batch_create(int32_t count, const int32_t* m, const int32_t* n, const double* vals,
                                           int32_t on_device, int32_t storage, const tacta_options* opt,
                                           tacta_batch* out) {
    g_batch_err.clear();
    if (!out) { g_batch_err = "out is NULL"; return TACTA_ERR_INVALID; }
    *out = nullptr;
    if (count < 0) { g_batch_err = "count must be >= 0"; return TACTA_ERR_INVALID; }
    if (count > 0 && (!m || !n || !vals)) { g_batch_err = "m, n or vals is NULL"; return TACTA_ERR_INVALID; }
    if (storage != TACTA_BATCH_FP64 && storage != TACTA_BATCH_FP32 && storage != TACTA_BATCH_BF16) {
        g_batch_err = "unknown storage";
        return TACTA_ERR_INVALID;
    }
    std::vector<SysDesc> d((size_t)count);
    int64_t a64 = 0, alo = 0, bo = 0, xo = 0;
    int32_t mmax = 1, nmax = 1;
    for (int32_t s = 0; s < count; ++s) {
        if (m[s] < 1 || n[s] < 1 || m[s] > kBatchMaxDim || n[s] > kBatchMaxDim) {
            g_batch_err = "system " + std::to_string(s) + ": m and n must be in 1.." + std::to_string(kBatchMaxDim);
            return TACTA_ERR_INVALID;
        }
        SysDesc& q = d[(size_t)s];
        std::memset(&q, 0, sizeof(q));
        q.m = m[s];
        q.n = n[s];
        // BF16 rows: 16-column tiles plus 8, so that ldmatrix's eight rows hit distinct banks
        q.ld = storage == TACTA_BATCH_BF16 ? ((n[s] + 15) & ~15) + 8 : (n[s] + 7) & ~7;
        q.a64 = a64;
        q.a_lo = alo;
        q.b_off = bo;
        q.x_off = xo;
        a64 += (int64_t)m[s] * n[s];
        alo += (int64_t)m[s] * q.ld;
        bo += m[s];
        xo += n[s];
        mmax = std::max(mmax, m[s]);
        nmax = std::max(nmax, n[s]);
    }
    tacta_batch_s* B = new tacta_batch_s();
    B->count = count;
    B->storage = storage;
    B->m_max = mmax;
    B->n_max = nmax;
    B->a64_len = a64;
    B->alo_len = alo;
    B->b_len = bo;
    B->x_len = xo;
    cudaStream_t s = opt && opt->stream ? (cudaStream_t)opt->stream : (cudaStream_t)0;
    auto fail = [&](cudaError_t e, const char* what) {
        g_batch_err = std::string(what) + ": " + cudaGetErrorString(e);
        free_batch(B);
        return e == cudaErrorMemoryAllocation ? TACTA_ERR_OOM : TACTA_ERR_CUDA;
    };
#define BCHK(expr) do { cudaError_t e_ = (expr); if (e_ != cudaSuccess) return fail(e_, #expr); } while (0)
    BCHK(cudaGetDevice(&B->device));
    BCHK(cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, B->device));
    BCHK(prepare_kernels());
    const size_t es = elem_size(storage);
    BCHK(cudaMalloc(&B->sys, sizeof(SysDesc) * std::max<int32_t>(count, 1)));
    BCHK(cudaMalloc(&B->order, sizeof(int32_t) * std::max<int32_t>(count, 1)));
    BCHK(cudaMalloc(&B->a64, sizeof(double) * std::max<int64_t>(a64, 1)));
    BCHK(cudaMalloc(&B->alo, es * std::max<int64_t>(alo, 8) + 16));
    BCHK(cudaMalloc(&B->b, sizeof(double) * std::max<int64_t>(bo, 1)));
    BCHK(cudaMalloc(&B->x, sizeof(double) * std::max<int64_t>(xo, 1)));
    BCHK(cudaMalloc(&B->iters, sizeof(int32_t) * std::max<int32_t>(count, 1)));
    BCHK(cudaMalloc(&B->reason, sizeof(int32_t) * std::max<int32_t>(count, 1)));
    BCHK(cudaMalloc(&B->rel, sizeof(double) * std::max<int32_t>(count, 1)));
    BCHK(cudaMalloc(&B->queue, 4 * sizeof(int32_t)));
    BCHK(cudaMalloc(&B->stamps, 2 * sizeof(int64_t) * std::max<int32_t>(count, 1)));
    BCHK(cudaMemsetAsync(B->stamps, 0, 2 * sizeof(int64_t) * std::max<int32_t>(count, 1), s));
    if (count > 0) {
        // largest systems first: the queue's tail is then made of short jobs
        std::vector<int32_t> ord((size_t)count);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b2) {
            return (int64_t)d[a].m * d[a].n > (int64_t)d[b2].m * d[b2].n;
        });
        B->ord = ord;
        B->m_of.assign(m, m + count);
        B->n_of.assign(n, n + count);
        B->dur.assign((size_t)count, 0.0);
        B->dur_meas.assign((size_t)count, 0);
        BCHK(cudaMemcpyAsync(B->sys, d.data(), sizeof(SysDesc) * count, cudaMemcpyHostToDevice, s));
        BCHK(cudaMemcpyAsync(B->order, ord.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s));
        BCHK(cudaMemcpyAsync(B->a64, vals, sizeof(double) * a64, on_device ? cudaMemcpyDeviceToDevice
                                                                           : cudaMemcpyHostToDevice, s));
        chain_scale<<<count, 256, 0, s>>>(B->sys, B->a64);
        BCHK(cudaGetLastError());
        switch (storage) {
        case TACTA_BATCH_FP64: pack_lo<double><<<count, 256, 0, s>>>(B->sys, B->a64, (double*)B->alo); break;
        case TACTA_BATCH_FP32: pack_lo<float><<<count, 256, 0, s>>>(B->sys, B->a64, (float*)B->alo); break;
        default: pack_lo<__nv_bfloat16><<<count, 256, 0, s>>>(B->sys, B->a64, (__nv_bfloat16*)B->alo); break;
        }
        BCHK(cudaGetLastError());
        BCHK(cudaStreamSynchronize(s));
    }
#undef BCHK
    *out = B;
    return TACTA_OK;
}

extern "C" void tacta_batch_destroy(tacta_batch B) {
    if (!B) return;
    cudaSetDevice(B->device);
    free_batch(B);
}

extern "C" tacta_status tacta_batch_set_config(tacta_batch B, int32_t config) {
    g_batch_err.clear();
    if (!B) { g_batch_err = "NULL batch"; return TACTA_ERR_INVALID; }
    if (config < -1 || config >= kNumConfigs) { g_batch_err = "unknown config"; return TACTA_ERR_INVALID; }
    B->config = config;
    return TACTA_OK;
}

extern "C" int32_t tacta_batch_num_configs(void) { return kNumConfigs; }

extern "C" int32_t tacta_batch_config_tensor_cores(int32_t config) {
    return config >= 0 && config < kNumConfigs && kConfigs[config].mma ? 1 : 0;
}

extern "C" int32_t tacta_batch_config_stage_bytes(int32_t config) {
    return config >= 0 && config < kNumConfigs ? kConfigs[config].stage_kb * 1024 : 0;
}

extern "C" tacta_status tacta_batch_timeline(tacta_batch B, int64_t* t_begin_ns, int64_t* t_end_ns) {
    g_batch_err.clear();
    if (!B || !t_begin_ns || !t_end_ns) { g_batch_err = "NULL argument"; return TACTA_ERR_INVALID; }
    BTRY(cudaSetDevice(B->device));
    if (B->count == 0) return TACTA_OK;
    BTRY(cudaMemcpy(t_begin_ns, B->stamps, sizeof(int64_t) * B->count, cudaMemcpyDefault));
    BTRY(cudaMemcpy(t_end_ns, B->stamps + B->count, sizeof(int64_t) * B->count, cudaMemcpyDefault));
    return TACTA_OK;
}

extern "C" tacta_status tacta_batch_config_shape(int32_t config, int32_t* threads, int32_t* blocks_per_sm) {
    if (config < 0 || config >= kNumConfigs || !threads || !blocks_per_sm) return TACTA_ERR_INVALID;
    *threads = kConfigs[config].nt + (kConfigs[config].streamed ? 32 : 0);
    *blocks_per_sm = kConfigs[config].per_sm;
    return TACTA_OK;
}

extern "C" tacta_status tacta_batch_cta(tacta_batch B, const double* b, double* x, int32_t* iters,
                                        double* rel_res, int32_t* reason, const tacta_options* opt) {
    g_batch_err.clear();
    if (!B) { g_batch_err = "NULL batch"; return TACTA_ERR_INVALID; }
    if (B->count > 0 && (!b || !x)) { g_batch_err = "b or x is NULL"; return TACTA_ERR_INVALID; }
    const tacta_options o = resolve_opts(opt);
    if (!batch_opts_ok(o)) return TACTA_ERR_INVALID;
    BTRY(cudaSetDevice(B->device));
    if (B->count == 0) return TACTA_OK;
    cudaStream_t s = (cudaStream_t)o.stream;
    const int cfg = B->config >= 0 ? B->config : kDefaultConfig;
    BatchParams P{};
    {
        size_t smem = 0;
        if (!make_params(B, o, cfg, &P, &smem)) {
            g_batch_err = "the largest system does not fit this launch configuration's shared memory: "
                          "lower t_max, pick another configuration, or solve it with a plan";
            return TACTA_ERR_INVALID;
        }
    }
    // the queue order and the clusters' share, from the times the last solves measured
    WidePlan plan{};
    std::vector<int32_t> ord;
    plan_batch(B, o, cfg, B->dur, &plan, &ord);
    if (B->wide_mode > 0 && plan.systems == 0) {
        g_batch_err = "the cluster kernel cannot take this batch (its vectors do not fit a block's shared memory)";
        return TACTA_ERR_INVALID;
    }
    if (ord != B->ord) {
        B->ord = ord;
        BTRY(cudaMemcpyAsync(B->order, B->ord.data(), sizeof(int32_t) * B->count, cudaMemcpyHostToDevice, s));
    }
    B->plan = plan;
    BTRY(cudaMemcpyAsync(B->b, b, sizeof(double) * B->b_len, cudaMemcpyDefault, s));
    if (o.use_graph) {
        // the solve is a queue reset and one or two persistent launches: replay it as a graph
        if (!B->graph || B->graph_key != cfg || std::memcmp(&P, &B->graph_params, sizeof(P)) != 0 ||
            !(B->graph_plan == plan)) {
            if (B->graph) { cudaGraphExecDestroy(B->graph); B->graph = nullptr; }
            cudaStream_t cs;
            BTRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t el = launch_batch(B, cs, o, cfg, plan);
                e = cudaStreamEndCapture(cs, &g);
                if (el != cudaSuccess) e = el;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&B->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            BTRY(e);
            B->graph_key = cfg;
            B->graph_params = P;
            B->graph_plan = plan;
        }
        BTRY(cudaGraphLaunch(B->graph, s));
    } else {
        BTRY(launch_batch(B, s, o, cfg, plan));
    }
    BTRY(cudaMemcpyAsync(x, B->x, sizeof(double) * B->x_len, cudaMemcpyDefault, s));
    if (iters) BTRY(cudaMemcpyAsync(iters, B->iters, sizeof(int32_t) * B->count, cudaMemcpyDefault, s));
    if (rel_res) BTRY(cudaMemcpyAsync(rel_res, B->rel, sizeof(double) * B->count, cudaMemcpyDefault, s));
    if (reason) BTRY(cudaMemcpyAsync(reason, B->reason, sizeof(int32_t) * B->count, cudaMemcpyDefault, s));
    int32_t timed_out = 0;
    BTRY(cudaMemcpyAsync(&timed_out, B->queue + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BTRY(cudaStreamSynchronize(s));
    if (timed_out) {
        g_batch_err = "a wait in the batched kernel gave up (systems reported with reason TIMEOUT)";
        return TACTA_ERR_TIMEOUT;
    }
    // What the next solve plans with (a system's result does not depend on the block or
    // the moment that takes it; on a cluster, its sums run in another order): each
    // system's time on one block -- measured where one block solved it -- and the step
    // counts. From the systems a cluster solved that have an earlier one-block time, the
    // per-step overhead h0 of the cluster-time model (cluster_time_model) is refitted: the
    // step-weighted mean of what the measured cluster time leaves over the model with
    // h0 = 0. A system without an earlier one-block time is given (cluster time - steps
    // (h0 + h1 C)) C, at least its cluster time.
    B->last_iters.resize((size_t)B->count);
    BTRY(cudaMemcpy(B->last_iters.data(), B->iters, sizeof(int32_t) * B->count, cudaMemcpyDeviceToHost));
    std::vector<int64_t> st((size_t)2 * B->count);
    BTRY(cudaMemcpy(st.data(), B->stamps, sizeof(int64_t) * 2 * B->count, cudaMemcpyDeviceToHost));
    const int64_t* tb = st.data();
    const int64_t* te = st.data() + B->count;
    const int K = std::min(plan.systems, B->count), C = plan.cluster;
    int64_t a_cap_w = 0;
    if (K > 0) {
        BatchParams Pw{};
        size_t smw = 0;
        if (wide_params(B, o, C, &Pw, &smw)) a_cap_w = Pw.a_cap;
    }
    const double tm = mean_order(o.t_max, o.cycle);
    double hnum = 0.0, hden = 0.0;
    for (int j = 0; j < B->count; ++j) {
        const int32_t q = B->ord[j];
        const double meas = std::max(1.0, (double)(te[q] - tb[q]));
        if (j >= K) {
            B->dur[q] = meas;
            B->dur_meas[q] = 1;
        } else if (B->dur_meas[q] && B->last_iters[q] > 0) {
            // the model's time with h0 = 0, subtracted from the measured time
            const double steps = (double)B->last_iters[q];
            hnum += meas - cluster_time_model(B->storage, B->m_of[q], B->n_of[q], C, a_cap_w, B->dur[q], steps,
                                              tm, 0.0);
            hden += steps;
        }
    }
    if (hden > 0.0) B->wide_h0 = std::min(2e5, std::max(0.0, hnum / hden));
    for (int j = 0; j < K; ++j) {
        const int32_t q = B->ord[j];
        if (!B->dur_meas[q]) {
            const double meas = std::max(1.0, (double)(te[q] - tb[q]));
            const double h0 = B->wide_h0 >= 0.0 ? B->wide_h0 : kWideH0;
            const double steps = (double)B->last_iters[q];
            B->dur[q] = std::max(meas, (meas - steps * (h0 + kWideH1 * C)) * C);
        }
    }
    return TACTA_OK;
}

extern "C" double tacta_batch_simulate_makespan(const double* w, int32_t nw, int32_t clusters, int32_t cluster,
                                                const double* d, int32_t nd, int32_t sms, int32_t per_sm) {
    if (nw < 0 || nd < 0 || clusters < 0 || cluster < 1 || sms < 1 || per_sm < 1 ||
        (int64_t)clusters * cluster > sms || (nw > 0 && (!w || clusters < 1)) || (nd > 0 && !d))
        return -1.0;
    std::vector<double> wv(w, w + nw), dv(d, d + nd);
    for (double v : wv)
        if (!(v >= 0.0)) return -1.0;
    for (double v : dv)
        if (!(v >= 0.0)) return -1.0;
    std::sort(wv.begin(), wv.end(), std::greater<double>());
    std::sort(dv.begin(), dv.end(), std::greater<double>());
    return simulate_makespan(wv, clusters, cluster, dv, sms, per_sm);
}

extern "C" double tacta_batch_plan_search(int32_t count, const double* dur, const int32_t* steps, const int32_t* m,
                                          const int32_t* n, int32_t storage, int32_t t_max, int32_t cycle,
                                          int32_t sms, int32_t per_sm, const int32_t* max_clusters,
                                          const int64_t* a_cap, int32_t wide_mode, int32_t wide_cluster,
                                          int32_t wide_clusters, double h0, int32_t* plan, int32_t* order) {
    if (count < 0 || (count > 0 && (!dur || !m || !n || !order)) || !plan || !max_clusters || !a_cap) return -1.0;
    if (storage != TACTA_BATCH_FP64 && storage != TACTA_BATCH_FP32 && storage != TACTA_BATCH_BF16) return -1.0;
    if (t_max < 1 || t_max > kTMax || cycle < 0 || cycle > 2 || sms < 1 || per_sm < 1) return -1.0;
    if (wide_mode < -1 || wide_cluster < 0 || wide_cluster > kWideMaxC || wide_clusters < 0) return -1.0;
    if (!(h0 >= 0.0) || !std::isfinite(h0)) return -1.0;
    for (int i = 0; i < kNumPlanSizes; ++i)
        if (max_clusters[i] < 0 || a_cap[i] < 0) return -1.0;
    for (int32_t q = 0; q < count; ++q) {
        if (!(dur[q] >= 0.0) || !std::isfinite(dur[q]) || m[q] < 1 || n[q] < 1) return -1.0;
        if (steps && steps[q] < 0) return -1.0;
    }
    std::vector<int32_t> ord0((size_t)count);
    std::iota(ord0.begin(), ord0.end(), 0);
    PlanInput in;
    in.count = count;
    in.dur = dur;
    in.steps = steps;
    in.m = m;
    in.n = n;
    in.ord = ord0.data();
    in.storage = storage;
    in.t_max = t_max;
    in.cycle = cycle;
    in.sms = sms;
    in.per_sm = per_sm;
    in.wide_mode = wide_mode;
    in.wide_cluster = wide_cluster;
    in.wide_clusters = wide_clusters;
    in.h0 = h0;
    for (int i = 0; i < kNumPlanSizes; ++i) {
        in.max_clusters[i] = max_clusters[i];
        in.a_cap[i] = a_cap[i];
    }
    WidePlan p{};
    std::vector<int32_t> ord;
    const double ms = plan_search(in, &p, &ord);
    plan[0] = p.systems;
    plan[1] = p.cluster;
    plan[2] = p.clusters;
    std::copy(ord.begin(), ord.end(), order);
    return ms;
}

extern "C" tacta_status tacta_batch_set_wide(tacta_batch B, int32_t systems, int32_t cluster, int32_t clusters) {
    g_batch_err.clear();
    if (!B) { g_batch_err = "NULL batch"; return TACTA_ERR_INVALID; }
    if (systems < -1 || cluster < 0 || cluster > kWideMaxC || clusters < 0) {
        g_batch_err = "systems must be >= -1, cluster in 0..16, clusters >= 0";
        return TACTA_ERR_INVALID;
    }
    B->wide_mode = systems;
    B->wide_cluster = cluster;
    B->wide_clusters = clusters;
    return TACTA_OK;
}

extern "C" tacta_status tacta_batch_wide_plan(tacta_batch B, const tacta_options* opt, int32_t* systems,
                                              int32_t* cluster, int32_t* clusters, double* predicted_ms) {
    g_batch_err.clear();
    if (!B) { g_batch_err = "NULL batch"; return TACTA_ERR_INVALID; }
    const tacta_options o = resolve_opts(opt);
    if (!batch_opts_ok(o)) return TACTA_ERR_INVALID;
    BTRY(cudaSetDevice(B->device));
    WidePlan plan{};
    std::vector<int32_t> ord;
    const double ms = plan_batch(B, o, B->config >= 0 ? B->config : kDefaultConfig, B->dur, &plan, &ord);
    if (systems) *systems = plan.systems;
    if (cluster) *cluster = plan.cluster;
    if (clusters) *clusters = plan.clusters;
    if (predicted_ms) *predicted_ms = ms;
    return TACTA_OK;
}

// Autotuner: times every launch configuration on the batch (each solve capped at
// max_iter of the given options, graphs off, single-block kernel only), keeps the best,
// and returns it. Before any full solve the score is the capped run's time; after one,
// it is the makespan predicted for a full solve: every system's one-block time taken as
// its time per step in the capped run times its step count in the last full solve (how
// a system shares its SM with other blocks depends on the launch shape), then the
// planner's simulated makespan with those times (the clusters' share included, see
// plan_batch). The best configuration's predicted times become the planner's.
extern "C" tacta_status tacta_batch_tune(tacta_batch B, const double* b, const tacta_options* opt,
                                         int32_t* best_config, double* best_ms) {
    g_batch_err.clear();
    if (!B || !b) { g_batch_err = "NULL argument"; return TACTA_ERR_INVALID; }
    tacta_options o = resolve_opts(opt);
    if (!batch_opts_ok(o)) return TACTA_ERR_INVALID;
    BTRY(cudaSetDevice(B->device));
    if (B->count == 0) { if (best_config) *best_config = kDefaultConfig; return TACTA_OK; }
    cudaStream_t s = (cudaStream_t)o.stream;
    BTRY(cudaMemcpyAsync(B->b, b, sizeof(double) * B->b_len, cudaMemcpyDefault, s));
    cudaEvent_t e0, e1;
    BTRY(cudaEventCreate(&e0));
    BTRY(cudaEventCreate(&e1));
    int best = -1;
    double best_t = 0.0;
    std::vector<double> best_dur;
    for (int c = 0; c < kNumConfigs; ++c) {
        size_t smem = 0;
        BatchParams P{};
        if (!make_params(B, o, c, &P, &smem)) continue;
        float tc = 0.0f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {      // the first run warms caches and loads the module
            ok = cudaEventRecord(e0, s) == cudaSuccess && launch_batch(B, s, o, c, WidePlan{}) == cudaSuccess &&
                 cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                 cudaEventElapsedTime(&tc, e0, e1) == cudaSuccess;
        }
        double score = tc;
        std::vector<double> dc;
        if (ok && B->last_iters.size() == (size_t)B->count) {
            std::vector<int64_t> st((size_t)2 * B->count);
            std::vector<int32_t> it((size_t)B->count);
            ok = cudaMemcpy(st.data(), B->stamps, sizeof(int64_t) * 2 * B->count, cudaMemcpyDeviceToHost) ==
                     cudaSuccess &&
                 cudaMemcpy(it.data(), B->iters, sizeof(int32_t) * B->count, cudaMemcpyDeviceToHost) == cudaSuccess;
            dc.assign((size_t)B->count, 0.0);
            for (int32_t q = 0; ok && q < B->count; ++q) {
                const double meas = std::max(1.0, (double)(st[(size_t)B->count + q] - st[q]));
                dc[q] = it[q] > 0 ? meas / it[q] * std::max<int32_t>(B->last_iters[q], it[q]) : meas;
            }
            WidePlan p{};
            std::vector<int32_t> ord;
            const double ms = ok ? plan_batch(B, o, c, dc, &p, &ord) : 0.0;
            if (ms > 0.0) score = ms;
        }
        if (ok && (best < 0 || score < best_t)) {
            best = c;
            best_t = score;
            best_dur = dc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BTRY(cudaGetLastError());
    if (best < 0) { g_batch_err = "no launch configuration fits this batch"; return TACTA_ERR_CUDA; }
    B->config = best;
    if (best_dur.size() == (size_t)B->count) {
        B->dur = best_dur;
        B->dur_meas.assign((size_t)B->count, 1);
    }
    if (best_config) *best_config = best;
    if (best_ms) *best_ms = best_t;
    return TACTA_OK;
}

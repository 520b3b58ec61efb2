// tacta_residual_static: the residual r = b - A x and its reductions without any
// device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// residual: code running inside a framework whose caching allocator has already
// reserved the device (a direct cudaMalloc then fails or fragments the pool),
// and latency-bound host loops that must not enter the driver's allocator
// (cudaMalloc and cudaFree may synchronize the device and take unbounded time).
// The plan-based entry points allocate their workspace (per-block reduction
// partials, the control block); this variant keeps that scratch in one
// file-scope device array instead, so a call only launches work on the
// caller's stream and copies 16 bytes of results back.
//
// Limits and sharing rules (also stated in include/tacta.h):
//   * the scratch array is kStaticScratchBytes (1 MiB) per device, holding the
//     per-block partials of one block per 256 rows, so m <= kStaticMaxRows;
//     larger m is rejected with TACTA_ERR_INVALID;
//   * every call on a device uses the same array and leaves its contents
//     behind; the ticket counter that must start at zero is cleared at the start
//     of every call; two calls whose work overlaps on the GPU race on the array;
//   * the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     outside any stream capture. The address is cached for the life of the
//     process: after a cudaDeviceReset of that device it is stale, so a caller
//     that resets a device must not call this entry point on it again.
#include <cuda_runtime.h>

#include <cfloat>
#include <mutex>
#include <string>

#include "internal.h"

namespace tacta {
namespace {

constexpr int kStaticBlock = 256;
constexpr size_t kStaticScratchBytes = size_t(1) << 20;
// layout: [0, 256) header (ticket counter, two results), then 2 doubles per block
constexpr size_t kStaticHeader = 256;
constexpr int64_t kStaticMaxBlocks = (int64_t)((kStaticScratchBytes - kStaticHeader) / (2 * sizeof(double)));
constexpr int64_t kStaticMaxRows = kStaticMaxBlocks * kStaticBlock;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct ScratchView {
    unsigned int* counter;
    double* result;     // [0] = ||r||², [1] = rᵀ b
    double* partials;   // 2 per block
};

__device__ __forceinline__ ScratchView view(unsigned char* base) {
    ScratchView v;
    v.counter = reinterpret_cast<unsigned int*>(base);
    v.result = reinterpret_cast<double*>(base + 64);
    v.partials = reinterpret_cast<double*>(base + kStaticHeader);
    return v;
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// One thread per row: r_i = b_i - (A x)_i, with the per-block sums of r_i² and
// r_i b_i in the scratch partials; the last block (atomic ticket, no waiting)
// adds the partials in block order and stores the two results.
template <bool DENSE>
__global__ void __launch_bounds__(kStaticBlock)
residual_static_kernel(int64_t m, int64_t n, const int32_t* __restrict__ rowptr,
                       const int32_t* __restrict__ colidx, const double* __restrict__ vals,
                       const double* __restrict__ x, const double* __restrict__ b,
                       double* __restrict__ r, unsigned char* scratch) {
    ScratchView sv = view(scratch);
    __shared__ double s0[kStaticBlock / 32], s1[kStaticBlock / 32];
    __shared__ int last;
    const int64_t row = (int64_t)blockIdx.x * kStaticBlock + threadIdx.x;
    double a0 = 0.0, a1 = 0.0;
    if (row < m) {
        const int64_t kb = DENSE ? row * n : rowptr[row];
        const int64_t ke = DENSE ? kb + n : rowptr[row + 1];
        double sum = 0.0;
        for (int64_t k = kb; k < ke; ++k)
            sum = fma(__ldg(vals + k), __ldg(x + (DENSE ? k - kb : (int64_t)colidx[k])), sum);
        const double bv = __ldg(b + row);
        const double v = bv - sum;
        r[row] = v;
        a0 = v * v;
        a1 = v * bv;
    }
    a0 = wsum(a0);
    a1 = wsum(a1);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { s0[w] = a0; s1[w] = a1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0.0, t1 = 0.0;
        for (int i = 0; i < kStaticBlock / 32; ++i) { t0 += s0[i]; t1 += s1[i]; }
        sv.partials[2 * blockIdx.x] = t0;
        sv.partials[2 * blockIdx.x + 1] = t1;
        __threadfence();
        last = (atomicAdd(sv.counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t0 = 0.0, t1 = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kStaticBlock) {
        t0 += __ldcg(sv.partials + 2 * i);
        t1 += __ldcg(sv.partials + 2 * i + 1);
    }
    t0 = wsum(t0);
    t1 = wsum(t1);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { s0[w] = t0; s1[w] = t1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double u0 = 0.0, u1 = 0.0;
        for (int i = 0; i < kStaticBlock / 32; ++i) { u0 += s0[i]; u1 += s1[i]; }
        sv.result[0] = u0;
        sv.result[1] = u1;
    }
}

std::mutex g_lock;
unsigned char* g_addr[kMaxDevices] = {};

// device address of the scratch array on the current device (looked up once per device)
cudaError_t scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> guard(g_lock);
    if (g_addr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace tacta

using namespace tacta;

extern "C" tacta_status tacta_residual_static(const tacta_matrix* A, const double* x, const double* b,
                                              double* r_out, double* norms_out, void* stream) {
    set_error("");
    if (!A || !x || !b || !r_out || !norms_out) { set_error("NULL argument"); return TACTA_ERR_INVALID; }
    if (!A->on_device) {
        set_error("tacta_residual_static needs device arrays (on_device = 1): it cannot allocate to copy host data");
        return TACTA_ERR_INVALID;
    }
    if (A->m < 1 || A->n < 1 || A->n >= (1LL << 31)) { set_error("A must have m, n >= 1 and n < 2^31"); return TACTA_ERR_INVALID; }
    if (A->m > kStaticMaxRows) {
        set_error("m = " + std::to_string(A->m) + " exceeds the static-scratch limit of " +
                  std::to_string(kStaticMaxRows) + " rows (1 MiB of per-block partials)");
        return TACTA_ERR_INVALID;
    }
    if (A->format == TACTA_CSR) {
        if (!A->rowptr || (A->nnz > 0 && (!A->colidx || !A->vals))) { set_error("CSR arrays missing"); return TACTA_ERR_INVALID; }
    } else if (A->format == TACTA_DENSE) {
        if (!A->vals) { set_error("A.vals is NULL"); return TACTA_ERR_INVALID; }
    } else {
        set_error("unknown format");
        return TACTA_ERR_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return TACTA_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device index " + std::to_string(dev) + " is beyond the " + std::to_string(kMaxDevices) +
                  " devices whose scratch address tacta_residual_static caches");
        return TACTA_ERR_INVALID;
    }
    unsigned char* scratch = nullptr;
    if ((e = scratch_address(dev, &scratch)) != cudaSuccess) {
        set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return TACTA_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t blocks = (A->m + kStaticBlock - 1) / kStaticBlock;
    // the ticket counter must start at zero; the rest of the scratch is written before it is read
    if ((e = cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s)) != cudaSuccess) {
        set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        return TACTA_ERR_CUDA;
    }
    if (A->format == TACTA_DENSE)
        residual_static_kernel<true><<<(unsigned)blocks, kStaticBlock, 0, s>>>(
            A->m, A->n, nullptr, nullptr, A->vals, x, b, r_out, scratch);
    else
        residual_static_kernel<false><<<(unsigned)blocks, kStaticBlock, 0, s>>>(
            A->m, A->n, A->rowptr, A->colidx, A->vals, x, b, r_out, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) {
        set_error(std::string("launch: ") + cudaGetErrorString(e));
        return TACTA_ERR_CUDA;
    }
    if ((e = cudaMemcpyAsync(norms_out, scratch + 64, 2 * sizeof(double), cudaMemcpyDefault, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        set_error(std::string("result copy: ") + cudaGetErrorString(e));
        return TACTA_ERR_CUDA;
    }
    return TACTA_OK;
}

// Plan-time setup kernels: CSR structure validation, CSR and dense transposes.
//
// The CTA chain alternates products with A and Aᵀ (z_i = Aᵀ u_{i-1},
// u_i = A z_i), and TA needs c = Aᵀ(b - b'). Both products run as row-parallel
// gathers, so the plan stores Aᵀ explicitly: no atomics in the hot loop.
//
// The CSR transpose is a stable radix sort of the nonzeros by column (CUB,
// shipped with the CUDA toolkit), so every row of Aᵀ lists its entries in
// increasing original row order and the products are run-to-run reproducible.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "internal.h"

namespace tacta {

namespace {

// flag bits: 1 rowptr[0] != 0, 2 decreasing rowptr, 4 rowptr[m] != nnz, 8 column out of range
__global__ void validate_rowptr(const int32_t* rowptr, int64_t m, int64_t nnz, int* flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int32_t a = rowptr[i], b = rowptr[i + 1];
        if (b < a) atomicOr(flag, 2);
        if (i == 0 && a != 0) atomicOr(flag, 1);
        if (i == m - 1 && (int64_t)b != nnz) atomicOr(flag, 4);
    }
}

__global__ void validate_colidx(const int32_t* colidx, int64_t nnz, int64_t n, int* flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
        const int32_t c = colidx[k];
        if (c < 0 || (int64_t)c >= n) atomicOr(flag, 8);
    }
}

// row index of every nonzero (binary search in rowptr)
__global__ void row_of_nonzero(const int32_t* rowptr, int64_t m, int64_t nnz, int32_t* rowof,
                               int32_t* seq) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
        int64_t lo = 0, hi = m;  // find the last row r with rowptr[r] <= k
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (rowptr[mid] <= k) lo = mid; else hi = mid;
        }
        rowof[k] = (int32_t)lo;
        seq[k] = (int32_t)k;
    }
}

__global__ void count_cols(const int32_t* colidx, int64_t nnz, int32_t* counts) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride)
        atomicAdd(counts + colidx[k], 1);
}

__global__ void gather_transposed(const int32_t* perm, const int32_t* rowof, const double* vals,
                                  int64_t nnz, int32_t* tcol, double* tval) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
        const int32_t k = perm[p];
        tcol[p] = rowof[k];
        tval[p] = vals[k];
    }
}

__global__ void dense_transpose_kernel(const double* __restrict__ A, int64_t rows, int64_t cols,
                                       double* __restrict__ T) {
    __shared__ double tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int64_t r = r0 + j, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[j][threadIdx.x] = A[r * cols + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int64_t c = c0 + j, r = r0 + threadIdx.x;
        if (r < rows && c < cols) T[c * rows + r] = tile[threadIdx.x][j];
    }
}

inline int blocks_for(int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (int)b;
}

}  // namespace

cudaError_t csr_validate(cudaStream_t s, const int32_t* rowptr, const int32_t* colidx, int64_t m,
                         int64_t n, int64_t nnz, int* flag_dev, int* flag_host) {
    cudaError_t e = cudaMemsetAsync(flag_dev, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    validate_rowptr<<<blocks_for(m), kBlock, 0, s>>>(rowptr, m, nnz, flag_dev);
    if (nnz > 0) validate_colidx<<<blocks_for(nnz), kBlock, 0, s>>>(colidx, nnz, n, flag_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(flag_host, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(s);
}

cudaError_t csr_transpose(cudaStream_t s, const DevCSR& A, DevCSR& T) {
    const int64_t nnz = A.nnz;
    cudaError_t e;
    T.rows = A.cols;
    T.cols = A.rows;
    T.nnz = nnz;
    // all allocations are the caller's to free (rowptr, colidx, vals of T)
    if ((e = cudaMalloc(&T.rowptr, sizeof(int32_t) * (T.rows + 1 + kPadRowptr))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&T.colidx, sizeof(int32_t) * (nnz + kPadColidx))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&T.vals, sizeof(double) * (nnz + kPadVals))) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(T.rowptr, 0, sizeof(int32_t) * (T.rows + 1 + kPadRowptr), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(T.colidx, 0, sizeof(int32_t) * (nnz + kPadColidx), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(T.vals, 0, sizeof(double) * (nnz + kPadVals), s)) != cudaSuccess) return e;
    if (nnz == 0) return cudaStreamSynchronize(s);

    int32_t *rowof = nullptr, *seq = nullptr, *keys_out = nullptr, *perm = nullptr, *counts = nullptr;
    void* temp = nullptr;
    size_t temp_sort = 0, temp_scan = 0;
    int bits = 1;
    while (bits < 31 && (1LL << bits) < A.cols) ++bits;
    cub::DeviceRadixSort::SortPairs(nullptr, temp_sort, A.colidx, keys_out, seq, perm, (int)nnz, 0, bits, s);
    cub::DeviceScan::ExclusiveSum(nullptr, temp_scan, counts, T.rowptr, (int)(T.rows + 1), s);
    const size_t temp_bytes = temp_sort > temp_scan ? temp_sort : temp_scan;
    do {
        if ((e = cudaMalloc(&rowof, sizeof(int32_t) * nnz)) != cudaSuccess) break;
        if ((e = cudaMalloc(&seq, sizeof(int32_t) * nnz)) != cudaSuccess) break;
        if ((e = cudaMalloc(&keys_out, sizeof(int32_t) * nnz)) != cudaSuccess) break;
        if ((e = cudaMalloc(&perm, sizeof(int32_t) * nnz)) != cudaSuccess) break;
        if ((e = cudaMalloc(&counts, sizeof(int32_t) * (T.rows + 1))) != cudaSuccess) break;
        if ((e = cudaMalloc(&temp, temp_bytes)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (T.rows + 1), s)) != cudaSuccess) break;
        row_of_nonzero<<<blocks_for(nnz), kBlock, 0, s>>>(A.rowptr, A.rows, nnz, rowof, seq);
        count_cols<<<blocks_for(nnz), kBlock, 0, s>>>(A.colidx, nnz, counts);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        size_t ts = temp_bytes;
        if ((e = cub::DeviceRadixSort::SortPairs(temp, ts, A.colidx, keys_out, seq, perm, (int)nnz, 0,
                                                 bits, s)) != cudaSuccess) break;
        ts = temp_bytes;
        if ((e = cub::DeviceScan::ExclusiveSum(temp, ts, counts, T.rowptr, (int)(T.rows + 1), s)) !=
            cudaSuccess) break;
        gather_transposed<<<blocks_for(nnz), kBlock, 0, s>>>(perm, rowof, A.vals, nnz, T.colidx, T.vals);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        e = cudaStreamSynchronize(s);
    } while (false);
    cudaFree(rowof);
    cudaFree(seq);
    cudaFree(keys_out);
    cudaFree(perm);
    cudaFree(counts);
    cudaFree(temp);
    return e;
}

cudaError_t dense_transpose(cudaStream_t s, const double* A, int64_t rows, int64_t cols, double* T) {
    dim3 block(32, 8);
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    dense_transpose_kernel<<<grid, block, 0, s>>>(A, rows, cols, T);
    return cudaGetLastError();
}

}  // namespace tacta

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

#include <algorithm>
#include <climits>

#include "internal.h"
#include "dia_plan.cuh"

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

// Run-staged layout of fixed 256-row tiles, one block per tile (plan time). Per
// tile: row range and nonzero range, the window [lo, hi] of columns, the runs of
// used columns (a gap of more than kRunGap columns starts a new run; each run starts
// on a column that is a multiple of 4 and has a length that is a multiple of 4, so that
// FP64 and FP32 copies of x both move in 16-byte units) and each nonzero's 16-bit slot in the
// runs laid end to end. stats: [0] failure bits (1: a tile holds more than kRunCap
// nonzeros, 2: its window spans more than kXSpan columns, 4: more than kRunMax
// runs, 8: more than kRunXs staged entries), [1] max nonzeros of a tile, [2] max
// window span.
__global__ void __launch_bounds__(kTileRows)
run_tiles(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int64_t rows, int4* tiles,
          int2* xwin, int2* runs, uint16_t* lcol, int32_t* stats) {
    constexpr int kWords = (kXSpan + 31) / 32;
    __shared__ uint32_t used[kWords];
    __shared__ int lo_s, hi_s, fail_s, nrun_s;
    __shared__ int2 rr[kRunMax];
    const int t = blockIdx.x, tid = threadIdx.x;
    const int64_t r0 = (int64_t)t * kTileRows, r1 = min(rows, r0 + kTileRows);
    const int z = rowptr[r0], w = rowptr[r1];
    if (tid == 0) {
        lo_s = INT_MAX;
        hi_s = -1;
        fail_s = 0;
        nrun_s = 0;
        tiles[t] = make_int4((int)r0, (int)r1, z, w);
    }
    for (int i = tid; i < kWords; i += blockDim.x) used[i] = 0u;
    __syncthreads();
    int lo = INT_MAX, hi = -1;
    for (int k = z + tid; k < w; k += blockDim.x) {
        const int c = colidx[k];
        lo = min(lo, c);
        hi = max(hi, c);
    }
    atomicMin(&lo_s, lo);
    atomicMax(&hi_s, hi);
    __syncthreads();
    const int wlo = hi_s < 0 ? 0 : lo_s, whi = hi_s < 0 ? 0 : hi_s;
    const int span = whi - (wlo & ~1) + 1;
    if (tid == 0) {
        xwin[t] = make_int2(wlo, whi);
        atomicMax(&stats[1], w - z);
        atomicMax(&stats[2], span);
        if (w - z > kRunCap) fail_s |= 1;
        if (whi - wlo + 1 > kXSpan) fail_s |= 2;
    }
    __syncthreads();
    if (fail_s) {
        if (tid == 0) atomicOr(&stats[0], fail_s);
        return;
    }
    for (int k = z + tid; k < w; k += blockDim.x) {
        const int c = colidx[k] - wlo;
        atomicOr(&used[c >> 5], 1u << (c & 31));
    }
    __syncthreads();
    if (tid == 0 && w > z) {
        // runs, scanning the window's bitmap in column order
        int nrun = 0, total = 0, first = -1, last = -1, f = 0;
        auto close = [&]() {
            if (nrun == kRunMax) { f |= 4; return; }
            const int c0 = (wlo + first) & ~3;
            const int len = (wlo + last + 1 - c0 + 3) & ~3;
            rr[nrun++] = make_int2(c0, len);
            total += len;
            if (total > kRunXs) f |= 8;
        };
        const int width = whi - wlo + 1;
        for (int wd = 0; wd * 32 < width && !f; ++wd) {
            uint32_t bits = used[wd];
            while (bits && !f) {
                const int c = wd * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                if (first >= 0 && c - last > kRunGap) {
                    close();
                    first = -1;
                }
                if (first < 0) first = c;
                last = c;
            }
        }
        if (!f) close();
        nrun_s = nrun;
        fail_s = f;
        if (f) atomicOr(&stats[0], f);
    }
    __syncthreads();
    if (fail_s) return;
    if (tid < kRunMax) runs[(size_t)t * kRunMax + tid] = tid < nrun_s ? rr[tid] : make_int2(0, 0);
    for (int k = z + tid; k < w; k += blockDim.x) {
        const int c = colidx[k];
        int off = 0, r = 0;
        while (r + 1 < nrun_s && c >= rr[r].x + rr[r].y) off += rr[r++].y;
        lcol[k] = (uint16_t)(off + c - rr[r].x);
    }
}


// ------------------------------------------------------------------ diagonal form

constexpr int kDiaEmpty = INT_MIN;   // no offset: col - row > INT_MIN for int32 indices

// off into a set of kDiaMax slots (shared or global memory), first free slot in order,
// so that concurrent inserts of one value land in one slot; *ovf set when the set is full
__device__ void dia_insert(int* slots, int* ovf, int off) {
    for (int j = 0; j < kDiaMax; ++j) {
        int v = *(volatile int*)&slots[j];
        if (v == off) return;
        if (v == kDiaEmpty) {
            v = atomicCAS(&slots[j], kDiaEmpty, off);
            if (v == kDiaEmpty || v == off) return;
        }
    }
    atomicOr(ovf, 1);
}

__global__ void dia_init(int* slots, int* ovf) {
    if (threadIdx.x < kDiaMax) slots[threadIdx.x] = kDiaEmpty;
    if (threadIdx.x == 0) *ovf = 0;
}

// the distinct diagonals col - row (a set per block in shared memory, merged at the end)
__global__ void dia_offsets(const int32_t* rowptr, const int32_t* colidx, int64_t rows, int* slots, int* ovf) {
    __shared__ int ls[kDiaMax];
    __shared__ int lovf;
    if (threadIdx.x < kDiaMax) ls[threadIdx.x] = kDiaEmpty;
    if (threadIdx.x == 0) lovf = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
        if (*(volatile int*)&lovf) break;
        for (int32_t j = rowptr[r]; j < rowptr[r + 1]; ++j) dia_insert(ls, &lovf, colidx[j] - (int32_t)r);
    }
    __syncthreads();
    if (threadIdx.x < kDiaMax && ls[threadIdx.x] != kDiaEmpty) dia_insert(slots, ovf, ls[threadIdx.x]);
    if (threadIdx.x == 0 && lovf) atomicOr(ovf, 1);
}

// one thread per 256-row tile: its runs of x and slot bases (dia_tile_plan); fail: a tile
// needs more than kRunMax runs or kRunXs staged entries
__global__ void dia_tiles(int ntiles, int64_t rows, int64_t cols, DiaOffsets d, int2* runs, int32_t* sbase,
                          int* fail) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    if (!dia_tile_plan(rows, cols, d, t, runs + (size_t)t * kRunMax, sbase + (size_t)t * 8)) atomicOr(fail, 1);
}

// one thread per row: its values into the diagonal-major layout and its mask byte;
// fail: an entry off the diagonals or two entries on one (a repeated column)
__global__ void dia_fill(const int32_t* rowptr, const int32_t* colidx, const double* vals, int64_t rows, DiaOffsets d,
                         double* dvals, uint8_t* mask, int* fail) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += stride) {
        const int64_t t = r / kTileRows;
        const int lr = (int)(r % kTileRows);
        unsigned m8 = 0;
        for (int32_t j = rowptr[r]; j < rowptr[r + 1]; ++j) {
            const int off = colidx[j] - (int32_t)r;
            int k = -1;
            for (int i = 0; i < d.k; ++i)
                if (d.off[i] == off) k = i;
            if (k < 0 || ((m8 >> k) & 1u)) {
                atomicOr(fail, 1);
                continue;
            }
            m8 |= 1u << k;
            dvals[((size_t)t * d.k + k) * kTileRows + lr] = vals[j];
        }
        mask[r] = (uint8_t)m8;
    }
}

}  // namespace

cudaError_t run_tiles_build(cudaStream_t s, const DevCSR& a, int4* tiles, int2* xwin, int2* runs, uint16_t* lcol,
                            int32_t* stats) {
    const int ntiles = (int)((a.rows + kTileRows - 1) / kTileRows);
    cudaError_t e = cudaMemsetAsync(stats, 0, sizeof(int32_t) * 4, s);
    if (e != cudaSuccess || ntiles == 0) return e;
    run_tiles<<<ntiles, kTileRows, 0, s>>>(a.rowptr, a.colidx, a.rows, tiles, xwin, runs, lcol, stats);
    return cudaGetLastError();
}

cudaError_t dia_build(cudaStream_t s, const DevCSR& a, DevDIA& d, int* flag_dev, int* flag_host) {
    d = DevDIA{};
    if (a.rows == 0 || a.nnz == 0) return cudaSuccess;
    int* set = nullptr;
    int h[kDiaMax + 1];
    cudaError_t e = cudaMalloc(&set, sizeof(int) * (kDiaMax + 1));
    if (e != cudaSuccess) return e;
    auto drop = [&](cudaError_t err) {
        cudaFree(set);
        cudaFree(d.vals); cudaFree(d.mask); cudaFree(d.runs); cudaFree(d.sbase);
        d = DevDIA{};
        return err;
    };
    dia_init<<<1, 32, 0, s>>>(set, set + kDiaMax);
    dia_offsets<<<blocks_for(a.rows), kBlock, 0, s>>>(a.rowptr, a.colidx, a.rows, set, set + kDiaMax);
    if ((e = cudaGetLastError()) != cudaSuccess) return drop(e);
    if ((e = cudaMemcpyAsync(h, set, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return drop(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return drop(e);
    if (h[kDiaMax] != 0) return drop(cudaSuccess);   // more than kDiaMax diagonals
    DiaOffsets off{};
    for (int i = 0; i < kDiaMax; ++i)
        if (h[i] != kDiaEmpty) off.off[off.k++] = h[i];
    std::sort(off.off, off.off + off.k);
    const int ntiles = (int)((a.rows + kTileRows - 1) / kTileRows);
    if ((e = cudaMalloc(&d.runs, sizeof(int2) * kRunMax * ntiles)) != cudaSuccess) return drop(e);
    if ((e = cudaMalloc(&d.sbase, sizeof(int32_t) * 8 * ntiles)) != cudaSuccess) return drop(e);
    if ((e = cudaMemsetAsync(flag_dev, 0, sizeof(int), s)) != cudaSuccess) return drop(e);
    dia_tiles<<<(ntiles + kBlock - 1) / kBlock, kBlock, 0, s>>>(ntiles, a.rows, a.cols, off, d.runs, d.sbase,
                                                                flag_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return drop(e);
    if ((e = cudaMemcpyAsync(flag_host, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return drop(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return drop(e);
    if (*flag_host) return drop(cudaSuccess);
    const size_t nv = (size_t)ntiles * off.k * kTileRows;
    if ((e = cudaMalloc(&d.vals, sizeof(double) * nv)) != cudaSuccess) return drop(e);
    if ((e = cudaMalloc(&d.mask, (size_t)ntiles * kTileRows)) != cudaSuccess) return drop(e);
    if ((e = cudaMemsetAsync(d.vals, 0, sizeof(double) * nv, s)) != cudaSuccess) return drop(e);
    if ((e = cudaMemsetAsync(d.mask, 0, (size_t)ntiles * kTileRows, s)) != cudaSuccess) return drop(e);
    dia_fill<<<blocks_for(a.rows), kBlock, 0, s>>>(a.rowptr, a.colidx, a.vals, a.rows, off, d.vals, d.mask, flag_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return drop(e);
    if ((e = cudaMemcpyAsync(flag_host, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return drop(e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return drop(e);
    if (*flag_host) return drop(cudaSuccess);
    cudaFree(set);
    d.k = off.k;
    d.ntiles = ntiles;
    for (int i = 0; i < off.k; ++i) d.offsets[i] = off.off[i];
    return cudaSuccess;
}

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

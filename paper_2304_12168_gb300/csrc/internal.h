// Internal declarations shared by the translation units of libtacta.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/tacta.h"

namespace tacta {

constexpr int kTMax = 8;            // largest CTA order supported
constexpr int kBlock = 256;         // threads per block of every streaming kernel

// ---------------------------------------------------------------- control block
// One per plan, in device memory. Written only by single-thread "finisher"
// code (the last block of a reducing kernel) or by one-thread kernels, read
// by every kernel at entry. Kernel boundaries order all accesses.
struct Ctl {
    int32_t status;        // 0 while running, else a TACTA_REASON_* stop reason
    int32_t k;             // completed iterations (of the current TA trip)
    int32_t need_true;     // the next gated residual kernel must run
    int32_t is_true;       // the carried residual equals b - A x
    int32_t pivot;         // TA: this iteration takes a pivot step
    int32_t rank;          // CTA: rank of the last auxiliary solve
    int32_t max_iter;
    int32_t R;             // true-residual period (0: never)
    int32_t hist_cap;
    int32_t hist_len;
    int32_t grow_rho;      // TA: 1 = Alg. 2.2 (rho grows), 0 = Alg. 2.1 (witness stops)
    int32_t nonneg;        // TA for LP feasibility (Sec. 6): c replaced by max(c, 0)
    uint32_t counter;      // last-block-done ticket
    int32_t matvecs;       // products with A or Aᵀ made by the iteration (setup included)
    int32_t enhanced;      // CTA: the enhanced stop of Sec. 3.2 is on
    int32_t enh_stop;      // CTA: this step applies x^ and ends the solve (reason ENHANCED)
    uint32_t chain_bar;    // fused CTA chain: grid-wide arrivals (reset by the step's auxiliary kernel)
    double bn2;            // ||b||²  (b = rhs of the operator in use)
    double inv_bn2;        // 1 / ||b||² (0 when b = 0): the history stores ||r||² / ||b||²
    double mtbn2;          // ||Mᵀ b||²
    double tol2, tol_n2, pivot_tol;
    double res_thr, nrm_thr;
    double rn2;            // ||r||² (CTA) or ||d||² with d = b - b' (TA)
    double db;             // TA: dᵀ b
    double cn2;            // TA: ||c||²
    double s;              // TA: rho / ||c||
    double ta_alpha;       // TA: step
    double rho;            // TA: radius
    double rho_max;        // TA: termination bound on rho (infinity: none)
    double cs2;            // chain scale²: the chain's moments are cs2^k phi_k (1 on the FP64 path)
    double ref_eta2;       // mixed CTA: refine once ||r||² <= ref_eta2 * ||r||² at the last refinement (0: off)
    double ref_thr;        // that threshold, set by each true residual
    int64_t wait_cycles;   // fused chain: a grid-wide wait gives up after this many SM cycles
    int32_t loops;         // on-device loop: bodies run by the current graph launch
    int32_t loop_limit;    // ... and its bound (the loop also ends once status != 0)
    double phi[2 * kTMax + 2];
    double alpha[kTMax];
    double red[4];         // scratch results of setup reductions
};

// ---------------------------------------------------------------- reductions
enum Finisher : int {
    FIN_NONE = 0,
    FIN_STORE = 1,        // red[0..1] -> ctl->red[idx], ctl->red[idx+1]
    FIN_PHI = 2,          // r0 -> phi[idx]
    FIN_UNUSED_3 = 3,
    FIN_CTA_UPDATE = 4,   // r0 = ||r||²: k++, history, R-gate, loop-top tests
    FIN_TRUE_RES = 5,     // r0 = ||r||² (r1 = rᵀb): is_true, history, loop-top tests
    FIN_TA_C = 6,         // r0 = ||c||²: normal test, pivot test, rho growth / witness
    FIN_TA_V = 7,         // r0 = dᵀ(v - b'), r1 = ||v - b'||²: alpha
    FIN_TA_UPDATE = 8,    // r0 = ||d||², r1 = dᵀb: k++, history, R-gate, loop-top tests
    FIN_SETUP_B = 9,      // r0 = ||b||²
    FIN_SETUP_MTB = 10,   // r0 = ||Mᵀb||²: thresholds
    FIN_TRIP_START = 11,  // r0 = ||d||², r1 = dᵀb at the start of a TA trip: loop-top tests
    FIN_SETUP_RHO = 12    // r0 = ||x0||²: rho = ||x0|| (TA warm start)
};

struct FinArgs {
    int kind;
    int idx;              // FIN_PHI / FIN_STORE slot
    double* hist;         // device history buffer (capacity ctl->hist_cap)
    int reset_bar = 0;    // the finisher also resets the fused step's grid-wide counter
};

// Epilogues of the matrix-vector kernels: y = A x, then per row
enum Epilogue : int {
    EPI_NONE = 0,      // y = A x
    EPI_NORM = 1,      // y = A x;          red0 += y²
    EPI_RESID = 2,     // y = b - A x;      red0 += y², red1 += y b
    EPI_TAPIVOT = 3,   // v = s (A x); y = w = v - b + d (= v - b'); red0 += d w, red1 += w²
    EPI_RESID_F32 = 4, // FP64 product, v = b - A x; yf = (float) v; red0 += v², red1 += v b
    EPI_NORM_POS = 5   // y = max(A x, 0);  red0 += y²  (c_+ of TA for LP feasibility)
};

struct EpiArgs {
    const double* b;   // EPI_RESID / EPI_TAPIVOT / EPI_RESID_F32: right-hand side
    const double* d;   // EPI_TAPIVOT: d = b - b'
    float* yf;         // EPI_RESID_F32: FP32 copy of the residual
};

// Gate: which device flag must be set for the kernel to run (all kernels
// also return immediately when ctl->status != 0).
enum Gate : int { GATE_ALWAYS = 0, GATE_NEED_TRUE = 1, GATE_PIVOT = 2,
                  GATE_FORCE = 3 /* runs even after a stop (exit diagnostics) */ };

// ---------------------------------------------------------------- device matrix
struct SpmvCfg {
    int kind;      // 0 scalar (thread per row), 1 warp per row, 2 TMA-staged row tiles
    int grid;      // blocks
};

// Row tiles of the staged CSR kernel: rows [x, y), nonzeros [z, w); at most
// kTileRows rows and `cap` nonzeros per tile (built at plan time).
constexpr int kTileRows = 256;
constexpr int kTileCapSmall = 2048;   // 4 blocks per SM
constexpr int kTileCapLarge = 8192;   // 1 block per SM

// Diagonal form of a banded operand whose nonzeros lie on at most kDiaMax diagonals
// (col - row = offset_k), in fixed kTileRows-row tiles: the values by tile, diagonal and
// row ([tile][k][kTileRows], zero where a row lacks diagonal k), one byte per row with bit
// k set where the row stores diagonal k, the tile's runs of x and, per tile and diagonal,
// the slot of x[first row + offset_k] in those runs laid end to end. Built on the device
// at plan time (transpose.cu); used by the fused chain.
constexpr int kDiaMax = 5;
struct DevDIA {
    int k = 0;                   // diagonals; 0 = not in diagonal form
    int ntiles = 0;
    int offsets[kDiaMax] = {};   // ascending (host copy)
    double* vals = nullptr;      // ntiles * k * kTileRows
    float* vals32 = nullptr;     // FP32 copy for the mixed-precision chain (made on first use)
    uint8_t* mask = nullptr;     // ntiles * kTileRows
    int2* runs = nullptr;        // ntiles * kRunMax {first column, length}
    int32_t* sbase = nullptr;    // ntiles * 8
};

struct DevCSR {          // CSR operand in device memory (rows x cols)
    int64_t rows = 0, cols = 0, nnz = 0;
    int32_t* rowptr = nullptr;   // rows + 1 (+ 4 padding)
    int32_t* colidx = nullptr;   // nnz (+ 4 padding)
    double* vals = nullptr;      // nnz (+ 2 padding)
    int4* tiles = nullptr;       // kind 2: tile descriptors
    int ntiles = 0;
    int cap = 0;                 // kind 2: nonzero capacity of a tile
    int2* xwin = nullptr;        // kind 3: per tile {first column, last column} of its x window
    // kind 3 operands whose tiles draw on at most kRunMax short runs of x also carry:
    uint16_t* lcol = nullptr;    // per nonzero: its column's slot in the tile's staged runs (nnz + kPadLcol)
    int2* runs = nullptr;        // per tile kRunMax {first column, length} (multiples of 4; length 0 = unused)
    SpmvCfg cfg{};
    DevDIA dia;                  // diagonal form, when the operand has one (fused chain)
};

// Banded operands (every tile's columns span at most kXSpan entries of x) also
// stage the tile's x window in shared memory: kind 3.
constexpr int kXSpan = 2560;
constexpr int kXCapCompactPlan = 1280, kXSpanCompactPlan = 2304;   // compact x-window instance
// Run-staged operands: a tile's distinct columns form at most kRunMax runs (a gap of
// more than kRunGap columns starts a new run) of kRunXs entries of x in total, and the
// tile holds at most kRunCap nonzeros. Only those runs of x are staged, and column
// indices shrink to 16-bit slots in them.
constexpr int kRunCap = 1280, kRunXs = 896, kRunMax = 4, kRunGap = 16;
constexpr int kPadLcol = 8;
// ring depth of the warp-specialised run-staged product
constexpr int kRwStages = 3;
// Mixed-precision CTA refines (FP64 residual, fold of the FP32 correction) as soon as
// the FP32 inner iteration has reduced the residual by kRefineEta over the last
// refinement; the FP32 chain cannot resolve much more than that.
constexpr double kRefineEta2 = 1e-6;
// batched dense systems: rows and columns of each system at most this
constexpr int32_t kBatchMaxDim = 4096;
// every plan vector that can be a product's input carries this many doubles of
// padding, so 16-byte-rounded x-window copies stay inside the allocation
constexpr int kPadVec = 4;

// padding (elements) after each CSR array so that 16-byte-rounded bulk copies
// of a tile window never leave the allocation
constexpr int kPadRowptr = 4, kPadColidx = 4, kPadVals = 2;

struct DevDense {        // dense row-major operand in device memory
    int64_t rows = 0, cols = 0;
    double* vals = nullptr;
    SpmvCfg cfg{};
};

struct DevOperand {      // A or Aᵀ
    int format = TACTA_CSR;
    DevCSR csr;
    DevDense dense;
    int64_t rows() const { return format == TACTA_CSR ? csr.rows : dense.rows; }
    int64_t cols() const { return format == TACTA_CSR ? csr.cols : dense.cols; }
    int64_t nnz() const { return format == TACTA_CSR ? csr.nnz : dense.rows * dense.cols; }
};

// FP32 copy of a CSR operand for the mixed-precision path: values in FP32, the
// structure (rowptr, colidx, tiles, x windows) shared with the FP64 operand.
struct DevCSR32 {
    const DevCSR* base = nullptr;
    float* vals = nullptr;       // nnz (+ 4 padding)
};
constexpr int kPadVals32 = 4;
constexpr int kPadVec32 = 4;     // FP32 vectors read by products carry 4 floats of padding

// ---------------------------------------------------------------- kernel launchers
struct LaunchCtx {
    cudaStream_t stream;
    Ctl* ctl;
    double* partials;     // >= 2 * max grid doubles
    int max_grid;         // blocks of reducing kernels (fixed per plan)
    int64_t* launches;    // counter of launched kernels
};

cudaError_t launch_spmv(const LaunchCtx& L, const DevOperand& A, const double* x, double* y,
                        int epi, EpiArgs e, FinArgs f, int gate);
cudaError_t launch_cta_update(const LaunchCtx& L, int t, int64_t m, int64_t n,
                              double* x, double* r, double* const* z, double* const* u,
                              FinArgs f);
cudaError_t launch_ta_update(const LaunchCtx& L, int64_t m, int64_t n, double* x, double* d,
                             const double* b, const double* v, const double* c, FinArgs f);
cudaError_t launch_reduce_vec(const LaunchCtx& L, int64_t len, const double* a, const double* b,
                              FinArgs f, int gate);
cudaError_t launch_ctl_init(const LaunchCtx& L, const Ctl& host_init);
cudaError_t launch_copy_gated(const LaunchCtx& L, double* dst, const double* src, int64_t len, int gate);
cudaError_t launch_fill(const LaunchCtx& L, double* dst, double v, int64_t len);
cudaError_t launch_hist_sqrt(cudaStream_t s, double* h, int64_t len);   // ||r||²/||b||² -> ||r||/||b||
// CTA step decision + auxiliary solve; with part != nullptr the moments phi_1..phi_2t are
// first summed from the fused chain's per-block partials (part[(i - 1) * G + block])
cudaError_t launch_cta_aux_step(const LaunchCtx& L, int t, const double* part = nullptr, int G = 0);

// The fused CTA chain (chain.cu): both operands run-staged; index 0 is Aᵀ, 1 is A.
template <typename V>
struct ChainOps {
    const int4* tiles[2];
    const int2* runs[2];
    const int32_t* rowptr[2];
    const uint16_t* lcol[2];
    const V* vals[2];
    int ntiles[2];
};
template <typename V>
struct ChainVecs {
    const V* r;          // u_0
    V* z[kTMax];         // z_i = Aᵀ u_{i-1}
    V* u[kTMax];         // u_i = A z_i
};
template <typename V>
struct ChainOpsDia {             // the fused chain on operands in diagonal form; index 0 is Aᵀ, 1 is A
    const V* vals[2];
    const uint8_t* mask[2];
    const int2* runs[2];
    const int32_t* sbase[2];
    int ntiles[2];
    int rows[2];
    int k;                       // diagonals (the same for A and Aᵀ)
};
// The rest of a fused F_t step (chain.cu): after the products every block solves the
// auxiliary equation and updates its slice of x and r; the last block runs the update's
// finisher (step count, history, stop tests).
template <typename V>
struct StepArgs {
    V* x = nullptr;          // FP64 chain: x; FP32 chain: dx, the correction since the last refinement
    V* r = nullptr;          // the residual, u_0 of the next step
    int64_t m = 0, n = 0;
    float xscale = 1.0f;     // FP32 chain: z_i carries a scale, x += xscale sum alpha_i z_i
    double* hist = nullptr;  // history buffer of the finisher
    double* upart = nullptr; // per-block partials of ||r||² (2 doubles per block)
    const double* b = nullptr; // FP64 chain: the right-hand side, for the true residual of
                               // a step that starts with one (ctl->need_true)
    double* rpart = nullptr;   // its per-block partials: ||r||² then rᵀb (G each)
    int nsteps = 1;            // F_t steps per launch (the launch stops early at a stop, and
                               // on the FP32 chain when a refinement is due)
    int t_max = 5, cycle = 0;  // the order of step k follows the cycle from the device's k
};
// blocks of the cooperative chain launch (all resident), 0 if it cannot run here
int cta_chain_grid(int sms, int max_tiles, bool fp32, bool dia);
// sa == nullptr: the 2t products only (cta_aux_step and the update kernel follow);
// else the whole F_t step in the one launch
cudaError_t launch_cta_chain_dia(const LaunchCtx& L, const ChainOpsDia<double>& ops, const ChainVecs<double>& v,
                                 int t, double* part, int grid, const StepArgs<double>* sa);
cudaError_t launch_cta_chain_dia32(const LaunchCtx& L, const ChainOpsDia<float>& ops, const ChainVecs<float>& v,
                                   int t, float scale, double* part, int grid, const StepArgs<float>* sa);
// diagonal form of a CSR operand (d.k = 0 when it has none); flag: 2 ints of device scratch
cudaError_t dia_build(cudaStream_t s, const DevCSR& a, DevDIA& d, int* flag_dev, int* flag_host);
cudaError_t launch_cta_chain(const LaunchCtx& L, const ChainOps<double>& ops, const ChainVecs<double>& v, int t,
                             double* part, int grid, const StepArgs<double>* sa);
cudaError_t launch_cta_chain32(const LaunchCtx& L, const ChainOps<float>& ops, const ChainVecs<float>& v, int t,
                               float scale, double* part, int grid, const StepArgs<float>* sa);

// mixed precision (FP32 chain, FP64 refinement)
cudaError_t launch_spmv32(const LaunchCtx& L, const DevCSR32& A, const float* x, float* y, float scale,
                          int epi, FinArgs f, int gate);
cudaError_t launch_cta_update32(const LaunchCtx& L, int t, int64_t m, int64_t n, float* dx, float* r,
                                float* const* z, float* const* u, float xscale, FinArgs f);
cudaError_t abs_row_sum_max(cudaStream_t s, const DevCSR& A, double* dev_out, double* host_out);
// dense FP32 product of the mixed-precision chain (row-major A, rows x cols): y = (A x) *
// scale, ||y||² to the finisher
cudaError_t launch_dense32(const LaunchCtx& L, int64_t rows, int64_t cols, const float* A, const float* x,
                           float* y, float scale, FinArgs f, int gate);
cudaError_t dense32_prepare();   // kernel attributes of the dense FP32 product (before any capture)
cudaError_t dense_abs_row_sum_max(cudaStream_t s, int64_t rows, int64_t cols, const double* vals, double* dev_out,
                                  double* host_out);
cudaError_t launch_outer_on_pattern(cudaStream_t s, int grid, const DevOperand& A, double alpha, const double* u,
                                    const double* v, double* out);
cudaError_t launch_fold_correction(const LaunchCtx& L, int64_t n, double* x, float* dx, int gate);
// on-device iteration loop (a graph WHILE node): loop_begin resets the body count and sets
// its bound before the graph launch; loop_continue, the body's last kernel, counts the
// body and sets the node's condition to (status == 0 and count < bound)
cudaError_t launch_loop_begin(cudaStream_t s, Ctl* ctl, int32_t limit);
cudaError_t launch_loop_continue(cudaStream_t s, Ctl* ctl, cudaGraphConditionalHandle h);
cudaError_t convert_to_f32(cudaStream_t s, const double* src, float* dst, int64_t len);
cudaError_t spmv32_prepare();

cudaError_t spmv_tiled_prepare();   // raises the dynamic shared-memory limit of the tiled kernels
size_t spmv_tiled_smem(int cap);

// plan-time helpers (transpose.cu)
cudaError_t csr_validate(cudaStream_t s, const int32_t* rowptr, const int32_t* colidx, int64_t m,
                         int64_t n, int64_t nnz, int* flag_dev, int* flag_host);
cudaError_t csr_transpose(cudaStream_t s, const DevCSR& A, DevCSR& T);
cudaError_t dense_transpose(cudaStream_t s, const double* A, int64_t rows, int64_t cols, double* T);
// run-staged layout of fixed kTileRows-row tiles built on the device (stats: 4 int32 on
// the device; [0] failure bits, [1] max nonzeros per tile, [2] max window span)
cudaError_t run_tiles_build(cudaStream_t s, const DevCSR& a, int4* tiles, int2* xwin, int2* runs, uint16_t* lcol,
                            int32_t* stats);

// ---------------------------------------------------------------- small dense A on chip
// CTA on a dense A that fits the shared memory of one thread-block cluster (dense_cluster.cu):
// whole F_t steps in one launch, A and Aᵀ split by rows over the cluster's blocks.
struct DenseClusterArgs {
    const double* A;         // m x n row-major (device)
    const double* At;        // n x m row-major (device)
    int64_t m, n;
    double* x;               // n: read at entry, written at exit
    double* r;               // m: the carried residual, read at entry, written at exit
    const double* b;         // m
    double* hist;            // history buffer
    int nsteps, t_max, cycle;
};
// blocks of the cluster (16 or 8) that hold an m x n system, 0 if none does on this device
int dense_cluster_size(int64_t m, int64_t n);
cudaError_t launch_cta_dense_cluster(const LaunchCtx& L, const DenseClusterArgs& a, int C);

// ---------------------------------------------------------------- per-device one-time setup
// Kernel attributes (the dynamic shared-memory opt-in above 48 KB) are per device, so a
// process-wide "done" flag would leave a second device without them. done_on_device(key)
// tells whether the setup identified by `key` (the address of a static of the caller) has
// succeeded on the current device; mark_done_on_device records it. Thread-safe; two threads
// racing through the same setup both run it, which is harmless for attribute setters.
bool done_on_device(const void* key);
void mark_done_on_device(const void* key);

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
const char* get_error();

}  // namespace tacta

// Host-side internals of libspgemm: plan, workspace layout, kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/spgemm.h"
#include "common.cuh"

namespace spg {
// Kernel ids for launch counting and per-kernel CUDA-event timing.
enum KernelId : int {
    K_FILL, K_CHECK_RPT, K_ZERO, K_IP_COUNT, K_SUM, K_GROUP_HIST, K_GROUP_SCAN, K_GROUP_SCATTER,
    K_SCAN_PART, K_SCAN_TOP, K_SCAN_FINAL, K_RESET, K_BPANEL, K_SYM_ESC, K_SYM_WARP, K_SYM_BLOCK,
    K_SYM_DENSE, K_NUM_ESC, K_NUM_WARP32, K_NUM_WARP64, K_NUM_BLOCK32, K_NUM_BLOCK64,
    K_NUM_DENSE32, K_NUM_DENSE64, K_BWD, K_GUARD, K_MCL, K_HOT, K_LAYER, K_SYM_NARROW,
    K_NUM_NARROW, K_GEMM, K_NUM_KERNELS
};
extern const char* const kKernelNames[K_NUM_KERNELS];

struct ProfState {
    int on = 0;
    int n = 0;
    int cap = 0;
    int* kid = nullptr;
    cudaEvent_t* ev = nullptr;
    unsigned long long launches = 0;        // all launches since plan creation
};
}  // namespace spg

struct spgemm_plan {
    spg::ProfState* prof;
    int device;
    int num_sms;
    size_t smem_optin;     // max dynamic shared memory per block
    spgemm_opts opts;
    // resident blocks per SM for each persistent kernel (filled at creation)
    int occ_sym_warp, occ_sym_block, occ_sym_dense;
    int occ_num_warp32, occ_num_warp64, occ_num_block32, occ_num_block64;
    int occ_num_block32s, occ_num_block64s;   // quarter- and half-size table launches of the block tier
    int occ_num_block32m, occ_num_block64m;
    int occ_num_dense32, occ_num_dense64, occ_num_dense_hot;
    int hot_ppp;           // table panels per pass of the fp64 dense tier
    int d32_ppp;           // and of the fp32 dense tier
    size_t rank_budget;    // dynamic shared memory of the rank-compacted fp32 dense kernel
    int occ_num_rank;
    int hotr_cap, hotr_pmax;   // rank-compacted fp64 dense kernel: value slots, panels per pass
    int occ_sym_staged;        // staged block hash tier of the allocation phase
    int occ_sym_block_small;   // its two lighter bins with a quarter-size table
    int occ_sym_block_mid;     // its second bin with a half-size table
};

namespace spg {

constexpr int kBinRows = 1024;      // rows per block in the grouping kernels
constexpr int kScanItems = 4096;    // rows per block in the row-pointer scan
constexpr int kWarpTableSym = 2048; // keys per warp, allocation warp tier
constexpr int kWarpsPerBlockSW = 8;
constexpr int kWarpTableNum = 1024; // entries per warp, accumulation warp tier
constexpr int kWarpsPerBlockNW = 8;
constexpr int kSymBlockThreads = 512;
constexpr int kSymDenseThreads = 1024;
constexpr int kNumBlockThreads = 512;
constexpr int kBlockThreadsFull = 1024;   // block tiers' full-size-table launches
// A entries a row of the fp32 rank-compacted dense kernel may have (its
// expansion tile); rows with more take the dense-array fallback kernel
constexpr int kRankTileEntries = 256;
constexpr int kNumDenseThreads = 1024;
constexpr int kMaxPanels = 1024;    // above this the heavy path filters whole B rows

// Bins (phase-specific meaning). Allocation phase:
//   0: in-register tier, 1: warp hash, 2..5: block hash (by log2 IP, heavy
//   first), 6..37: dense bitmap (by log2 IP, heavy first), 63: nothing to do.
// Accumulation phase:
//   0: in-register tier, 1/2: warp hash fp32/fp64, 3/4: block hash fp32/fp64,
//   5..20: dense panels fp32, 21..36: dense panels fp64 (by log2 IP, heavy
//   first), 39/40: block hash fp32/fp64 for rows of at most a quarter of
//   block_max_nnz entries (a quarter-size table, several blocks per SM),
//   41/42: the same for rows of at most half (a half-size table),
//   63: nothing to do.
enum : int {
    SB_ESC = 0, SB_WARP = 1, SB_BLOCK0 = 2, SB_BLOCK_N = 4, SB_DENSE0 = 6, SB_DENSE_N = 32,
    NB_ESC = 0, NB_WARP32 = 1, NB_WARP64 = 2, NB_BLOCK32 = 3, NB_BLOCK64 = 4,
    NB_DENSE32_0 = 5, NB_DENSE_N = 16, NB_DENSE64_0 = 21,
    SB_NARROW = 38, NB_NARROW32 = 37, NB_NARROW64 = 38, NB_BLOCK32S = 39, NB_BLOCK64S = 40,
    NB_BLOCK32M = 41, NB_BLOCK64M = 42
};

// rows of the accumulation block tier that take the quarter- and half-size
// table launches
__host__ __device__ inline int block_small_nnz(const spgemm_opts& o) { return o.block_max_nnz / 4; }
__host__ __device__ inline int block_mid_nnz(const spgemm_opts& o) { return o.block_max_nnz / 2; }

// Narrow tiers: when B has at most kNarrowCols columns, rows with at most
// kNarrowMaxIP products take one warp each with a dense per-warp
// accumulator over all of B's columns (no hashing, no sort).
constexpr int kNarrowCols = 1024;
constexpr long long kNarrowMaxIP = 32768;   // default of opts.narrow_max_ip
constexpr int kNarrowWarpsDefault = 8;      // default of opts.narrow_warps
constexpr int kNarrowMaxWarps = 16;
inline int narrow_warps(const spgemm_plan* p) {
    return p->opts.narrow_warps > 0 ? p->opts.narrow_warps : kNarrowWarpsDefault;
}
inline int hash_load(const spgemm_plan* p) {
    return p->opts.hash_load_pct > 0 ? p->opts.hash_load_pct : 50;
}
__host__ __device__ inline long long narrow_max_ip(const spgemm_opts& o) {
    return o.narrow_max_ip > 0 ? o.narrow_max_ip : kNarrowMaxIP;
}

// Backward tiers (grouping phase 3, by nnz of the row of C): dense lookup
// when B has few columns, warp hash, block hash, dense column panels.
constexpr int kBwdDenseCols = 2048;
constexpr int kBwdWarpSlots = 1024;
constexpr int kBwdBlockSlots = 16384;
enum : int { BW_DENSE = 0, BW_WARP = 1, BW_BLOCK = 2, BW_PANEL = 3 };

// Workspace layout: all offsets 256-byte aligned, derived from shapes only.
struct WsLayout {
    size_t ctl = 0;          // Ctl
    size_t map = 0;          // int32 [m]
    size_t blk_counts = 0;   // int32 [kNumBins][nblk]
    size_t scan_part = 0;    // int64 [nscan + 1]
    size_t bpanel = 0;       // int32 [B.rows][P+1]  (0 bytes when P > kMaxPanels)
    size_t colcnt = 0;       // int32 [B.cols+1]  entries per column of B, then hot flags
    size_t hot_rank = 0;     // int32 [B.cols+1]  exclusive prefix of the hot flags
    size_t hot_col = 0;      // int32 [B.cols]    hot columns in ascending order
    size_t bhot = 0;         // int32 [B.nnz]     each B entry's column, or (sign bit | hot rank)
    size_t bhv = 0;          // int2 [B.nnz]      (bhot, value bits) per B entry, packed per call
    size_t bcv = 0;          // int2 [B.nnz]      (column, value bits) per B entry, packed per call
    size_t rc_slot = 0;      // int32 [m]         row -> bitmap slot (-1: none)
    size_t rc_bits = 0;      // u32 [rc_nslots][rc_wpr] row bitmaps of the allocation phase
    size_t rc_pc = 0;        // int [rc_nslots][panels] entries of each table panel of a cached row
    int rc_nslots = 0, rc_wpr = 0;
    bool has_hot = false;
    size_t total = 0;
    int m = 0, nblk = 0, nscan = 0, panels = 0;
};

WsLayout ws_layout(const spgemm_plan* p, long long m, long long b_rows, long long b_cols,
                   long long b_nnz = 0);

struct WsPtrs {
    Ctl* ctl;
    int* map;
    int* blk_counts;
    long long* scan_part;
    int* bpanel;
    int* colcnt;
    int* hot_rank;
    int* hot_col;
    int* bhot;
    int2* bhv;
    int2* bcv;
    int* rc_slot;            // nullptr: no row bitmap cache
    unsigned* rc_bits;
    int* rc_pc;              // per-panel entry counts of the cached rows, or nullptr
    int rc_nslots, rc_wpr;
    int nblk, nscan, panels, panel_cols;
};

// Row bitmap cache: rows of B.cols bits, written by the allocation phase's
// bitmap tier for rows the accumulation phase takes in a dense tier.
constexpr int kRowCacheMaxWords = 48 * 1024;   // one bitmap pass of the allocation tier

WsPtrs ws_ptrs(const WsLayout& L, void* ws, int panel_cols);

// Launchers (stream-ordered, no host synchronisation).
void launch_fill_i64(const spgemm_plan* pl, long long* p, long long n, long long v, cudaStream_t s);
void launch_ip_count(const spgemm_plan* p, const CsrDev& A, const CsrDev& B, long long* ip,
                     const WsPtrs& w, cudaStream_t s);

// Grouping: phase 0 = allocation, 1 = accumulation, 2 = generic thresholds.
struct GroupArgs {
    int phase;
    int row_begin, n;          // rows [row_begin, row_begin + n) of A
    const long long* ip;       // indexed by absolute row
    const int* rptA;           // A row pointers (absolute rows)
    const int* rptC;           // accumulation: block-relative row pointers of C
    int* row_nnz;              // allocation: rows settled during grouping (IP <= 1)
    const long long* key;      // generic: keys (n)
    const long long* thr;      // generic: thresholds
    int nthr;
    int bcols;                 // columns of B (narrow tiers, backward dense tier)
    const int* rc_slot;        // accumulation: row bitmap cache slots, or nullptr
    spgemm_opts opts;
};
void launch_group(const spgemm_plan* p, const GroupArgs& g, const WsPtrs& w, int* map_out,
                  int* offsets_out, cudaStream_t s);

void launch_row_ptr(const spgemm_plan* p, const int* row_nnz, int n, const WsPtrs& w,
                    int* row_ptr, cudaStream_t s);

void launch_symbolic(const spgemm_plan* p, const CsrDev& A, const CsrDev& B, const long long* ip,
                     const WsPtrs& w, int* row_nnz, cudaStream_t s);
void launch_nnz_total(const spgemm_plan* p, const int* row_nnz, int n, const WsPtrs& w, cudaStream_t s);

// capacity >= 0: the tiers run only if rptC[n] <= capacity and no overflow
// was flagged (otherwise ST_BUDGET is recorded and nothing is written).
void launch_numeric(const spgemm_plan* p, const CsrDev& A, const CsrDev& B, const long long* ip,
                    int row_begin, int row_end, const int* rptC, const WsPtrs& w, int* colC,
                    float* valC, cudaStream_t s, long long capacity = -1);
void launch_bpanel(const spgemm_plan* p, const CsrDev& B, const WsPtrs& w, cudaStream_t s);
void launch_hot(const spgemm_plan* p, const CsrDev& B, const WsPtrs& w, cudaStream_t s);
void launch_copy_total(const spgemm_plan* p, const WsPtrs& w, int which, long long* dst,
                       cudaStream_t s);

void launch_backward(const spgemm_plan* p, const CsrDev& A, const CsrDev& B, const int* rptC,
                     const int* colC, const float* dC, float* dA, float* dB, const WsPtrs& w,
                     double* dB64, double* dA64, cudaStream_t s);
size_t backward_extra_bytes(long long a_nnz, long long b_nnz);
__global__ void k_fill_i32(int* p, long long n, int v);
void launch_sample_rows(const spgemm_plan* p, const CsrDev& P, int s, const float* u, int mode,
                        const WsPtrs& w, int* rpt_out, int* col_out, float* val_out,
                        cudaStream_t st);
void launch_select_columns(const spgemm_plan* p, const CsrDev& Q, const WsPtrs& w, int* S_rpt,
                           int* S_col, float* S_val, int* F_rpt, int* F_col, float* F_val,
                           cudaStream_t st);
void launch_topk(const spgemm_plan* p, const float* X, int n, int d, long long ldx, int k,
                 int* rpt, int* col, float* val, cudaStream_t s);
void launch_scatter_dense(const spgemm_plan* p, const CsrDev& M, const float* vals, float* X,
                          long long ldx, Ctl* ctl, cudaStream_t s);
void launch_gather_dense(const spgemm_plan* p, const CsrDev& M, const float* D, long long ldd,
                         float* out, Ctl* ctl, cudaStream_t s);
void launch_mcl_step(const spgemm_plan* p, const CsrDev& E, float theta, int k, double r,
                     int order, const WsPtrs& w, int* rpt_out, int* col_out, float* val_out,
                     cudaStream_t s);

// Dense fp32 GEMM C = op(A) * op(B) (row-major, leading dimensions); with
// acc (fp64, M*N) the reduction is split over ksplit blocks along K.
void launch_sgemm(const spgemm_plan* p, int M, int N, int K, const float* A, long long lda,
                  bool ta, const float* B, long long ldb, bool tb, float* C, long long ldc,
                  double* acc, int ksplit, cudaStream_t s);
int gemm_ksplit(const spgemm_plan* p, int M, int N, int K);

void init_occupancy(spgemm_plan* p);
// Lets kernel f take as much dynamic shared memory as the device allows
// beside f's static arrays. The limit is a per-kernel, process-wide
// attribute, so plans with different table sizes must not set it to their
// own request (a later plan with smaller tables would lower it under an
// earlier plan's launches); each plan's occupancy uses its actual request.
void allow_max_dynamic_smem(const void* f, const spgemm_plan* p);

void prof_begin(const spgemm_plan* p, int kid, cudaStream_t s);
void prof_end(const spgemm_plan* p, int kid, cudaStream_t s);

// Launch a kernel with launch counting and (when enabled) event timing.
#define SPG_LAUNCH(plan, kid, stream, ...)            \
    do {                                              \
        ::spg::prof_begin((plan), (kid), (stream));   \
        __VA_ARGS__;                                  \
        ::spg::prof_end((plan), (kid), (stream));     \
    } while (0)

}  // namespace spg

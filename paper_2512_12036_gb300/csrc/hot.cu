// Hot columns of B, for the precision split of the heavy-row accumulation.
//
// An output entry c_ij gathers one product per stored entry of B in column j
// that row i of A selects, so at most colcount_B(j) products: a column that
// at most fp32_max_terms entries of B hold ("cold") can be summed in fp32 in
// any row within the 1e-5 * sum|a||b| bound, whatever the row's length.
// Only the remaining ("hot") columns need fp64. This pass, run once per B
// with the panel table, builds
//   colcnt   entries of B per column, then turned into hot flags (0/1),
//   hot_rank exclusive prefix of the flags (the rank of a hot column),
//   hot_col  the hot columns in ascending order,
//   bhot     for every stored entry of B its column, or for a hot column
//            (sign bit | hot rank),
// so the fp64 dense tier reads an entry's column and hotness with one
// coalesced load beside val.
#include "internal.h"

namespace spg {

__global__ void k_fill_i32(int* p, long long n, int v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// Entries per column. Few columns (<= kColSmem): a shared-memory histogram
// per block, added to cnt once per block (B = a narrow feature matrix puts
// millions of entries on each column). Otherwise lanes of a warp that hold
// the same column add their count with one atomic.
constexpr int kColSmem = 8192;

__global__ void k_colcount_smem(CsrDev B, int* cnt) {
    __shared__ int h[kColSmem];
    for (int i = threadIdx.x; i < B.cols; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const long long J0 = B.rows > 0 ? B.rpt[0] : 0;
    const long long J1 = B.rows > 0 ? B.rpt[B.rows] : 0;
    if (J0 >= 0 && J1 >= J0 && J1 <= B.nnz) {
        for (long long j = J0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; j < J1;
             j += (long long)gridDim.x * blockDim.x) {
            const int c = B.col[j];
            if ((unsigned)c < (unsigned)B.cols) atomicAdd(&h[c], 1);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < B.cols; i += blockDim.x)
        if (h[i]) atomicAdd(&cnt[i], h[i]);
}

__global__ void k_colcount(CsrDev B, int* cnt) {
    const long long J0 = B.rows > 0 ? B.rpt[0] : 0;
    const long long J1 = B.rows > 0 ? B.rpt[B.rows] : 0;
    if (J0 < 0 || J1 < J0 || J1 > B.nnz) return;
    const int lane = lane_id();
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    // warp-uniform trip count: all 32 lanes take part in every match
    for (long long base = J0 + warp * 32; base < J1; base += nwarps * 32) {
        const long long j = base + lane;
        const int c = j < J1 ? B.col[j] : -1;
        const bool ok = (unsigned)c < (unsigned)B.cols;
        const unsigned peers = __match_any_sync(kFull, ok ? c : -1);
        if (ok && lane == __ffs(peers) - 1) atomicAdd(&cnt[c], __popc(peers));
    }
}

__global__ void k_hot_flags(int* cnt, int ncols, int thr) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncols;
         c += (long long)gridDim.x * blockDim.x)
        cnt[c] = cnt[c] > thr ? 1 : 0;
}

__global__ void k_hot_cols(const int* flag, const int* rank, int ncols, int* hot_col) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncols;
         c += (long long)gridDim.x * blockDim.x)
        if (flag[c]) hot_col[rank[c]] = (int)c;
}

// bhot[j]: B's column j with hot columns replaced by (sign bit | hot rank),
// and out-of-range columns by INT_MAX (which every column check rejects)
__global__ void k_bhot(CsrDev B, const int* flag, const int* rank, int* bhot) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < B.nnz;
         j += (long long)gridDim.x * blockDim.x) {
        const int c = B.col[j];
        if ((unsigned)c >= (unsigned)B.cols) bhot[j] = 0x7fffffff;
        else bhot[j] = flag[c] ? (int)(0x80000000u | (unsigned)rank[c]) : c;
    }
}

void launch_hot(const spgemm_plan* p, const CsrDev& B, const WsPtrs& w, cudaStream_t s) {
    // only rows with more than block_max_nnz entries (so B.cols > block_max_nnz)
    // reach the fp64 dense tier, the one reader of these tables
    if (!w.colcnt || B.cols <= 0 || B.cols <= p->opts.block_max_nnz) return;
    const int grid = p->num_sms * 8;
    SPG_LAUNCH(p, K_HOT, s, k_fill_i32<<<grid, 256, 0, s>>>(w.colcnt, (long long)B.cols + 1, 0));
    if (B.nnz > 0) {
        if (B.cols <= kColSmem)
            SPG_LAUNCH(p, K_HOT, s, k_colcount_smem<<<grid, 256, 0, s>>>(B, w.colcnt));
        else
            SPG_LAUNCH(p, K_HOT, s, k_colcount<<<grid, 256, 0, s>>>(B, w.colcnt));
    }
    SPG_LAUNCH(p, K_HOT, s, k_hot_flags<<<grid, 256, 0, s>>>(w.colcnt, B.cols, p->opts.fp32_max_terms));
    launch_row_ptr(p, w.colcnt, B.cols, w, w.hot_rank, s);
    SPG_LAUNCH(p, K_HOT, s, k_hot_cols<<<grid, 256, 0, s>>>(w.colcnt, w.hot_rank, B.cols, w.hot_col));
    if (B.nnz > 0)
        SPG_LAUNCH(p, K_HOT, s, k_bhot<<<grid, 256, 0, s>>>(B, w.colcnt, w.hot_rank, w.bhot));
}

}  // namespace spg

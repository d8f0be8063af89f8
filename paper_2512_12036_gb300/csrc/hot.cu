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
//   bhot     for every stored entry of B its column's hot rank, or -1,
// so a kernel learns an entry's hotness with one coalesced load beside
// col/val.
#include "internal.h"

namespace spg {

__global__ void k_fill_i32(int* p, long long n, int v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_colcount(CsrDev B, int* cnt) {
    const long long J0 = B.rows > 0 ? B.rpt[0] : 0;
    const long long J1 = B.rows > 0 ? B.rpt[B.rows] : 0;
    if (J0 < 0 || J1 < J0 || J1 > B.nnz) return;
    for (long long j = J0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; j < J1;
         j += (long long)gridDim.x * blockDim.x) {
        const int c = B.col[j];
        if ((unsigned)c < (unsigned)B.cols) atomicAdd(&cnt[c], 1);
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

__global__ void k_bhot(CsrDev B, const int* flag, const int* rank, int* bhot) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < B.nnz;
         j += (long long)gridDim.x * blockDim.x) {
        const int c = B.col[j];
        bhot[j] = ((unsigned)c < (unsigned)B.cols && flag[c]) ? rank[c] : -1;
    }
}

void launch_hot(const spgemm_plan* p, const CsrDev& B, const WsPtrs& w, cudaStream_t s) {
    if (!w.colcnt || B.cols <= 0) return;
    const int grid = p->num_sms * 8;
    SPG_LAUNCH(p, K_HOT, s, k_fill_i32<<<grid, 256, 0, s>>>(w.colcnt, (long long)B.cols + 1, 0));
    if (B.nnz > 0) SPG_LAUNCH(p, K_HOT, s, k_colcount<<<grid, 256, 0, s>>>(B, w.colcnt));
    SPG_LAUNCH(p, K_HOT, s, k_hot_flags<<<grid, 256, 0, s>>>(w.colcnt, B.cols, p->opts.fp32_max_terms));
    launch_row_ptr(p, w.colcnt, B.cols, w, w.hot_rank, s);
    SPG_LAUNCH(p, K_HOT, s, k_hot_cols<<<grid, 256, 0, s>>>(w.colcnt, w.hot_rank, B.cols, w.hot_col));
    if (B.nnz > 0)
        SPG_LAUNCH(p, K_HOT, s, k_bhot<<<grid, 256, 0, s>>>(B, w.colcnt, w.hot_rank, w.bhot));
}

}  // namespace spg

// Matrix-based bulk neighbourhood sampling around the SpGEMM (the mini-batch
// GNN application of Section IV-C): per layer P = Q^l * A (the SpGEMM),
// NORM(P), Q^{l-1} = SAMPLE(P, s) by inverse transform sampling of s
// non-zeros per row, and EXTRACT(A, Q^l, Q^{l-1}) as a product with the
// selector of Q^{l-1}'s vertices.
//
// SAMPLE (k_sample_rows): one warp per row of P, one uniform u in [0, 1) per
// lane (s <= 32, supplied by the caller, so a run is reproducible). A row
// with at most s entries keeps all of them. Otherwise lane t draws entry
// F^{-1}(u_t) of the row's distribution:
//   mode 0: uniform over the row's entries, index floor(u * len) (exact);
//   mode 1: proportional to the values (negative values count as 0);
//   mode 2: proportional to the squared values (the layer-wise LADIES
//           importance weights);
// for modes 1-2 the cumulative weights are fp64 and the draw is the first
// entry whose inclusive prefix exceeds u * total (a row of zero weight
// falls back to mode 0). The s draws are sorted across the warp, repeats
// dropped, and the distinct columns written in ascending order, value 1.
//
// Column selection (k_select_flags, k_select_write): the distinct columns
// of Q^{l-1} become the next frontier. S (n x m) maps a selected vertex v
// to its rank r (S[v, r] = 1) and F (m x n) is its transpose (F[r, v] = 1):
// EXTRACT is (Q^l * A) * S, and F is Q for the next layer.
#include "internal.h"

namespace spg {

constexpr int kSampleThreads = 256;

// Ascending sort of one int per lane across the warp (bitonic network).
__device__ __forceinline__ int warp_sort_int(int v) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int o = __shfl_xor_sync(kFull, v, j);
            const bool up = (lane & k) == 0;
            const bool lower = (lane & j) == 0;
            v = (lower == up) ? min(v, o) : max(v, o);
        }
    }
    return v;
}

__device__ __forceinline__ double warp_incl_scan_f64(double v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

__device__ __forceinline__ double sample_weight(float v, int mode) {
    const double d = (double)v;
    if (mode == 2) return d * d;
    return d > 0.0 ? d : 0.0;
}

// kWrite = false: count[row] = distinct sampled columns; true: write them.
template <bool kWrite>
__global__ void __launch_bounds__(kSampleThreads) k_sample_rows(CsrDev P, int s, const float* u,
                                                                int mode, int* count,
                                                                const int* rpt_out, int* col_out,
                                                                float* val_out, Ctl* ctl) {
    const int lane = lane_id();
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    constexpr int kNone = 0x7fffffff;
    for (long long row = gw; row < P.rows; row += nw) {
        int rs, re;
        row_extent(P, (int)row, rs, re, ctl);
        const int len = re - rs;
        int c = kNone;
        if (len <= s) {
            if (lane < len) c = P.col[rs + lane];
        } else {
            const double ut = lane < s ? (double)u[row * (long long)s + lane] : 0.0;
            int pick = -1;
            double total = 0.0;
            if (mode != 0) {
                // the total through the same chunked scan the search uses below, so
                // u * total always falls inside the row's cumulative range
                for (int c0 = 0; c0 < len; c0 += 32) {
                    const double wq = c0 + lane < len ? sample_weight(P.val[rs + c0 + lane], mode) : 0.0;
                    total = __shfl_sync(kFull, total + warp_incl_scan_f64(wq), 31);
                }
            }
            if (mode == 0 || !(total > 0.0)) {
                int idx = (int)(ut * (double)len);
                pick = idx < len ? idx : len - 1;
            } else {
                const double target = ut * total;
                double base = 0.0;
                for (int c0 = 0; c0 < len; c0 += 32) {      // warp-uniform trip count
                    const int q = rs + c0 + lane;
                    const double wq = c0 + lane < len ? sample_weight(P.val[q], mode) : 0.0;
                    const double incl = base + warp_incl_scan_f64(wq);
                    const double chunk_end = __shfl_sync(kFull, incl, 31);
                    // lanes of this chunk whose inclusive prefix is <= target
                    int pos = 0;
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const double v = __shfl_sync(kFull, incl, pos + step - 1);
                        if (v <= target) pos += step;
                    }
                    if (pick < 0 && target < chunk_end && c0 + pos < len) pick = c0 + pos;
                    base = chunk_end;
                }
                if (pick < 0) pick = len - 1;               // unreachable: target < total
            }
            if (lane < s) c = P.col[rs + pick];
        }
        if ((unsigned)c >= (unsigned)P.cols && c != kNone) {
            set_status(ctl, ST_INVALID);
            c = kNone;
        }
        c = warp_sort_int(c);
        const int prev = __shfl_up_sync(kFull, c, 1);
        const bool keep = c != kNone && (lane == 0 || prev != c);
        const unsigned kb = __ballot_sync(kFull, keep);
        if (!kWrite) {
            if (lane == 0) count[row] = __popc(kb);
        } else {
            const int o = rpt_out[row] + __popc(kb & lanemask_lt());
            if (keep && o < rpt_out[row + 1]) {
                col_out[o] = c;
                val_out[o] = 1.f;
            }
        }
    }
}

__global__ void k_select_flags(CsrDev Q, int* flag, Ctl* ctl) {
    const long long J0 = Q.rows > 0 ? Q.rpt[0] : 0;
    const long long J1 = Q.rows > 0 ? Q.rpt[Q.rows] : 0;
    if (J0 < 0 || J1 < J0 || J1 > Q.nnz) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(ctl, ST_INVALID);
        return;
    }
    for (long long j = J0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; j < J1;
         j += (long long)gridDim.x * blockDim.x) {
        const int c = Q.col[j];
        if ((unsigned)c < (unsigned)Q.cols) flag[c] = 1;       // benign races: all write 1
        else set_status(ctl, ST_INVALID);
    }
}

// rank = exclusive scan of the flags: S row v holds (rank[v], 1) when flagged,
// F row r holds (v, 1) for the r-th selected vertex.
__global__ void k_select_write(const int* flag, const int* rank, int n, int* S_col, float* S_val,
                               int* F_rpt, int* F_col, float* F_val) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        if (flag[v]) {
            const int r = rank[v];
            S_col[r] = r;
            S_val[r] = 1.f;
            F_rpt[r] = r;
            F_col[r] = (int)v;
            F_val[r] = 1.f;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) F_rpt[rank[n]] = rank[n];
}

void launch_sample_rows(const spgemm_plan* p, const CsrDev& P, int s, const float* u, int mode,
                        const WsPtrs& w, int* rpt_out, int* col_out, float* val_out,
                        cudaStream_t st) {
    if (P.rows == 0) {
        launch_row_ptr(p, w.map, 0, w, rpt_out, st);
        return;
    }
    long long blocks = ((long long)P.rows * 32 + kSampleThreads - 1) / kSampleThreads;
    if (blocks > (long long)p->num_sms * 16) blocks = (long long)p->num_sms * 16;
    int* counts = w.map;
    SPG_LAUNCH(p, K_LAYER, st,
               k_sample_rows<false><<<(int)blocks, kSampleThreads, 0, st>>>(
                   P, s, u, mode, counts, nullptr, nullptr, nullptr, w.ctl));
    launch_row_ptr(p, counts, P.rows, w, rpt_out, st);
    SPG_LAUNCH(p, K_LAYER, st,
               k_sample_rows<true><<<(int)blocks, kSampleThreads, 0, st>>>(
                   P, s, u, mode, counts, rpt_out, col_out, val_out, w.ctl));
}

void launch_select_columns(const spgemm_plan* p, const CsrDev& Q, const WsPtrs& w, int* S_rpt,
                           int* S_col, float* S_val, int* F_rpt, int* F_col, float* F_val,
                           cudaStream_t st) {
    const int n = Q.cols;
    const int grid = p->num_sms * 8;
    int* flag = w.map;
    SPG_LAUNCH(p, K_LAYER, st, k_fill_i32<<<grid, 256, 0, st>>>(flag, (long long)n, 0));
    if (Q.nnz > 0) SPG_LAUNCH(p, K_LAYER, st, k_select_flags<<<grid, 256, 0, st>>>(Q, flag, w.ctl));
    launch_row_ptr(p, flag, n, w, S_rpt, st);
    SPG_LAUNCH(p, K_LAYER, st,
               k_select_write<<<grid, 256, 0, st>>>(flag, S_rpt, n, S_col, S_val, F_rpt, F_col,
                                                    F_val));
}

}  // namespace spg

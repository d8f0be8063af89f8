// Kernels around the SpGEMM for a GNN layer with a pruning (top-k) layer
// (Section IV-C, Eqs. 1-3): X_l = A * TopK(X_{l-1}, k) * W_l.
//
//   TopK (Eq. 2): the k largest values of each row of a dense matrix, as a
//     CSR matrix with exactly min(k, d) entries per row in column order (the
//     mask M_k and the kept values). Order: fp32 values compared through an
//     order-preserving 32-bit key (IEEE total order: -NaN < -inf < ... <
//     +inf < +NaN); equal keys go to the smaller column. The k-th largest
//     key is found by a radix selection (one warp per row: four 8-bit digits
//     on a 256-bin histogram) or a bitwise binary search with block counts
//     (rows longer than a warp holds), so no sort is needed.
//   scatter: a CSR matrix added into a dense matrix (M_k (.) G of Eq. 3 when
//     the values are a gradient on the mask's pattern).
//   gather: a dense matrix read at a CSR pattern (the gradient of A*TopK(X)
//     needed only where that product has entries).
#include "internal.h"

namespace spg {

constexpr int kTopkWarpMax = 1024;   // row length handled by one warp (32 values per lane)
constexpr int kTopkThreads = 256;
constexpr int kTopkBlockThreads = 1024;

__device__ __forceinline__ unsigned topk_key(float x) {
    const unsigned b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// One warp per row (d <= kTopkWarpMax).
// kPer: 32-column groups a lane holds (rows of up to 32 * kPer columns).
template <int kPer>
__global__ void __launch_bounds__(kTopkThreads) k_topk_warp(const float* X, int n, int d,
                                                            long long ldx, int k, int* rpt,
                                                            int* col, float* val) {
    __shared__ int whist[kTopkThreads / 32][256];
    int* hist = whist[threadIdx.x >> 5];
    const int lane = lane_id();
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int kk = k < 0 ? 0 : (k < d ? k : d);
    for (long long row = gw; row < n; row += nw) {
        const float* x = X + row * ldx;
        unsigned key[kPer];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int c = lane + 32 * i;
            key[i] = c < d ? topk_key(x[c]) : 0u;   // columns past d are never counted
        }
        // (the loops below stop at the row's last 32-column group: d is
        // uniform, so the unrolled groups past it are skipped by the warp)
        // K = the kk-th largest key (the largest K with #(keys >= K) >= kk),
        // by radix selection: 8 bits a pass from the top, a per-warp 256-bin
        // histogram of the keys sharing the prefix found so far
        unsigned K = 0u;
        int need_eq = kk;
        if (kk == 0) {
            K = 0xffffffffu;                         // nothing kept
            need_eq = 0;
        } else if (kk < d) {
            unsigned prefix = 0u, pmask = 0u;
            int above = 0;
            for (int sh = 24; sh >= 0; sh -= 8) {
#pragma unroll
                for (int b = 0; b < 8; ++b) hist[8 * lane + b] = 0;
                __syncwarp();
#pragma unroll
                for (int i = 0; i < kPer; ++i) {
                    if (32 * i >= d) break;                         // warp-uniform
                    if (lane + 32 * i < d && (key[i] & pmask) == prefix)
                        atomicAdd(&hist[(key[i] >> sh) & 255u], 1);
                }
                __syncwarp();
                int dig, run_at;
                radix_digit256(hist, above, kk, dig, run_at);
                prefix |= (unsigned)dig << sh;
                pmask |= 255u << sh;
                above = run_at;
                __syncwarp();
            }
            K = prefix;
            need_eq = kk - above;
        }
        // write kept entries in column order (column 32*i + lane)
        const long long base = row * (long long)kk;
        int pos = 0, eq_seen = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            if (32 * i >= d) break;                                 // warp-uniform
            const int c = lane + 32 * i;
            bool keep;
            if (kk == d) {
                keep = c < d;
            } else {
                const bool eq = c < d && key[i] == K;
                const unsigned eqb = __ballot_sync(kFull, eq);
                const int rank = eq_seen + __popc(eqb & lanemask_lt());
                eq_seen += __popc(eqb);
                keep = c < d && (key[i] > K || (eq && rank < need_eq));
            }
            const unsigned kb = __ballot_sync(kFull, keep);
            if (keep) {
                const int o = pos + __popc(kb & lanemask_lt());
                if (o < kk) {
                    col[base + o] = c;
                    val[base + o] = x[c];
                }
            }
            pos += __popc(kb);
        }
        if (lane == 0) rpt[row] = (int)base;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rpt[n] = (int)((long long)n * kk);
}

// One block per row (d > kTopkWarpMax), rows taken by stride.
__global__ void __launch_bounds__(kTopkBlockThreads) k_topk_block(const float* X, int n, int d,
                                                                  long long ldx, int k, int* rpt,
                                                                  int* col, float* val) {
    __shared__ int red[33];
    __shared__ int scratch[33];
    const int kk = k < 0 ? 0 : (k < d ? k : d);
    for (long long row = blockIdx.x; row < n; row += gridDim.x) {
        const float* x = X + row * ldx;
        unsigned K = 0u;
        int need_eq = kk;
        if (kk < d) {
            unsigned lo = 0u, hi = 0xffffffffu;
            while (lo < hi) {
                const unsigned mid = lo + (unsigned)(((unsigned long long)hi - lo + 1ull) >> 1);
                int c = 0;
                for (int q = threadIdx.x; q < d; q += blockDim.x) c += topk_key(x[q]) >= mid;
                if (block_sum(c, red) >= kk) lo = mid;
                else hi = mid - 1u;
            }
            K = lo;
            int gt = 0;
            for (int q = threadIdx.x; q < d; q += blockDim.x) gt += topk_key(x[q]) > K;
            need_eq = kk - block_sum(gt, red);
        }
        const long long base = row * (long long)kk;
        int pos = 0, eq_seen = 0;
        for (int c0 = 0; c0 < d; c0 += blockDim.x) {
            const int c = c0 + threadIdx.x;
            const unsigned kc = c < d ? topk_key(x[c]) : 0u;
            int eq_tot;
            const int eq_rank =
                eq_seen + block_excl_scan((kk < d && c < d && kc == K) ? 1 : 0, scratch, &eq_tot);
            eq_seen += eq_tot;
            const bool keep = c < d && (kk == d || kc > K || (kc == K && eq_rank < need_eq));
            int ktot;
            const int o = pos + block_excl_scan(keep ? 1 : 0, scratch, &ktot);
            if (keep && o < kk) {
                col[base + o] = c;
                val[base + o] = x[c];
            }
            pos += ktot;
        }
        if (threadIdx.x == 0) rpt[row] = (int)base;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) rpt[n] = (int)((long long)n * kk);
}

// X[i, j] += v for every entry (i, j, v) of M; one warp per row.
__global__ void k_scatter_dense(CsrDev M, const float* vals, float* X, long long ldx, Ctl* ctl) {
    const int lane = lane_id();
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = gw; row < M.rows; row += nw) {
        int s, e;
        if (!row_extent(M, (int)row, s, e, ctl)) continue;
        for (int q = s + lane; q < e; q += 32) {
            const int c = M.col[q];
            if ((unsigned)c < (unsigned)M.cols) atomicAdd(&X[row * ldx + c], vals[q]);
            else set_status(ctl, ST_INVALID);
        }
    }
}

// out[q] = D[i, j] for every entry q = (i, j) of M; one warp per row.
__global__ void k_gather_dense(CsrDev M, const float* D, long long ldd, float* out, Ctl* ctl) {
    const int lane = lane_id();
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = gw; row < M.rows; row += nw) {
        int s, e;
        if (!row_extent(M, (int)row, s, e, ctl)) continue;
        for (int q = s + lane; q < e; q += 32) {
            const int c = M.col[q];
            if ((unsigned)c < (unsigned)M.cols) {
                out[q] = D[row * ldd + c];
            } else {
                out[q] = 0.f;
                set_status(ctl, ST_INVALID);
            }
        }
    }
}

void launch_topk(const spgemm_plan* p, const float* X, int n, int d, long long ldx, int k,
                 int* rpt, int* col, float* val, cudaStream_t s) {
    const int sms = p->num_sms;
    if (n == 0 || d <= kTopkWarpMax) {
        long long blocks = ((long long)n * 32 + kTopkThreads - 1) / kTopkThreads;
        if (blocks > (long long)sms * 16) blocks = (long long)sms * 16;
        if (blocks < 1) blocks = 1;
        SPG_LAUNCH(p, K_LAYER, s,
                   (d <= 256 ? k_topk_warp<8> : k_topk_warp<kTopkWarpMax / 32>)<<<(int)blocks, kTopkThreads, 0, s>>>(
                       X, n, d, ldx, k, rpt, col, val));
    } else {
        const int blocks = n < sms * 2 ? (n > 0 ? n : 1) : sms * 2;
        SPG_LAUNCH(p, K_LAYER, s,
                   k_topk_block<<<blocks, kTopkBlockThreads, 0, s>>>(X, n, d, ldx, k, rpt, col, val));
    }
}

void launch_scatter_dense(const spgemm_plan* p, const CsrDev& M, const float* vals, float* X,
                          long long ldx, Ctl* ctl, cudaStream_t s) {
    if (M.rows == 0) return;
    long long blocks = ((long long)M.rows * 32 + 255) / 256;
    if (blocks > (long long)p->num_sms * 16) blocks = (long long)p->num_sms * 16;
    SPG_LAUNCH(p, K_LAYER, s, k_scatter_dense<<<(int)blocks, 256, 0, s>>>(M, vals, X, ldx, ctl));
}

void launch_gather_dense(const spgemm_plan* p, const CsrDev& M, const float* D, long long ldd,
                         float* out, Ctl* ctl, cudaStream_t s) {
    if (M.rows == 0) return;
    long long blocks = ((long long)M.rows * 32 + 255) / 256;
    if (blocks > (long long)p->num_sms * 16) blocks = (long long)p->num_sms * 16;
    SPG_LAUNCH(p, K_LAYER, s, k_gather_dense<<<(int)blocks, 256, 0, s>>>(M, D, ldd, out, ctl));
}

}  // namespace spg

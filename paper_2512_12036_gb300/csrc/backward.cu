// Backward of C = A*B with respect to the stored values of A and B (the
// gradient rule of the pruned-GNN layer, Eq. 3, read at the value level):
//   dA[j] = sum_{t in B_k} dC(i, colB[t]) * valB[t]        for A entry j = (i, k)
//   dB[t] = sum_{j = (i,k) in A} valA[j] * dC(i, colB[t])  for B entry t in row k
// C's structure (sorted rows, as the forward produced it) holds every (i, c)
// a product reaches, so dC(i, c) is looked up in row i of C.
//
// Schedule: rows of A (= rows of C) are grouped by nnz(C_i); a row's dC
// values are staged in shared memory (a dense array when B has few columns,
// an open-addressing table otherwise, or dense column panels for very long
// rows); then one warp per A entry walks the entry's B row with its lanes,
// reduces dA[j] in fp64 registers and writes it once, and adds each dB
// contribution with an fp64 global atomic (converted to fp32 at the end).
#include "internal.h"

namespace spg {

constexpr int kBwdWarps = 8;                 // warps per block in the warp-per-row tiers
constexpr int kBwdBlockThreads = 1024;
constexpr int kBwdPanel = 32768;             // dense-panel width of the heavy tier

struct BwdArgs {
    CsrDev A, B;
    const int* rptC;
    const int* colC;
    const float* dC;
    float* dA;            // nullable
    double* dB64;         // nullable (fp64 accumulation of dB)
    Ctl* ctl;
    const int* map;
    const int* tab;       // panel table (panel_cols wide panels), or null
    int P, PW;
};

__global__ void k_bwd_zero(double* p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

__global__ void k_bwd_convert(const double* src, float* dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

// A warp handles A entries [j0, j0 + cnt) of one row (cnt <= 32): lane l
// first gathers entry j0 + l's B segment (seg(j, ts, te)) and value, so the
// 32 entries' index loads are in flight together; then the entries are
// walked four at a time (independent loads and reductions overlap), each
// entry's products spread over the lanes; lane l returns entry j0 + l's dA
// (the caller writes them, coalesced). dB contributions go out as fp64
// atomics on the way.
//
// Precision without fp64 arithmetic on the SM (GB300's fp64 pipe is slow):
// a segment of L products is summed as 32 per-lane fp32 partial sums of at
// most ceil(L/32) products and a 5-level fp32 tree, so every product meets
// at most ceil(L/32) + 6 roundings (its own product included): the error
// stays within gamma_(ceil(L/32)+6) * sum|g b| <= 1e-5 * sum|g b| for L up to
// kBwdF32Len; longer segments are summed in fp64. A dB term a*g is rounded
// once to fp32 (relative error 2^-24) and added in fp64.
constexpr int kBwdF32Len = 32 * 160;

template <class Seg, class Look>
__device__ __forceinline__ double bwd_chunk(const BwdArgs& x, int j0, int cnt, Seg&& seg,
                                            Look&& look) {
    const int lane = lane_id();
    int ts = 0, te = 0;
    float a = 0.f;
    if (lane < cnt) {
        seg(j0 + lane, ts, te);
        a = x.A.val[j0 + lane];
    }
    auto lookup = [&](int t, float& g) {
        const int c = x.B.col[t];
        g = 0.f;
        if ((unsigned)c < (unsigned)x.B.cols) {
            if (!look(c, g)) set_status(x.ctl, ST_INVALID);   // C lacks a product's column
        } else {
            set_status(x.ctl, ST_INVALID);
        }
    };
    double mine = 0.0;
    for (int q = 0; q < cnt; q += 4) {
        float acc[4];
        double wide[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int qq = q + u;
            const int sts = __shfl_sync(kFull, ts, qq & 31);
            const int ste = qq < cnt ? __shfl_sync(kFull, te, qq & 31) : sts;
            const float sa = __shfl_sync(kFull, a, qq & 31);
            acc[u] = 0.f;
            wide[u] = 0.0;
            if (ste - sts <= kBwdF32Len) {                      // warp-uniform
                for (int t = sts + lane; t < ste; t += 32) {
                    float g;
                    lookup(t, g);
                    acc[u] = fmaf(g, x.B.val[t], acc[u]);
                    if (x.dB64) atomicAdd(&x.dB64[t], (double)(sa * g));
                }
            } else {
                for (int t = sts + lane; t < ste; t += 32) {
                    float g;
                    lookup(t, g);
                    wide[u] += (double)g * (double)x.B.val[t];
                    if (x.dB64) atomicAdd(&x.dB64[t], (double)(sa * g));
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += __shfl_xor_sync(kFull, acc[u], o);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int qq = q + u;
            const bool is_wide = qq < cnt &&
                                 __shfl_sync(kFull, te, qq & 31) - __shfl_sync(kFull, ts, qq & 31) >
                                     kBwdF32Len;
            double v = acc[u];
            if (is_wide) v = warp_sum(wide[u]);                  // warp-uniform
            if (lane == qq) mine = v;
        }
    }
    return mine;
}

// ---------------------------------------------------------------------------
// Tier BW_DENSE: B has <= kBwdDenseCols columns; dC row i scattered into a
// per-warp dense array (untouched columns read 0, which only happens for
// columns no product reaches).
__global__ void __launch_bounds__(kBwdWarps * 32) k_bwd_dense(BwdArgs x, int bin) {
    extern __shared__ float sm_dense[];
    const int begin = x.ctl->bin_off[bin], end = x.ctl->bin_off[bin + 1];
    const int lane = lane_id();
    float* dense = sm_dense + (threadIdx.x >> 5) * x.B.cols;
    for (int c = lane; c < x.B.cols; c += 32) dense[c] = 0.f;
    __syncwarp();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int idx = begin + gw; idx < end; idx += nw) {
        const int i = x.map[idx];
        const int cs = x.rptC[i], ce = x.rptC[i + 1];
        for (int q = cs + lane; q < ce; q += 32) {
            const int c = x.colC[q];
            if ((unsigned)c < (unsigned)x.B.cols) dense[c] = x.dC[q];
        }
        __syncwarp();
        int rs, re;
        row_extent(x.A, i, rs, re, x.ctl);
        for (int j0 = rs; j0 < re; j0 += 32) {
            const double d = bwd_chunk(
                x, j0, re - j0 < 32 ? re - j0 : 32,
                [&](int j, int& ts, int& te) {
                    int bs, len;
                    a_entry(x.A, x.B, j, bs, len, x.ctl);
                    ts = bs;
                    te = bs + len;
                },
                [&](int c, float& g) {
                    g = dense[c];
                    return true;
                });
            if (x.dA && j0 + lane < re) x.dA[j0 + lane] = (float)d;
        }
        __syncwarp();
        for (int q = cs + lane; q < ce; q += 32) {
            const int c = x.colC[q];
            if ((unsigned)c < (unsigned)x.B.cols) dense[c] = 0.f;
        }
        __syncwarp();
    }
}

// Open-addressing (column -> dC) table; C's columns in a row are distinct.
__device__ __forceinline__ void bwd_insert(int* keys, float* vals, int bits, int key, float v) {
    const unsigned mask = (1u << bits) - 1u;
    unsigned h = hash_slot(key, bits);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int old = atomicCAS(&keys[h], kEmpty, key);
        if (old == kEmpty || old == key) {
            vals[h] = v;
            return;
        }
        h = (h + 1u) & mask;
    }
}

__device__ __forceinline__ bool bwd_lookup(const int* keys, const float* vals, int bits, int key,
                                           float& v) {
    const unsigned mask = (1u << bits) - 1u;
    unsigned h = hash_slot(key, bits);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int k = keys[h];
        if (k == key) {
            v = vals[h];
            return true;
        }
        if (k == kEmpty) break;
        h = (h + 1u) & mask;
    }
    v = 0.f;
    return false;
}

// Tier BW_WARP: warp per row, per-warp table of kBwdWarpSlots.
__global__ void __launch_bounds__(kBwdWarps * 32) k_bwd_warp(BwdArgs x, int bin) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    int* keys = reinterpret_cast<int*>(sm_raw) + warp * kBwdWarpSlots;
    float* vals = reinterpret_cast<float*>(sm_raw + sizeof(int) * kBwdWarps * kBwdWarpSlots) +
                  warp * kBwdWarpSlots;
    const int begin = x.ctl->bin_off[bin], end = x.ctl->bin_off[bin + 1];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int idx = begin + gw; idx < end; idx += nw) {
        const int i = x.map[idx];
        const int cs = x.rptC[i], ce = x.rptC[i + 1];
        int bits = 5;
        while (bits < 10 && (1 << bits) < 2 * (ce - cs)) ++bits;
        for (int s = lane; s < (1 << bits); s += 32) keys[s] = kEmpty;
        __syncwarp();
        for (int q = cs + lane; q < ce; q += 32) bwd_insert(keys, vals, bits, x.colC[q], x.dC[q]);
        __syncwarp();
        int rs, re;
        row_extent(x.A, i, rs, re, x.ctl);
        for (int j0 = rs; j0 < re; j0 += 32) {
            const double d = bwd_chunk(
                x, j0, re - j0 < 32 ? re - j0 : 32,
                [&](int j, int& ts, int& te) {
                    int bs, len;
                    a_entry(x.A, x.B, j, bs, len, x.ctl);
                    ts = bs;
                    te = bs + len;
                },
                [&](int c, float& g) { return bwd_lookup(keys, vals, bits, c, g); });
            if (x.dA && j0 + lane < re) x.dA[j0 + lane] = (float)d;
        }
        __syncwarp();
    }
}

// Tier BW_BLOCK: block per row, table of kBwdBlockSlots; warps take the
// row's A entries round-robin.
__global__ void __launch_bounds__(kBwdBlockThreads) k_bwd_block(BwdArgs x, int bin, int tier) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    int* keys = reinterpret_cast<int*>(sm_raw);
    float* vals = reinterpret_cast<float*>(sm_raw + sizeof(int) * kBwdBlockSlots);
    __shared__ int s_idx;
    const int begin = x.ctl->bin_off[bin], end = x.ctl->bin_off[bin + 1];
    const int warp = threadIdx.x >> 5, lane = lane_id(), nwarps = blockDim.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_idx = begin + atomicAdd(&x.ctl->work[tier], 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= end) break;
        const int i = x.map[idx];
        const int cs = x.rptC[i], ce = x.rptC[i + 1];
        int bits = 6;
        while (bits < 14 && (1 << bits) < 2 * (ce - cs)) ++bits;
        for (int s = threadIdx.x; s < (1 << bits); s += blockDim.x) keys[s] = kEmpty;
        __syncthreads();
        for (int q = cs + threadIdx.x; q < ce; q += blockDim.x)
            bwd_insert(keys, vals, bits, x.colC[q], x.dC[q]);
        __syncthreads();
        int rs, re;
        row_extent(x.A, i, rs, re, x.ctl);
        for (int j0 = rs + 32 * warp; j0 < re; j0 += 32 * nwarps) {
            const double d = bwd_chunk(
                x, j0, re - j0 < 32 ? re - j0 : 32,
                [&](int j, int& ts, int& te) {
                    int bs, len;
                    a_entry(x.A, x.B, j, bs, len, x.ctl);
                    ts = bs;
                    te = bs + len;
                },
                [&](int c, float& g) { return bwd_lookup(keys, vals, bits, c, g); });
            if (x.dA && j0 + lane < re) x.dA[j0 + lane] = (float)d;
        }
        __syncthreads();
    }
}

// Tier BW_PANEL: block per row with more than 8192 entries in C: dC row i
// staged one column panel (kBwdPanel columns) at a time as a dense array;
// the B segment of each A entry inside the panel comes from the panel table
// (or a filtered walk of the whole B row when B is not sorted); dA partial
// sums of every panel are added in fp64 and written after the last panel.
__global__ void __launch_bounds__(kBwdBlockThreads) k_bwd_panel(BwdArgs x, int bin, int tier,
                                                                double* dA64) {
    extern __shared__ float dense[];
    __shared__ int s_idx;
    const int begin = x.ctl->bin_off[bin], end = x.ctl->bin_off[bin + 1];
    if (begin >= end) return;
    const int warp = threadIdx.x >> 5, lane = lane_id(), nwarps = blockDim.x >> 5;
    for (int c = threadIdx.x; c < kBwdPanel; c += blockDim.x) dense[c] = 0.f;
    const bool use_tab = x.tab != nullptr && (x.ctl->b_unsorted & 1) == 0;
    const int per = kBwdPanel / x.PW;                    // table panels per pass
    const int npass = (int)((x.B.cols + (long long)kBwdPanel - 1) / kBwdPanel);
    for (;;) {
        if (threadIdx.x == 0) s_idx = begin + atomicAdd(&x.ctl->work[tier], 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= end) break;
        const int i = x.map[idx];
        const int cs = x.rptC[i], ce = x.rptC[i + 1];
        int rs, re;
        row_extent(x.A, i, rs, re, x.ctl);
        for (int j = rs + threadIdx.x; j < re; j += blockDim.x) dA64[j] = 0.0;
        __syncthreads();
        int q0 = cs;                                      // first C entry of the pass
        for (int pass = 0; pass < npass; ++pass) {
            const int c0 = pass * kBwdPanel;
            const int c1 = c0 + kBwdPanel;
            // C row entries with columns in [c0, c1): contiguous (sorted row)
            int lo = q0, hi = ce;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (x.colC[mid] < c1) lo = mid + 1;
                else hi = mid;
            }
            const int q1 = lo;
            for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
                const int c = x.colC[q] - c0;
                if (c >= 0 && c < kBwdPanel) dense[c] = x.dC[q];
            }
            __syncthreads();
            const int p0 = pass * per;
            const int p1 = p0 + per < x.P ? p0 + per : x.P;
            for (int j0 = rs + 32 * warp; j0 < re; j0 += 32 * nwarps) {
                const double d = bwd_chunk(
                    x, j0, re - j0 < 32 ? re - j0 : 32,
                    [&](int j, int& ts, int& te) {
                        int bs, len;
                        a_entry(x.A, x.B, j, bs, len, x.ctl);
                        ts = bs;
                        te = bs + len;
                        if (use_tab && len > 0) {
                            const int* tk = x.tab + (long long)x.A.col[j] * (x.P + 1);
                            ts = tk[p0];
                            te = tk[p1];
                            if (ts < bs || te < ts || te > bs + len) {
                                set_status(x.ctl, ST_INTERNAL);
                                ts = te = bs;
                            }
                        }
                    },
                    [&](int c, float& g) {
                        const int cc = c - c0;
                        if (cc < 0 || cc >= kBwdPanel) {
                            g = 0.f;       // outside this pass (filtered walk of an unsorted row)
                            return true;
                        }
                        g = dense[cc];
                        return true;
                    });
                // one warp owns entries [j0, j0 + 32)
                if (j0 + lane < re && d != 0.0) dA64[j0 + lane] += d;
            }
            __syncthreads();
            for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
                const int c = x.colC[q] - c0;
                if (c >= 0 && c < kBwdPanel) dense[c] = 0.f;
            }
            q0 = q1;
            __syncthreads();
        }
        if (x.dA)
            for (int j = rs + threadIdx.x; j < re; j += blockDim.x) x.dA[j] = (float)dA64[j];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------

void occupancy_backward(spgemm_plan* p) {
    allow_max_dynamic_smem((const void*)k_bwd_dense, p);
    allow_max_dynamic_smem((const void*)k_bwd_warp, p);
    allow_max_dynamic_smem((const void*)k_bwd_block, p);
    allow_max_dynamic_smem((const void*)k_bwd_panel, p);
}

size_t backward_extra_bytes(long long a_nnz, long long b_nnz) {
    // dB in fp64 and the dA panel partials in fp64
    return sizeof(double) * (size_t)(b_nnz > 0 ? b_nnz : 1) +
           sizeof(double) * (size_t)(a_nnz > 0 ? a_nnz : 1) + 512;
}

void launch_bpanel(const spgemm_plan* p, const CsrDev& B, const WsPtrs& w, cudaStream_t s);

void launch_backward(const spgemm_plan* p, const CsrDev& A, const CsrDev& B, const int* rptC,
                     const int* colC, const float* dC, float* dA, float* dB, const WsPtrs& w,
                     double* dB64, double* dA64, cudaStream_t s) {
    const int m = A.rows;
    const int sms = p->num_sms;
    BwdArgs x{A, B, rptC, colC, dC, dA, dB ? dB64 : nullptr, w.ctl, w.map, nullptr, w.panels,
              w.panel_cols};
    if (dB && B.nnz > 0)
        SPG_LAUNCH(p, K_BWD, s, k_bwd_zero<<<sms * 4, 256, 0, s>>>(dB64, B.nnz));
    // rows whose C row is empty are never visited: their A entries have no
    // product, so their gradient is 0
    if (dA && A.nnz > 0) cudaMemsetAsync(dA, 0, sizeof(float) * (size_t)A.nnz, s);
    // the heavy tier needs B's panel table (built into this workspace)
    launch_bpanel(p, B, w, s);
    x.tab = w.bpanel;
    GroupArgs g{};
    g.phase = 3;
    g.n = m;
    g.rptC = rptC;
    g.bcols = B.cols;
    g.opts = p->opts;
    launch_group(p, g, w, w.map, nullptr, s);
    if (m > 0) {
        // warp-per-row tiers are latency-bound: as many resident blocks as
        // their shared memory allows
        auto resident = [&](const void* f, size_t smem) {
            int occ = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kBwdWarps * 32, smem);
            return sms * (occ > 0 ? occ : 1);
        };
        if (B.cols <= kBwdDenseCols) {
            const size_t sd = (size_t)kBwdWarps * B.cols * 4;
            SPG_LAUNCH(p, K_BWD, s,
                       k_bwd_dense<<<resident((const void*)k_bwd_dense, sd), kBwdWarps * 32, sd, s>>>(
                           x, BW_DENSE));
        }
        const size_t sw = (size_t)kBwdWarps * kBwdWarpSlots * 8;
        SPG_LAUNCH(p, K_BWD, s,
                   k_bwd_warp<<<resident((const void*)k_bwd_warp, sw), kBwdWarps * 32, sw, s>>>(
                       x, BW_WARP));
        SPG_LAUNCH(p, K_BWD, s,
                   k_bwd_block<<<sms, kBwdBlockThreads, kBwdBlockSlots * 8, s>>>(x, BW_BLOCK, 6));
        SPG_LAUNCH(p, K_BWD, s,
                   k_bwd_panel<<<sms, kBwdBlockThreads, kBwdPanel * 4, s>>>(x, BW_PANEL, 7, dA64));
    }
    if (dB && B.nnz > 0)
        SPG_LAUNCH(p, K_BWD, s, k_bwd_convert<<<sms * 4, 256, 0, s>>>(dB64, dB, B.nnz));
}

}  // namespace spg

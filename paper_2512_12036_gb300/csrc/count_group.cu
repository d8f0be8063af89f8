// Intermediate-product counting (Algorithm 1), row grouping (Section III-B)
// and the row-pointer scan of the allocation phase.
#include "internal.h"

namespace spg {

// ---------------------------------------------------------------------------
// Small utilities
// ---------------------------------------------------------------------------

__global__ void k_fill_i64(long long* p, long long n, long long v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

void launch_fill_i64(const spgemm_plan* pl, long long* p, long long n, long long v, cudaStream_t s) {
    if (n <= 0) return;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    SPG_LAUNCH(pl, K_FILL, s, k_fill_i64<<<(int)blocks, 256, 0, s>>>(p, n, v));
}

template <typename T>
__global__ void k_sum_to(const T* x, long long n, long long* out) {
    __shared__ long long red[33];
    long long acc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        acc += (long long)x[i];
    acc = block_sum(acc, red);
    if (threadIdx.x == 0 && acc != 0) atomicAdd((unsigned long long*)out, (unsigned long long)acc);
}

__global__ void k_zero_total(Ctl* ctl, int which) { ctl->totals[which] = 0; }

// Row pointers must be monotone and inside [0, nnz].
__global__ void k_check_rpt(CsrDev M, Ctl* ctl) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M.rows;
         i += (long long)gridDim.x * blockDim.x) {
        const int s = M.rpt[i], e = M.rpt[i + 1];
        if (s < 0 || e < s || (long long)e > M.nnz) set_status(ctl, ST_INVALID);
    }
}

// ---------------------------------------------------------------------------
// Algorithm 1, balanced over nonzeros: each block takes a tile of A's stored
// entries, so a row of 60k entries costs the same as 60k rows of one entry.
// The owning row of an entry is found by binary search over the block's row
// range; per-warp segmented sums then add into ip[row] with one atomic per
// (warp, row) segment.
// ---------------------------------------------------------------------------

constexpr int kCountThreads = 256;
constexpr int kCountItems = 8;
constexpr int kCountTile = kCountThreads * kCountItems;

__device__ __forceinline__ int row_of(const int* rpt, long long j, int lo, int hi) {
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)rpt[mid] <= j) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kCountThreads) k_ip_count(CsrDev A, CsrDev B, long long* ip,
                                                            Ctl* ctl) {
    __shared__ int s_r0, s_r1;
    const int m = A.rows;
    const long long J0 = A.rpt[0], J1 = A.rpt[m];
    if (J0 < 0 || J1 < J0 || J1 > A.nnz) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(ctl, ST_INVALID);
        return;
    }
    const long long jb = J0 + (long long)blockIdx.x * kCountTile;
    if (jb >= J1) return;
    const long long je = jb + kCountTile < J1 ? jb + kCountTile : J1;
    if (threadIdx.x == 0) {
        const int r0 = row_of(A.rpt, jb, 0, m - 1);
        s_r0 = r0;
        s_r1 = row_of(A.rpt, je - 1, r0, m - 1);
    }
    __syncthreads();
    const int r0 = s_r0, r1 = s_r1;
    const int lane = lane_id();
    for (int it = 0; it < kCountItems; ++it) {
        const long long j = jb + (long long)it * kCountThreads + threadIdx.x;
        int row = -1;
        long long v = 0;
        if (j < je) {
            row = row_of(A.rpt, j, r0, r1);
            int bs, len;
            a_entry(A, B, (int)j, bs, len, ctl);
            v = len;
        }
        // segmented inclusive scan over contiguous equal rows
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long n = __shfl_up_sync(kFull, v, o);
            const int rp = __shfl_up_sync(kFull, row, o);
            if (lane >= o && rp == row) v += n;
        }
        const int rn = __shfl_down_sync(kFull, row, 1);
        const bool last = (lane == 31) || rn != row;
        if (last && row >= 0 && v != 0) atomicAdd((unsigned long long*)&ip[row], (unsigned long long)v);
    }
}

void launch_ip_count(const spgemm_plan* p, const CsrDev& A, const CsrDev& B, long long* ip,
                     const WsPtrs& w, cudaStream_t s) {
    if (A.rows == 0) return;
    launch_fill_i64(p, ip, A.rows, 0, s);
    {
        const int blocks = (int)((A.rows + 255) / 256 < 4096 ? (A.rows + 255) / 256 : 4096);
        SPG_LAUNCH(p, K_CHECK_RPT, s, k_check_rpt<<<blocks, 256, 0, s>>>(A, w.ctl));
    }
    if (B.rows > 0) {
        const int blocks = (int)((B.rows + 255) / 256 < 4096 ? (B.rows + 255) / 256 : 4096);
        SPG_LAUNCH(p, K_CHECK_RPT, s, k_check_rpt<<<blocks, 256, 0, s>>>(B, w.ctl));
    }
    SPG_LAUNCH(p, K_ZERO, s, k_zero_total<<<1, 1, 0, s>>>(w.ctl, 0));
    if (A.nnz > 0) {
        const long long tiles = (A.nnz + kCountTile - 1) / kCountTile;
        SPG_LAUNCH(p, K_IP_COUNT, s, k_ip_count<<<(unsigned)tiles, kCountThreads, 0, s>>>(A, B, ip, w.ctl));
    }
    SPG_LAUNCH(p, K_SUM, s, k_sum_to<long long><<<256, 256, 0, s>>>(ip, A.rows, &w.ctl->totals[0]));
}

void launch_nnz_total(const spgemm_plan* p, const int* row_nnz, int n, const WsPtrs& w, cudaStream_t s) {
    SPG_LAUNCH(p, K_ZERO, s, k_zero_total<<<1, 1, 0, s>>>(w.ctl, 1));
    if (n > 0) SPG_LAUNCH(p, K_SUM, s, k_sum_to<int><<<256, 256, 0, s>>>(row_nnz, n, &w.ctl->totals[1]));
}

// ---------------------------------------------------------------------------
// Row grouping. Every row gets a bin id; the map is a stable partition of
// the rows by bin (ascending bin, ascending row inside a bin), built from
// per-block histograms, one exclusive scan over (bin, block) and a scatter
// that ranks rows inside a warp with __match_any_sync. One pass of atomics
// in shared memory per block replaces the per-row global atomics that the
// paper names as the grouping phase's cost.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

__device__ __forceinline__ int bin_of(const GroupArgs& g, int r, bool settle) {
    if (g.phase == 2) {
        const long long k = g.key[r];
        int b = 0;
        while (b < g.nthr && k >= g.thr[b]) ++b;
        return b;
    }
    if (g.phase == 3) {       // backward tiers, by nnz of row r of C
        const int nc = g.rptC[r + 1] - g.rptC[r];
        if (nc <= 0) return kSkipBin;
        if (g.bcols <= kBwdDenseCols) return BW_DENSE;
        if (nc <= kBwdWarpSlots / 2) return BW_WARP;
        if (nc <= kBwdBlockSlots / 2) return BW_BLOCK;
        return BW_PANEL;
    }
    const int row = g.row_begin + r;
    const long long ip = g.ip[row];
    const int na = g.rptA[row + 1] - g.rptA[row];
    const spgemm_opts& o = g.opts;
    if (g.phase == 0) {
        if (ip <= 1) {
            if (settle) g.row_nnz[row] = ip < 0 ? 0 : (int)ip;
            return kSkipBin;
        }
        if (ip <= o.esc_max && na <= o.esc_max) return SB_ESC;
        if (g.bcols <= kNarrowCols && ip <= narrow_max_ip(o)) return SB_NARROW;
        if (ip <= o.warp_max_ip) return SB_WARP;
        const int L = log2_ceil_ll(ip);
        if (ip <= o.block_max_ip) {
            const int Lmax = log2_ceil_ll(o.block_max_ip);
            return SB_BLOCK0 + clampi(Lmax - L, 0, SB_BLOCK_N - 1);
        }
        return SB_DENSE0 + clampi(46 - L, 0, SB_DENSE_N - 1);
    }
    const int nnz = g.rptC[r + 1] - g.rptC[r];
    if (nnz <= 0) return kSkipBin;
    const bool f64 = na > o.fp32_max_terms && ip > o.fp32_max_terms;
    if (ip <= o.esc_max && na <= o.esc_max) return NB_ESC;
    if (g.bcols <= kNarrowCols && ip <= narrow_max_ip(o)) return f64 ? NB_NARROW64 : NB_NARROW32;
    if (nnz <= o.warp_max_nnz && ip <= 16ll * o.warp_max_nnz) return f64 ? NB_WARP64 : NB_WARP32;
    if (nnz <= block_small_nnz(o)) return f64 ? NB_BLOCK64S : NB_BLOCK32S;
    if (nnz <= block_mid_nnz(o)) return f64 ? NB_BLOCK64M : NB_BLOCK32M;
    if (nnz <= o.block_max_nnz) return f64 ? NB_BLOCK64 : NB_BLOCK32;
    const int L = log2_ceil_ll(ip);
    return (f64 ? NB_DENSE64_0 : NB_DENSE32_0) + clampi(46 - L, 0, NB_DENSE_N - 1);
}

__global__ void __launch_bounds__(kBinRows) k_group_hist(GroupArgs g, int nblk, int* blk_counts) {
    __shared__ int hist[kNumBins];
    if (threadIdx.x < kNumBins) hist[threadIdx.x] = 0;
    __syncthreads();
    const int r = blockIdx.x * kBinRows + threadIdx.x;
    if (r < g.n) atomicAdd(&hist[bin_of(g, r, true)], 1);
    __syncthreads();
    if (threadIdx.x < kNumBins) blk_counts[threadIdx.x * nblk + blockIdx.x] = hist[threadIdx.x];
}

// One block: exclusive scan of the (bin-major) block counts in place; bin
// starts into ctl->bin_off (and offsets_out for the public grouping call).
__global__ void __launch_bounds__(1024) k_group_scan(int nblk, int* blk_counts, Ctl* ctl,
                                                     int* offsets_out, int ngroups) {
    __shared__ int scratch[33];
    const long long total_n = (long long)kNumBins * nblk;
    int carry = 0;
    for (long long base = 0; base < total_n; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        const int v = i < total_n ? blk_counts[i] : 0;
        int tot;
        const int ex = block_excl_scan(v, scratch, &tot);
        if (i < total_n) blk_counts[i] = carry + ex;
        carry += tot;
    }
    __syncthreads();
    if (threadIdx.x <= kNumBins) {
        const int b = threadIdx.x;
        int off;
        if (b == kNumBins) off = carry;
        else off = nblk > 0 ? blk_counts[(long long)b * nblk] : 0;
        ctl->bin_off[b] = off;
        if (offsets_out && b <= ngroups) offsets_out[b] = b == ngroups ? carry : off;
    }
    if (threadIdx.x < kMaxTiers) ctl->work[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        ctl->dense_wide = 0;
        ctl->dense_uncached = 0;
    }
}

__global__ void __launch_bounds__(kBinRows) k_group_scatter(GroupArgs g, int nblk,
                                                            const int* blk_counts, int* map,
                                                            Ctl* ctl) {
    __shared__ int wcount[kBinRows / 32][kNumBins];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    for (int i = threadIdx.x; i < (kBinRows / 32) * kNumBins; i += blockDim.x)
        (&wcount[0][0])[i] = 0;
    __syncthreads();
    const int r = blockIdx.x * kBinRows + threadIdx.x;
    const int b = r < g.n ? bin_of(g, r, false) : -1;
    // accumulation: flag an fp32 dense row too wide for the rank-compacted
    // kernel, so the fallback kernel runs only when it has rows
    // and an fp64-bound dense row without a cached bitmap, so the kernel
    // for those runs only when there are some
    if (g.phase == 1 && b >= NB_DENSE32_0 && b < NB_DENSE32_0 + NB_DENSE_N) {
        const int row = g.row_begin + r;
        if (g.rptA[row + 1] - g.rptA[row] > kRankTileEntries) ctl->dense_wide = 1;
    }
    if (g.phase == 1 && b >= NB_DENSE64_0 && b < NB_DENSE64_0 + NB_DENSE_N &&
        (g.rc_slot == nullptr || g.rc_slot[g.row_begin + r] < 0))
        ctl->dense_uncached = 1;
    const unsigned peers = __match_any_sync(kFull, b);
    const int rank = __popc(peers & lanemask_lt());
    if (b >= 0 && rank == 0) wcount[warp][b] = __popc(peers);
    __syncthreads();
    if (threadIdx.x < kNumBins) {
        int acc = 0;
        for (int w = 0; w < kBinRows / 32; ++w) {
            const int c = wcount[w][threadIdx.x];
            wcount[w][threadIdx.x] = acc;
            acc += c;
        }
    }
    __syncthreads();
    if (b >= 0) map[blk_counts[(long long)b * nblk + blockIdx.x] + wcount[warp][b] + rank] = r;
}

void launch_group(const spgemm_plan* p, const GroupArgs& g, const WsPtrs& w, int* map_out,
                  int* offsets_out, cudaStream_t s) {
    const int nblk = (g.n + kBinRows - 1) / kBinRows;
    if (nblk > 0)
        SPG_LAUNCH(p, K_GROUP_HIST, s, k_group_hist<<<nblk, kBinRows, 0, s>>>(g, nblk, w.blk_counts));
    SPG_LAUNCH(p, K_GROUP_SCAN, s,
               k_group_scan<<<1, 1024, 0, s>>>(nblk, w.blk_counts, w.ctl, offsets_out,
                                               g.phase == 2 ? g.nthr + 1 : 0));
    if (nblk > 0)
        SPG_LAUNCH(p, K_GROUP_SCATTER, s,
                   k_group_scatter<<<nblk, kBinRows, 0, s>>>(g, nblk, w.blk_counts, map_out, w.ctl));
}

// ---------------------------------------------------------------------------
// Row pointers: exclusive scan of int32 counts with an int64 running total
// (reduce, scan of block sums, local scan). Overflow past INT32_MAX is
// flagged; the caller then works on blocks of rows.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(1024) k_scan_part(const int* x, int n, long long* part) {
    __shared__ long long red[33];
    const long long base = (long long)blockIdx.x * kScanItems;
    long long acc = 0;
    for (int i = threadIdx.x; i < kScanItems; i += blockDim.x) {
        const long long q = base + i;
        if (q < n) acc += x[q];
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__device__ __forceinline__ long long block_excl_scan64(long long v, long long* scratch,
                                                       long long* total) {
    const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    long long incl = warp_incl_scan64(v);
    if (lane == 31) scratch[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long wv = lane < nwarps ? scratch[lane] : 0;
        long long wi = warp_incl_scan64(wv);
        scratch[lane] = wi - wv;
        if (lane == 31) scratch[32] = wi;
    }
    __syncthreads();
    const long long r = scratch[warp] + incl - v;
    *total = scratch[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) k_scan_top(long long* part, int nscan, Ctl* ctl,
                                                   int* row_ptr, int n) {
    __shared__ long long scratch[33];
    long long carry = 0;
    for (int base = 0; base < nscan; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long v = i < nscan ? part[i] : 0;
        long long tot;
        const long long ex = block_excl_scan64(v, scratch, &tot);
        if (i < nscan) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        part[nscan] = carry;
        ctl->totals[2] = carry;
        if (carry > 2147483647ll) set_status(ctl, ST_OVERFLOW);
        row_ptr[n] = (int)carry;
    }
}

__global__ void __launch_bounds__(1024) k_scan_final(const int* x, int n, const long long* part,
                                                     int* row_ptr) {
    __shared__ long long scratch[33];
    constexpr int kPer = kScanItems / 1024;
    const long long base = (long long)blockIdx.x * kScanItems + (long long)threadIdx.x * kPer;
    int v[kPer];
    long long sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        v[q] = base + q < n ? x[base + q] : 0;
        sum += v[q];
    }
    long long tot;
    long long ex = block_excl_scan64(sum, scratch, &tot) + part[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        if (base + q < n) row_ptr[base + q] = (int)ex;
        ex += v[q];
    }
}

void launch_row_ptr(const spgemm_plan* p, const int* row_nnz, int n, const WsPtrs& w,
                    int* row_ptr, cudaStream_t s) {
    const int nscan = (n + kScanItems - 1) / kScanItems;
    if (nscan > 0)
        SPG_LAUNCH(p, K_SCAN_PART, s, k_scan_part<<<nscan, 1024, 0, s>>>(row_nnz, n, w.scan_part));
    SPG_LAUNCH(p, K_SCAN_TOP, s,
               k_scan_top<<<1, 1024, 0, s>>>(w.scan_part, nscan, w.ctl, row_ptr, n));
    if (nscan > 0)
        SPG_LAUNCH(p, K_SCAN_FINAL, s,
                   k_scan_final<<<nscan, 1024, 0, s>>>(row_nnz, n, w.scan_part, row_ptr));
}

}  // namespace spg

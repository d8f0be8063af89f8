// Allocation (symbolic) phase: nnz of every row of C (Algorithms 2-4).
//
// Row tiers (bins from the grouping phase):
//   ESC   IP <= 32 and |A_i| <= 32: one warp, one product per lane; distinct
//         columns counted with __match_any_sync, no table at all.
//   WARP  IP <= 1024: one warp per row, open-addressing table of keys in
//         shared memory (Algorithm 4's InsertIntoTable), sized 2*IP.
//   BLOCK IP <= 16384: one block per row, shared table sized 2*IP.
//   DENSE larger rows: one block per row, a bitmap over the columns in
//         shared memory (192 KB = 1.5M columns per pass); every product is a
//         single atomicOr and nnz is a popcount, so no row ever overflows a
//         table and no global-memory table is needed.
#include "internal.h"

namespace spg {

constexpr int kSymDenseUnroll = 6;   // products per warp step batch (4 / 6 / 8 -> 108.5 / 101.7 / 103.4 ms)
constexpr int kSymBlockUnroll = 4;   // block hash tier (2 / 4 -> 11.8 / 11.2 ms)

constexpr int kSymDenseWords = 48 * 1024;   // 192 KB bitmap (1.5M columns per pass)

__device__ __forceinline__ int hash_insert(int* table, int bits, int key, Ctl* ctl) {
    const unsigned mask = (1u << bits) - 1u;
    unsigned h = hash_slot(key, bits);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int cur = *(volatile int*)&table[h];
        if (cur == key) return 0;
        if (cur == kEmpty) {
            const int old = atomicCAS(&table[h], kEmpty, key);
            if (old == kEmpty) return 1;
            if (old == key) return 0;
        }
        h = (h + 1u) & mask;
    }
    set_status(ctl, ST_INTERNAL);
    return 0;
}

__device__ __forceinline__ bool key_ok(int key, const CsrDev& B, Ctl* ctl) {
    if ((unsigned)key >= (unsigned)B.cols) {
        set_status(ctl, ST_INVALID);
        return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_sym_esc(CsrDev A, CsrDev B, const int* map, Ctl* ctl,
                                                 int* row_nnz, int bin) {
    const int begin = ctl->bin_off[bin], end = ctl->bin_off[bin + 1];
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int idx = begin + gw; idx < end; idx += nw) {
        const int row = map[idx];
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        int bs = 0, len = 0;
        if (rs + lane < re) a_entry(A, B, rs + lane, bs, len, ctl);
        const int incl = warp_incl_scan(len);
        const int excl = incl - len;
        const int total = __shfl_sync(kFull, incl, 31);
        const int s = warp_find_src(excl, lane);
        const int sbs = __shfl_sync(kFull, bs, s);
        const int sex = __shfl_sync(kFull, excl, s);
        int key = -1;
        if (lane < total) {
            key = B.col[sbs + lane - sex];
            if (!key_ok(key, B, ctl)) key = -1;
        }
        const unsigned peers = __match_any_sync(kFull, key);
        const bool first = key >= 0 && (peers & lanemask_lt()) == 0;
        const int nnz = __popc(__ballot_sync(kFull, first));
        if (lane == 0) {
            if (total > 32 || re - rs > 32) set_status(ctl, ST_INTERNAL);
            row_nnz[row] = nnz;
        }
    }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kWarpsPerBlockSW * 32) k_sym_warp(CsrDev A, CsrDev B,
                                                                    const long long* ip,
                                                                    const int* map, Ctl* ctl,
                                                                    int* row_nnz, int bin,
                                                                    int load_pct) {
    extern __shared__ int sm_tables[];
    int* table = sm_tables + (threadIdx.x >> 5) * kWarpTableSym;
    const int begin = ctl->bin_off[bin], end = ctl->bin_off[bin + 1];
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    constexpr int kMaxBits = 11;   // 2048 slots
    for (int idx = begin + gw; idx < end; idx += nw) {
        const int row = map[idx];
        const int bits = table_bits(ip[row], load_pct, 5, kMaxBits);
        const int T = 1 << bits;
        for (int t = lane; t < T; t += 32) table[t] = kEmpty;
        __syncwarp();
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        int cnt = 0;
        warp_expand(A, B, rs, re, 32, ctl, [&](int t, int) {
            const int key = B.col[t];
            if (key_ok(key, B, ctl)) cnt += hash_insert(table, bits, key, ctl);
        });
        cnt = warp_sum(cnt);
        if (lane == 0) row_nnz[row] = cnt;
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// kT threads per block: kSymBlockThreads, or kBlockThreadsFull for the
// full-size table's launch (one block per SM)
template <int kT>
__global__ void __launch_bounds__(kT) k_sym_block(CsrDev A, CsrDev B,
                                                                const long long* ip,
                                                                const int* map, Ctl* ctl,
                                                                int* row_nnz, int bin_lo,
                                                                int bin_hi, int tier,
                                                                int max_bits, int load_pct) {
    extern __shared__ int table[];
    __shared__ int s_idx;
    __shared__ int red[33];
    __shared__ ExpandTile<kT, float> tile;
    const int begin = ctl->bin_off[bin_lo], end = ctl->bin_off[bin_hi];
    for (;;) {
        if (threadIdx.x == 0) s_idx = begin + atomicAdd(&ctl->work[tier], 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= end) break;
        const int row = map[idx];
        const int bits = table_bits(ip[row], load_pct, 6, max_bits);
        const int T = 1 << bits;
        for (int t = threadIdx.x; t < T; t += blockDim.x) table[t] = kEmpty;
        __syncthreads();
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        int cnt = 0;
        block_expand<kT, float, kSymBlockUnroll>(
            rs, re, tile,
            [&](int j, int& bs, int& len, float&) { a_entry(A, B, j, bs, len, ctl); },
            [&](int t) { return B.col[t]; },
            [&](int key, float) {
                if (key_ok(key, B, ctl)) cnt += hash_insert(table, bits, key, ctl);
            });
        cnt = block_sum(cnt, red);
        if (threadIdx.x == 0) row_nnz[row] = cnt;
    }
}

// ---------------------------------------------------------------------------
// Staged block hash tier: a software form of the near-memory range-2 access
// the paper's AIA hardware performs (Section IV-D). For a row, the
// row-pointer pairs of B selected by its A entries are gathered first, tile
// by tile (the range-2 gather), then every B-row segment the row needs is
// copied into shared memory with cp.async, so that the hash inserts read
// their keys from shared memory in order, with no segment search and no
// global load in the insert loop. Rows are double-buffered: the copies of
// the next row are in flight while the current row is inserted. Rows of at
// most kStageMax products (the bins of the block tier below 2^13) take this
// kernel when opts.stage_b is set; the result is the same as k_sym_block's.
constexpr int kStageMax = 8192;
constexpr int kStageThreads = 512;

__device__ __forceinline__ void cp_async4(int* smem, const int* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(kStageThreads) k_sym_block_staged(CsrDev A, CsrDev B,
                                                                    const long long* ip,
                                                                    const int* map, Ctl* ctl,
                                                                    int* row_nnz, int bin_lo,
                                                                    int bin_hi, int tier,
                                                                    int load_pct) {
    extern __shared__ int sm_staged[];
    int* table = sm_staged;                        // [2 * kStageMax] keys
    int* stage = sm_staged + 2 * kStageMax;        // [2][kStageMax] staged columns of B
    __shared__ int s_idx;
    __shared__ int s_off[kStageThreads + 1];       // prefix of the tile's segment lengths
    __shared__ int s_bs[kStageThreads];
    __shared__ int red[33];
    const int t = threadIdx.x;
    const int begin = ctl->bin_off[bin_lo], end = ctl->bin_off[bin_hi];

    auto next_row = [&]() -> int {
        if (t == 0) {
            const int idx = begin + atomicAdd(&ctl->work[tier], 1);
            s_idx = idx < end ? map[idx] : -1;
        }
        __syncthreads();
        const int row = s_idx;
        __syncthreads();
        return row;
    };
    // range-2 gather and copies of one row into stage buffer q; returns its
    // products (rows above kStageMax products are flagged and cut short,
    // which the host's bin choice rules out)
    auto stage_row = [&](int row, int q) -> int {
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        int pos = 0;
        for (int tb = rs; tb < re; tb += kStageThreads) {
            const int j = tb + t;
            int bs = 0, len = 0;
            if (j < re) a_entry(A, B, j, bs, len, ctl);
            int tot;
            const int ex = block_excl_scan(len, red, &tot);
            s_off[t] = ex;
            s_bs[t] = bs;
            if (t == 0) s_off[kStageThreads] = tot;
            __syncthreads();
            if (pos + tot > kStageMax) {
                if (t == 0) set_status(ctl, ST_INTERNAL);
                tot = kStageMax - pos;
            }
            int* dst = stage + q * kStageMax + pos;
            for (int p = t; p < tot; p += kStageThreads) {
                // entry holding product p: the last e with s_off[e] <= p
                int lo = 0, hi = kStageThreads - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= p) lo = mid;
                    else hi = mid - 1;
                }
                cp_async4(dst + p, B.col + s_bs[lo] + (p - s_off[lo]));
            }
            pos += tot;
            __syncthreads();                       // s_off / s_bs are rewritten next tile
        }
        return pos;
    };

    int q = 0;
    int row = next_row();
    int n = row >= 0 ? stage_row(row, 0) : 0;
    cp_async_commit();
    while (row >= 0) {
        const int row_next = next_row();
        const int n_next = row_next >= 0 ? stage_row(row_next, q ^ 1) : 0;
        cp_async_commit();
        cp_async_wait<1>();                        // this row's copies (the older group)
        __syncthreads();
        const int bits = table_bits(ip[row], load_pct, 6, 14);
        const int T = 1 << bits;
        for (int i = t; i < T; i += kStageThreads) table[i] = kEmpty;
        __syncthreads();
        const int* keys = stage + q * kStageMax;
        int cnt = 0;
        for (int p = t; p < n; p += kStageThreads) {
            const int key = keys[p];
            if (key_ok(key, B, ctl)) cnt += hash_insert(table, bits, key, ctl);
        }
        cnt = block_sum(cnt, red);
        if (t == 0) row_nnz[row] = cnt;
        row = row_next;
        n = n_next;
        q ^= 1;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// With a row bitmap cache (rc_slot != nullptr), a row that fits one pass and
// whose entry count puts it in a dense accumulation tier (nnz > cache_min)
// takes the next free slot and leaves its column bitmap there for the
// accumulation phase.
__global__ void __launch_bounds__(kSymDenseThreads, 1) k_sym_dense(CsrDev A, CsrDev B,
                                                                const int* map, Ctl* ctl,
                                                                int* row_nnz, int bin_lo,
                                                                int bin_hi, int tier,
                                                                int nwords, int* rc_slot,
                                                                unsigned* rc_bits, int rc_nslots,
                                                                int rc_wpr, int cache_min,
                                                                int* rc_pc, int P, int wpp) {
    extern __shared__ unsigned bm[];
    __shared__ int s_idx, s_slot;
    __shared__ int red[33];
    __shared__ int s_pc[kMaxPanels];    // entries per table panel of a one-pass row
    __shared__ ExpandTile<kSymDenseThreads, float> tile;
    const int begin = ctl->bin_off[bin_lo], end = ctl->bin_off[bin_hi];
    const long long span_max = (long long)nwords * 32;
    for (;;) {
        if (threadIdx.x == 0) s_idx = begin + atomicAdd(&ctl->work[tier], 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= end) break;
        const int row = map[idx];
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        int nnz = 0;
        for (long long c0l = 0; c0l < B.cols; c0l += span_max) {
            const int c0 = (int)c0l;                  // below B.cols, so it fits
            const int span = (int)(B.cols - c0l < span_max ? B.cols - c0l : span_max);
            const int nw = (span + 31) >> 5;
            for (int q = threadIdx.x; q < nw; q += blockDim.x) bm[q] = 0u;
            __syncthreads();
            block_expand<kSymDenseThreads, float, kSymDenseUnroll>(
                rs, re, tile,
                [&](int j, int& bs, int& len, float&) { a_entry(A, B, j, bs, len, ctl); },
                [&](int t) { return B.col[t]; },
                [&](int key, float) {
                    // one unsigned compare: in [c0, c0 + span) or not (a column
                    // outside B never is; it is flagged on the slow side)
                    const unsigned kk = (unsigned)key - (unsigned)c0;
                    if (kk < (unsigned)span) atomicOr(&bm[kk >> 5], 1u << (kk & 31));
                    else key_ok(key, B, ctl);
                });
            int cnt = 0;
            // one-pass rows with a cache: the count by table panel (a warp
            // per panel), kept for the accumulation phase's pass offsets
            const bool by_panel = rc_pc != nullptr && c0l == 0 && B.cols <= span_max && P <= kMaxPanels;
            if (by_panel) {
                const int lane = lane_id(), nwarp = blockDim.x >> 5;
                for (int p = threadIdx.x >> 5; p < P; p += nwarp) {
                    const int w0 = p * wpp, w1 = w0 + wpp < nw ? w0 + wpp : nw;
                    int c = 0;
                    for (int q = w0 + lane; q < w1; q += 32) c += __popc(bm[q]);
                    c = warp_sum(c);
                    if (lane == 0) {
                        s_pc[p] = c;
                        cnt += c;
                    }
                }
            } else {
                for (int q = threadIdx.x; q < nw; q += blockDim.x) cnt += __popc(bm[q]);
            }
            nnz += block_sum(cnt, red);
            // (block_sum ends with a barrier: bm and s_pc are final here)
            if (rc_slot != nullptr && c0l == 0 && B.cols <= span_max && nnz > cache_min &&
                nw == rc_wpr) {
                if (threadIdx.x == 0) {
                    const int slot = atomicAdd(&ctl->rc_used, 1);
                    s_slot = slot < rc_nslots ? slot : -1;
                    rc_slot[row] = s_slot;
                }
                __syncthreads();
                const int slot = s_slot;
                if (slot >= 0) {
                    unsigned* dst = rc_bits + (size_t)slot * rc_wpr;
                    for (int q = threadIdx.x; q < nw; q += blockDim.x) dst[q] = bm[q];
                    if (by_panel)
                        for (int p = threadIdx.x; p < P; p += blockDim.x) rc_pc[(size_t)slot * P + p] = s_pc[p];
                }
            }
        }
        if (threadIdx.x == 0) row_nnz[row] = nnz;
    }
}

// Every row starts without a cached bitmap; the slot counter restarts.
__global__ void k_rc_reset(int* rc_slot, int m, Ctl* ctl) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x)
        rc_slot[i] = -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->rc_used = 0;
}

// Narrow B (<= kNarrowCols columns): one warp per row marks the row's
// columns in a per-warp bitmap of 32 words (word w holds columns 32w..32w+31)
// and counts them; no table, no probing.
__global__ void __launch_bounds__(kNarrowMaxWarps * 32) k_sym_narrow(CsrDev A, CsrDev B,
                                                                     const int* map, Ctl* ctl,
                                                                     int* row_nnz, int bin) {
    extern __shared__ unsigned bmw[];           // 32 words per warp
    const int lane = lane_id();
    unsigned* bm = bmw + (threadIdx.x >> 5) * 32;
    bm[lane] = 0u;
    __syncwarp();
    const int begin = ctl->bin_off[bin], end = ctl->bin_off[bin + 1];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int idx = begin + gw; idx < end; idx += nw) {
        const int row = map[idx];
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        warp_expand(A, B, rs, re, 32, ctl, [&](int t, int) {
            const int key = B.col[t];
            if (key_ok(key, B, ctl)) atomicOr(&bm[key >> 5], 1u << (key & 31));
        });
        __syncwarp();
        const int cnt = warp_sum(__popc(bm[lane]));
        bm[lane] = 0u;
        __syncwarp();
        if (lane == 0) row_nnz[row] = cnt;
    }
}

// ---------------------------------------------------------------------------

// table of the block tier's two lighter bins: their rows hold at most
// 2^(Lmax - 2) products (Lmax = log2 of block_max_ip, rounded up), so at most
// that many distinct columns, at most half of 2^(Lmax - 1) slots
static size_t sym_block_small_smem(const spgemm_plan* p) {
    const int Lmax = log2_ceil_ll(p->opts.block_max_ip);
    const int bits = Lmax - 1 > 6 ? Lmax - 1 : 6;
    return (size_t)4 << bits;
}
// and of its second bin (at most 2^(Lmax - 1) products)
static size_t sym_block_mid_smem(const spgemm_plan* p) {
    const int Lmax = log2_ceil_ll(p->opts.block_max_ip);
    const int bits = Lmax > 6 ? Lmax : 6;
    return (size_t)4 << bits;
}

static size_t sym_dense_smem(const spgemm_plan* p) {
    size_t words = kSymDenseWords;
    const size_t stat = sizeof(ExpandTile<kSymDenseThreads, float>) + sizeof(int) * kMaxPanels + 1024;
    const size_t cap = (p->smem_optin > stat + 4096 ? p->smem_optin - stat : 4096) / 4;
    if (words > cap) words = cap;
    return words * 4;
}

static size_t staged_smem() { return sizeof(int) * 4 * (size_t)kStageMax; }

void occupancy_symbolic(spgemm_plan* p) {
    allow_max_dynamic_smem((const void*)k_sym_block_staged, p);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occ_sym_staged, k_sym_block_staged,
                                                  kStageThreads, staged_smem());
    if (p->occ_sym_staged < 1) p->occ_sym_staged = 1;
    const size_t sw = (size_t)kWarpsPerBlockSW * kWarpTableSym * 4;
    const size_t sb = (size_t)pow2_ceil(2u * (unsigned)p->opts.block_max_ip) * 4;
    const size_t sd = sym_dense_smem(p);
    allow_max_dynamic_smem((const void*)k_sym_warp, p);
    allow_max_dynamic_smem((const void*)k_sym_block<kBlockThreadsFull>, p);
    allow_max_dynamic_smem((const void*)k_sym_block<kSymBlockThreads>, p);
    allow_max_dynamic_smem((const void*)k_sym_dense, p);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occ_sym_warp, k_sym_warp,
                                                  kWarpsPerBlockSW * 32, sw);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occ_sym_block, k_sym_block<kBlockThreadsFull>,
                                                  kBlockThreadsFull, sb);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occ_sym_block_small, k_sym_block<kSymBlockThreads>,
                                                  kSymBlockThreads, sym_block_small_smem(p));
    if (p->occ_sym_block_small < 1) p->occ_sym_block_small = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occ_sym_block_mid, k_sym_block<kSymBlockThreads>,
                                                  kSymBlockThreads, sym_block_mid_smem(p));
    if (p->occ_sym_block_mid < 1) p->occ_sym_block_mid = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p->occ_sym_dense, k_sym_dense,
                                                  kSymDenseThreads, sd);
    if (p->occ_sym_warp < 1) p->occ_sym_warp = 1;
    if (p->occ_sym_block < 1) p->occ_sym_block = 1;
    if (p->occ_sym_dense < 1) p->occ_sym_dense = 1;
}

void launch_symbolic(const spgemm_plan* p, const CsrDev& A, const CsrDev& B, const long long* ip,
                     const WsPtrs& w, int* row_nnz, cudaStream_t s) {
    GroupArgs g{};
    g.phase = 0;
    g.row_begin = 0;
    g.n = A.rows;
    g.ip = ip;
    g.rptA = A.rpt;
    g.row_nnz = row_nnz;
    g.bcols = B.cols;
    g.opts = p->opts;
    launch_group(p, g, w, w.map, nullptr, s);
    if (A.rows == 0) return;
    const int sms = p->num_sms;
    if (w.rc_slot)
        SPG_LAUNCH(p, K_FILL, s, k_rc_reset<<<sms * 4, 256, 0, s>>>(w.rc_slot, A.rows, w.ctl));
    SPG_LAUNCH(p, K_SYM_ESC, s, k_sym_esc<<<sms * 8, 256, 0, s>>>(A, B, w.map, w.ctl, row_nnz, SB_ESC));
    const size_t sw = (size_t)kWarpsPerBlockSW * kWarpTableSym * 4;
    SPG_LAUNCH(p, K_SYM_WARP, s,
               k_sym_warp<<<sms * p->occ_sym_warp, kWarpsPerBlockSW * 32, sw, s>>>(
                   A, B, ip, w.map, w.ctl, row_nnz, SB_WARP, hash_load(p)));
    const unsigned tb = pow2_ceil(2u * (unsigned)p->opts.block_max_ip);
    int max_bits = 0;
    while ((1u << max_bits) < tb) ++max_bits;
    // staged tier (opts.stage_b): the block-tier bins whose rows hold at most
    // kStageMax products; bin SB_BLOCK0 + q holds IP <= 2^(Lmax - q)
    int staged_lo = SB_BLOCK0 + SB_BLOCK_N;
    if (p->opts.stage_b) {
        const int Lmax = log2_ceil_ll(p->opts.block_max_ip);
        for (int q = 0; q < SB_BLOCK_N; ++q)
            if ((1ll << (Lmax - q > 0 ? Lmax - q : 0)) <= kStageMax ||
                (q == 0 && p->opts.block_max_ip <= kStageMax)) {
                staged_lo = SB_BLOCK0 + q;
                break;
            }
    }
    // bin SB_BLOCK0 with the full table (one block per SM), bin +1 (IP at
    // most half of block_max_ip) with a half-size table, the two lighter
    // bins (at most a quarter) with a quarter-size table: the smaller the
    // table, the more blocks share an SM
    const int mid = staged_lo < SB_BLOCK0 + 1 ? staged_lo : SB_BLOCK0 + 1;
    const int split = staged_lo < SB_BLOCK0 + 2 ? staged_lo : SB_BLOCK0 + 2;
    SPG_LAUNCH(p, K_SYM_BLOCK, s,
               k_sym_block<kBlockThreadsFull><<<sms * p->occ_sym_block, kBlockThreadsFull, (size_t)tb * 4, s>>>(
                   A, B, ip, w.map, w.ctl, row_nnz, SB_BLOCK0, mid, 0, max_bits,
                   hash_load(p)));
    if (mid < split) {
        const size_t sm = sym_block_mid_smem(p);
        int mid_bits = 0;
        while (((size_t)4 << mid_bits) < sm) ++mid_bits;
        SPG_LAUNCH(p, K_SYM_BLOCK, s,
                   k_sym_block<kSymBlockThreads><<<sms * p->occ_sym_block_mid, kSymBlockThreads, sm, s>>>(
                       A, B, ip, w.map, w.ctl, row_nnz, mid, split, 4, mid_bits,
                       hash_load(p)));
    }
    if (split < staged_lo) {
        const size_t ss = sym_block_small_smem(p);
        int small_bits = 0;
        while (((size_t)4 << small_bits) < ss) ++small_bits;
        SPG_LAUNCH(p, K_SYM_BLOCK, s,
                   k_sym_block<kSymBlockThreads><<<sms * p->occ_sym_block_small, kSymBlockThreads, ss, s>>>(
                       A, B, ip, w.map, w.ctl, row_nnz, split, staged_lo, 3, small_bits,
                       hash_load(p)));
    }
    if (staged_lo < SB_BLOCK0 + SB_BLOCK_N)
        SPG_LAUNCH(p, K_SYM_BLOCK, s,
                   k_sym_block_staged<<<sms * p->occ_sym_staged, kStageThreads, staged_smem(), s>>>(
                       A, B, ip, w.map, w.ctl, row_nnz, staged_lo, SB_BLOCK0 + SB_BLOCK_N, 2,
                       hash_load(p)));
    if (B.cols <= kNarrowCols)
        SPG_LAUNCH(p, K_SYM_NARROW, s,
                   k_sym_narrow<<<sms * (64 / narrow_warps(p) > 1 ? 64 / narrow_warps(p) : 1),
                                  narrow_warps(p) * 32, (size_t)narrow_warps(p) * 128, s>>>(
                       A, B, w.map, w.ctl, row_nnz, SB_NARROW));
    const size_t sd = sym_dense_smem(p);
    SPG_LAUNCH(p, K_SYM_DENSE, s,
               k_sym_dense<<<sms * p->occ_sym_dense, kSymDenseThreads, sd, s>>>(
                   A, B, w.map, w.ctl, row_nnz, SB_DENSE0, SB_DENSE0 + SB_DENSE_N, 1, (int)(sd / 4),
                   w.rc_slot, w.rc_bits, w.rc_nslots, w.rc_wpr, p->opts.block_max_nnz, w.rc_pc,
                   w.panels, w.panel_cols / 32));
}

}  // namespace spg

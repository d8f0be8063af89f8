// Accumulation (numeric) phase with compaction and column sort
// (Algorithm 5, element gathering and column-index sorting steps).
//
// Row tiers (bins by the row's nnz, IP and A-row length):
//   ESC   IP <= 32: one warp, one product per lane; equal columns summed in
//         a fixed lane order and ranked by comparison, written sorted.
//   WARP  nnz <= 512: warp per row, (key, value) table in shared memory
//         (Algorithm 4's AddInTable), then in-place compaction and a bitonic
//         sort of the occupied slots.
//   BLOCK nnz <= 8192: block per row, same scheme with a block-wide table.
//   DENSE larger rows: block per row, a dense accumulator over one column
//         panel at a time (values + occupancy bitmap in shared memory). The
//         B entries of a panel are found through a per-B-row panel offset
//         table, so each product is read once; the bitmap is scanned in
//         column order, which emits the row already sorted (no sort step).
// Accumulators are fp32 where a row's A length keeps every output entry at
// <= fp32_max_terms products, fp64 otherwise.
#include "internal.h"

namespace spg {

template <typename Acc>
__device__ __forceinline__ void hash_add(int* keys, Acc* vals, int bits, int key, Acc v, Ctl* ctl) {
    const unsigned mask = (1u << bits) - 1u;
    unsigned h = hash_slot(key, bits);
    for (unsigned probe = 0; probe <= mask; ++probe) {
        const int cur = *(volatile int*)&keys[h];
        if (cur == key) {
            atomicAdd(&vals[h], v);
            return;
        }
        if (cur == kEmpty) {
            const int old = atomicCAS(&keys[h], kEmpty, key);
            if (old == kEmpty || old == key) {
                atomicAdd(&vals[h], v);
                return;
            }
        }
        h = (h + 1u) & mask;
    }
    set_status(ctl, ST_INTERNAL);
}

struct KeyVal {
    int key;
    float v;
};

__device__ __forceinline__ bool key_in(int key, const CsrDev& B, Ctl* ctl) {
    if ((unsigned)key >= (unsigned)B.cols) {
        set_status(ctl, ST_INVALID);
        return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_num_esc(CsrDev A, CsrDev B, const int* map, Ctl* ctl,
                                                 const int* rptC, int row_begin, int* colC,
                                                 float* valC, int bin) {
    const int begin = ctl->bin_off[bin], end = ctl->bin_off[bin + 1];
    const int lane = lane_id();
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int idx = begin + gw; idx < end; idx += nw) {
        const int r = map[idx];
        const int row = row_begin + r;
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        int bs = 0, len = 0;
        float a = 0.f;
        if (rs + lane < re) {
            a_entry(A, B, rs + lane, bs, len, ctl);
            a = A.val[rs + lane];
        }
        const int incl = warp_incl_scan(len);
        const int excl = incl - len;
        const int total = __shfl_sync(kFull, incl, 31);
        const int s = warp_find_src(excl, lane);
        const int sbs = __shfl_sync(kFull, bs, s);
        const int sex = __shfl_sync(kFull, excl, s);
        const float sa = __shfl_sync(kFull, a, s);
        int key = -1;
        float prod = 0.f;
        if (lane < total) {
            const int t = sbs + lane - sex;
            key = B.col[t];
            if (key_in(key, B, ctl)) prod = sa * B.val[t];
            else key = -1;
        }
        const unsigned peers = __match_any_sync(kFull, key);
        const int leader = (key >= 0 && (peers & lanemask_lt()) == 0) ? 1 : 0;
        float sum = 0.f;
        int rank = 0;
        for (int q = 0; q < 32; ++q) {
            const int kq = __shfl_sync(kFull, key, q);
            const float vq = __shfl_sync(kFull, prod, q);
            const int lq = __shfl_sync(kFull, leader, q);
            if (kq == key) sum += vq;
            if (lq && kq < key) ++rank;
        }
        const int out = rptC[r];
        const int nnz_row = rptC[r + 1] - out;
        const int distinct = __popc(__ballot_sync(kFull, leader));
        if (lane == 0 && (distinct != nnz_row || total > 32)) set_status(ctl, ST_INTERNAL);
        if (leader && rank < nnz_row) {
            colC[out + rank] = key;
            valC[out + rank] = sum;
        }
    }
}

// ---------------------------------------------------------------------------
// Bitonic sort of n2 (power of two) (key, value) pairs in shared memory,
// ascending by key, by `nthreads` cooperating threads starting at `tid`.
template <typename Acc, bool kBlock>
__device__ __forceinline__ void bitonic_sort(int* keys, Acc* vals, int n2, int tid, int nthreads) {
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < n2; i += nthreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const int ki = keys[i], kj = keys[ixj];
                    const bool asc = (i & k) == 0;
                    if ((ki > kj) == asc) {
                        keys[i] = kj;
                        keys[ixj] = ki;
                        const Acc t = vals[i];
                        vals[i] = vals[ixj];
                        vals[ixj] = t;
                    }
                }
            }
            if (kBlock) __syncthreads();
            else __syncwarp();
        }
    }
}

// Block-wide sort of n distinct keys keys[0, n) with their values, into
// keys[off, off + n) (the two ranges must not overlap): keys are bucketed on
// the high bits of key - min (about four per bucket), counted, scattered to
// their bucket's range and each bucket is then insertion-sorted by one
// thread. A few barriers instead of the log^2 stages of a sorting network.
// Returns false, with keys[0, n) untouched, when some bucket would hold more
// than kSortBucketMax keys (strongly clustered columns); the caller then
// sorts in place by other means. cnt holds kSortBuckets ints, mm 3 ints.
constexpr int kSortBuckets = 2048;
constexpr int kSortBucketMax = 32;

template <typename Acc>
__device__ bool block_bucket_sort(int* keys, Acc* vals, int n, int off, int* cnt, int* mm,
                                  int* scratch) {
    const int tid = threadIdx.x, bd = blockDim.x;
    int nb = (int)pow2_ceil((unsigned)((n + 3) >> 2));
    nb = nb < 32 ? 32 : (nb > kSortBuckets ? kSortBuckets : nb);
    const int lognb = 31 - __clz(nb);
    for (int b = tid; b < nb; b += bd) cnt[b] = 0;
    if (tid == 0) {
        mm[0] = 0x7fffffff;
        mm[1] = 0;
        mm[2] = 0;
    }
    __syncthreads();
    int lo = 0x7fffffff, hi = 0;
    for (int t = tid; t < n; t += bd) {
        const int k = keys[t];
        lo = k < lo ? k : lo;
        hi = k > hi ? k : hi;
    }
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    if (lane_id() == 0) {
        atomicMin(&mm[0], lo);
        atomicMax(&mm[1], hi);
    }
    __syncthreads();
    const int kmin = mm[0];
    const long long span = (long long)mm[1] - kmin + 1;
    int sh = log2_ceil_ll(span > 1 ? span : 1) - lognb;
    sh = sh < 0 ? 0 : sh;
    for (int t = tid; t < n; t += bd) atomicAdd(&cnt[(keys[t] - kmin) >> sh], 1);
    __syncthreads();
    // exclusive offsets of the buckets; largest bucket into mm[2]
    const int cpt = (nb + bd - 1) / bd;
    const int b0 = tid * cpt;
    int sum = 0, big = 0;
    for (int q = 0; q < cpt; ++q)
        if (b0 + q < nb) {
            const int c = cnt[b0 + q];
            sum += c;
            big = c > big ? c : big;
        }
    if (big > kSortBucketMax) atomicMax(&mm[2], big);
    int tot;
    int run = block_excl_scan(sum, scratch, &tot);
    for (int q = 0; q < cpt; ++q)
        if (b0 + q < nb) {
            const int c = cnt[b0 + q];
            cnt[b0 + q] = run;
            run += c;
        }
    __syncthreads();
    if (mm[2] > kSortBucketMax) return false;
    for (int t = tid; t < n; t += bd) {
        const int k = keys[t];
        const int p = atomicAdd(&cnt[(k - kmin) >> sh], 1);
        keys[off + p] = k;
        vals[off + p] = vals[t];
    }
    __syncthreads();
    // cnt[b] is now the end of bucket b
    for (int b = tid; b < nb; b += bd) {
        const int s0 = off + (b > 0 ? cnt[b - 1] : 0), e0 = off + cnt[b];
        for (int i = s0 + 1; i < e0; ++i) {
            const int k = keys[i];
            const Acc v = vals[i];
            int j = i - 1;
            while (j >= s0 && keys[j] > k) {
                keys[j + 1] = keys[j];
                vals[j + 1] = vals[j];
                --j;
            }
            keys[j + 1] = k;
            vals[j + 1] = v;
        }
    }
    __syncthreads();
    return true;
}

template <typename Acc>
__global__ void __launch_bounds__(kWarpsPerBlockNW * 32) k_num_warp(CsrDev A, CsrDev B,
                                                                    const int* map, Ctl* ctl,
                                                                    const int* rptC, int row_begin,
                                                                    int* colC, float* valC,
                                                                    int bin, int load_pct) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    Acc* vals = reinterpret_cast<Acc*>(sm_raw) + warp * kWarpTableNum;
    int* keys = reinterpret_cast<int*>(sm_raw + sizeof(Acc) * kWarpsPerBlockNW * kWarpTableNum) +
                warp * kWarpTableNum;
    const int begin = ctl->bin_off[bin], end = ctl->bin_off[bin + 1];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    constexpr int kMaxBits = 10;
    for (int idx = begin + gw; idx < end; idx += nw) {
        const int r = map[idx];
        const int row = row_begin + r;
        const int out = rptC[r];
        const int nnz_row = rptC[r + 1] - out;
        const int bits = table_bits(nnz_row, load_pct, 5, kMaxBits);
        const int T = 1 << bits;
        for (int t = lane; t < T; t += 32) {
            keys[t] = kEmpty;
            vals[t] = Acc(0);
        }
        __syncwarp();
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        warp_expand(A, B, rs, re, 32, ctl, [&](int t, int ja) {
            const int key = B.col[t];
            if (key_in(key, B, ctl))
                hash_add<Acc>(keys, vals, bits, key, (Acc)A.val[ja] * (Acc)B.val[t], ctl);
        });
        __syncwarp();
        int n = 0;
        for (int c = 0; c < T; c += 32) {
            const int k = keys[c + lane];
            const Acc v = vals[c + lane];
            const bool occ = k != kEmpty;
            const unsigned bal = __ballot_sync(kFull, occ);
            const int pos = n + __popc(bal & lanemask_lt());
            __syncwarp();
            if (occ) {
                keys[pos] = k;
                vals[pos] = v;
            }
            n += __popc(bal);
            __syncwarp();
        }
        if (lane == 0 && n != nnz_row) set_status(ctl, ST_INTERNAL);
        const int nn = n < nnz_row ? n : nnz_row;
        const int n2 = (int)pow2_ceil((unsigned)(nn > 1 ? nn : 1));
        for (int t = nn + lane; t < n2; t += 32) keys[t] = 0x7fffffff;
        __syncwarp();
        bitonic_sort<Acc, false>(keys, vals, n2, lane, 32);
        for (int t = lane; t < nn; t += 32) {
            colC[out + t] = keys[t];
            valC[out + t] = (float)vals[t];
        }
        __syncwarp();
    }
}

// Narrow B (<= kNarrowCols columns): one warp per row accumulates into a
// per-warp dense array over all of B's columns (fp32, or fp64 for rows
// where more than fp32_max_terms products can meet) and marks the columns in
// a 32-word bitmap; lane l owns word l, so a warp scan of the popcounts
// writes the row in column order with no sort. Touched entries are cleared
// on the way out, so the array stays zero between rows.
template <typename Acc>
__global__ void __launch_bounds__(kNarrowMaxWarps * 32) k_num_narrow(CsrDev A, CsrDev B,
                                                                     const int* map, Ctl* ctl,
                                                                     const int* rptC, int row_begin,
                                                                     int* colC, float* valC,
                                                                     int bin, int ncols_pad) {
    // per warp: a dense accumulator over B's columns, then a 32-word bitmap
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int warp = threadIdx.x >> 5, lane = lane_id();
    const int nwarps = blockDim.x >> 5;
    Acc* dense = reinterpret_cast<Acc*>(sm_raw) + warp * ncols_pad;
    unsigned* bm = reinterpret_cast<unsigned*>(reinterpret_cast<Acc*>(sm_raw) + nwarps * ncols_pad) +
                   warp * 32;
    for (int c = lane; c < ncols_pad; c += 32) dense[c] = Acc(0);
    bm[lane] = 0u;
    __syncwarp();
    const int begin = ctl->bin_off[bin], end = ctl->bin_off[bin + 1];
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int idx = begin + gw; idx < end; idx += nw) {
        const int r = map[idx];
        const int row = row_begin + r;
        const int out = rptC[r];
        const int nnz_row = rptC[r + 1] - out;
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        warp_expand(A, B, rs, re, 32, ctl, [&](int t, int ja) {
            const int key = B.col[t];
            if (key_in(key, B, ctl)) {
                atomicOr(&bm[key >> 5], 1u << (key & 31));
                atomicAdd(&dense[key], (Acc)A.val[ja] * (Acc)B.val[t]);
            }
        });
        __syncwarp();
        unsigned bits = bm[lane];
        const int cnt = __popc(bits);
        const int incl = warp_incl_scan(cnt);
        int pos = incl - cnt;
        const int tot = __shfl_sync(kFull, incl, 31);
        while (bits) {
            const int c = lane * 32 + __ffs(bits) - 1;
            bits &= bits - 1;
            if (pos < nnz_row) {
                colC[out + pos] = c;
                valC[out + pos] = (float)dense[c];
            }
            dense[c] = Acc(0);
            ++pos;
        }
        bm[lane] = 0u;
        if (lane == 0 && tot != nnz_row) set_status(ctl, ST_INTERNAL);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// kT threads per block: kNumBlockThreads, or kBlockThreadsFull for the
// launch whose full-size table leaves one block per SM (more warps to hide
// latency with)
template <typename Acc, int kT = kNumBlockThreads>
__global__ void __launch_bounds__(kT) k_num_block(CsrDev A, CsrDev B,
                                                                const int* map, Ctl* ctl,
                                                                const int* rptC, int row_begin,
                                                                int* colC, float* valC, int bin,
                                                                int tier, int max_bits,
                                                                int load_pct) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    Acc* vals = reinterpret_cast<Acc*>(sm_raw);
    int* keys = reinterpret_cast<int*>(sm_raw + sizeof(Acc) * (1u << max_bits));
    __shared__ int s_idx;
    __shared__ int scratch[33];
    __shared__ int s_cnt[kSortBuckets];
    __shared__ int s_mm[3];
    __shared__ ExpandTile<kT, Acc> tile;
    const int begin = ctl->bin_off[bin], end = ctl->bin_off[bin + 1];
    for (;;) {
        if (threadIdx.x == 0) s_idx = begin + atomicAdd(&ctl->work[tier], 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= end) break;
        const int r = map[idx];
        const int row = row_begin + r;
        const int out = rptC[r];
        const int nnz_row = rptC[r + 1] - out;
        const int bits = table_bits(nnz_row, load_pct, 6, max_bits);
        const int T = 1 << bits;
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            keys[t] = kEmpty;
            vals[t] = Acc(0);
        }
        __syncthreads();
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        // two products per lane per step (4 measured slower: 20.3 -> 21.6 ms)
        block_expand<kT, Acc, 2>(
            rs, re, tile,
            [&](int j, int& bs, int& len, Acc& a) {
                a_entry(A, B, j, bs, len, ctl);
                a = (Acc)A.val[j];
            },
            [&](int t) { return KeyVal{B.col[t], B.val[t]}; },
            [&](KeyVal kv, Acc a) {
                if (key_in(kv.key, B, ctl)) hash_add<Acc>(keys, vals, bits, kv.key, a * (Acc)kv.v, ctl);
            });
        // stable in-place compaction, 4 slots per thread per round
        int n = 0;
        const int per_round = blockDim.x * 4;
        for (int base = 0; base < T; base += per_round) {
            int k[4];
            Acc v[4];
            int cnt = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int slot = base + threadIdx.x * 4 + q;
                k[q] = slot < T ? keys[slot] : kEmpty;
                v[q] = slot < T ? vals[slot] : Acc(0);
                cnt += k[q] != kEmpty;
            }
            int tot;
            int pos = n + block_excl_scan(cnt, scratch, &tot);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (k[q] != kEmpty) {
                    keys[pos] = k[q];
                    vals[pos] = v[q];
                    ++pos;
                }
            }
            n += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0 && n != nnz_row) set_status(ctl, ST_INTERNAL);
        const int nn = n < nnz_row ? n : nnz_row;
        int so = T >> 1;                 // sorted run: keys[so, so + nn)
        if (nn > so || !block_bucket_sort<Acc>(keys, vals, nn, so, s_cnt, s_mm, scratch)) {
            const int n2 = (int)pow2_ceil((unsigned)(nn > 1 ? nn : 1));
            for (int t = nn + threadIdx.x; t < n2; t += blockDim.x) keys[t] = 0x7fffffff;
            __syncthreads();
            bitonic_sort<Acc, true>(keys, vals, n2, threadIdx.x, blockDim.x);
            so = 0;
        }
        for (int t = threadIdx.x; t < nn; t += blockDim.x) {
            colC[out + t] = keys[so + t];
            valC[out + t] = (float)vals[so + t];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Panel offset table of B: for row k and panel p, tab[k*(P+1)+p] is the
// first position of row k whose column is >= p*PW (valid when rows are
// sorted; an unsorted row sets bit 0 of ctl->b_unsorted and the dense tier
// then filters whole B rows instead; a sorted row that repeats a column sets
// bit 1). A warp per row; a binary search per table entry, so the table is
// written coalesced (3.8 -> 1.3 ms per benchmark step against lanes that
// each wrote the entries between their column and the one before).
__global__ void k_bpanel(CsrDev B, int P, int PW, int* tab, Ctl* ctl) {
    const int lane = lane_id();
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    // panel of a column (clamped to [0, P - 1], as the dense tiers clamp)
    auto panel = [&](int c) { return c < 0 ? 0 : (c / PW >= P ? P - 1 : c / PW); };
    for (long long k = gw; k < B.rows; k += nw) {
        int s, e;
        int* row = tab + k * (P + 1);
        if (!row_extent(B, (int)k, s, e, ctl)) {
            for (int p = lane; p <= P; p += 32) row[p] = 0;
            continue;
        }
        // sortedness and repeated columns: one coalesced sweep
        bool unsorted = false, dup = false;
        for (int t = s + 1 + lane; t < e; t += 32) {
            const int c = B.col[t], cp = B.col[t - 1];
            unsorted |= c < cp;
            dup |= c == cp;
        }
        // lane l owns entries l, l + 32, ... of the table row: the first
        // position whose column's panel is >= p (a binary search of the
        // row's sorted columns), so each table row is written coalesced
        for (int p = lane; p <= P; p += 32) {
            int lo = s, hi = e;
            if (p == P) {
                lo = e;
            } else {
                while (lo < hi) {
                    const int mid = lo + ((hi - lo) >> 1);
                    if (panel(B.col[mid]) < p) lo = mid + 1;
                    else hi = mid;
                }
            }
            row[p] = lo;
        }
        const int flags = (__any_sync(kFull, unsorted) ? 1 : 0) | (__any_sync(kFull, dup) ? 2 : 0);
        if (flags && lane == 0) atomicOr(&ctl->b_unsorted, flags);
    }
}

// Dense-panel accumulation of heavy rows. A pass covers W columns: a value
// array and an occupancy bitmap in shared memory; each product is one
// atomicOr and one fp32 atomicAdd; the pass is emitted in column order.
//
// kMode 0 (rows where at most fp32_max_terms products can meet in an entry):
//   fp32 values, W = 3 table panels.
// kMode 1 (rows with more A entries): the row's A entries are taken in
//   groups of kGroup (<= 165) entries. Inside a group at most kGroup
//   products meet in an entry, so fp32 accumulation stays within
//   gamma_kGroup of sum|a||b|; after each group its touched columns are
//   added into an fp64 array and cleared. With the final rounding to fp32
//   the total stays below 1e-5 * sum|a||b|, using fp32 shared-memory
//   atomics only (fp64 shared atomics run ~3.5x slower and collapse under
//   contention on hub columns). W = 1 table panel.
//
// A row with at most kNumDenseThreads A entries keeps each entry's B row,
// multiplier and current panel boundary in registers of "its" thread, and
// prefetches the next boundary before the pass runs. Longer rows re-read
// their entries (and the panel table) in tiles every pass.
constexpr int kGroup = 160;

// fp32 dense tier: threads per block, blocks per SM its passes are sized
// for, and products per warp step batch (512 x 2 and 256 x 4 blocks, and
// unroll 2 or 8, measured no faster on GB300)
constexpr int kD32Threads = 1024;
constexpr int kD32Blocks = 1;
constexpr int kD32Unroll = 4;

template <int kMode, int kT>
__global__ void __launch_bounds__(kT, 1024 / kT) k_num_dense(CsrDev A, CsrDev B, const int* map,
                                                            Ctl* ctl, const int* rptC,
                                                            int row_begin, int* colC,
                                                            float* valC, int bin_lo, int bin_hi,
                                                            int tier, const int* tab, int P,
                                                            int PW, int ppp, int rank_na) {
    constexpr int kNumDenseThreads = kT;
    const int kPanelsPerPass = kMode == 0 ? ppp : 1;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int W = PW * kPanelsPerPass;                 // columns per pass
    const int nwords_pass = W >> 5;
    double* acc = reinterpret_cast<double*>(sm_raw);   // kMode 1 only
    float* st = reinterpret_cast<float*>(sm_raw + (kMode == 1 ? sizeof(double) * W : 0));
    unsigned* bm = reinterpret_cast<unsigned*>(reinterpret_cast<unsigned char*>(st) + sizeof(float) * W);
    unsigned* gbm = bm + nwords_pass;                   // kMode 1 only
    __shared__ int s_idx;
    __shared__ int scratch[33];
    __shared__ ExpandTile<kNumDenseThreads, float> tile;
    const int begin = ctl->bin_off[bin_lo], end = ctl->bin_off[bin_hi];
    if (begin >= end) return;
    const bool use_tab = tab != nullptr && (ctl->b_unsorted & 1) == 0;
    // beside the rank-compacted kernel, only rows wider than its tile are
    // this kernel's; the grouping flags whether there are any
    if (rank_na > 0 && use_tab && ctl->dense_wide == 0) return;
    const int wpt = (nwords_pass + kNumDenseThreads - 1) / kNumDenseThreads;   // words per thread
    const int w0 = threadIdx.x * wpt;
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        st[i] = 0.f;
        if (kMode == 1) acc[i] = 0.0;
    }
    for (int i = threadIdx.x; i < nwords_pass; i += blockDim.x) {
        bm[i] = 0u;
        if (kMode == 1) gbm[i] = 0u;
    }
    const int npass = (int)((B.cols + (long long)W - 1) / W);
    const long long stride = P + 1;
    unsigned* obm = kMode == 1 ? gbm : bm;             // bitmap the products mark

    int c0 = 0, span = 0;
    auto load = [&](int t) { return KeyVal{B.col[t], B.val[t]}; };
    auto apply = [&](KeyVal kv, float a) {
        if (!key_in(kv.key, B, ctl)) return;
        const int kk = kv.key - c0;
        if (kk >= 0 && kk < span) {
            atomicOr(&obm[kk >> 5], 1u << (kk & 31));
            atomicAdd(&st[kk], a * kv.v);
        } else if (use_tab) {
            set_status(ctl, ST_INTERNAL);
        }
    };
    // kMode 1: move this group's sums into fp64 (thread owns words [w0, w0+wpt))
    auto flush = [&]() {
        for (int q = 0; q < wpt; ++q) {
            const int w = w0 + q;
            if (w >= nwords_pass) break;
            unsigned g = gbm[w];
            if (!g) continue;
            bm[w] |= g;
            gbm[w] = 0u;
            while (g) {
                const int kk = w * 32 + __ffs(g) - 1;
                g &= g - 1;
                acc[kk] += (double)st[kk];
                st[kk] = 0.f;
            }
        }
        __syncthreads();
    };

    for (;;) {
        if (threadIdx.x == 0) s_idx = begin + atomicAdd(&ctl->work[tier], 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= end) break;
        const int r = map[idx];
        const int row = row_begin + r;
        const int out = rptC[r];
        const int nnz_row = rptC[r + 1] - out;
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        const int na = re - rs;
        const bool cached = use_tab && na <= kNumDenseThreads;
        if (use_tab && na <= rank_na) continue;      // the rank-compacted kernel's row
        int myk = -1, cur = 0, nxt = 0;
        float mya = 0.f;
        if (cached && (int)threadIdx.x < na) {
            const int j = rs + threadIdx.x;
            const int k = A.col[j];
            if ((unsigned)k < (unsigned)B.rows) {
                myk = k;
                mya = A.val[j];
                cur = tab[(long long)k * stride];
                nxt = tab[(long long)k * stride + (kPanelsPerPass < P ? kPanelsPerPass : P)];
            } else {
                set_status(ctl, ST_INVALID);
            }
        }
        int written = 0;
        for (int pass = 0; pass < npass; ++pass) {
            c0 = pass * W;
            span = (int)(B.cols - (long long)c0 < W ? B.cols - (long long)c0 : W);
            const int p0 = pass * kPanelsPerPass;
            const int p1 = p0 + kPanelsPerPass < P ? p0 + kPanelsPerPass : P;
            if (cached) {
                int nxt2 = 0;
                if (myk >= 0 && pass + 1 < npass) {
                    const int pn = p1 + kPanelsPerPass < P ? p1 + kPanelsPerPass : P;
                    nxt2 = tab[(long long)myk * stride + pn];
                }
                int bs = 0, len = 0;
                if (myk >= 0) {
                    if (cur < 0 || nxt < cur || (long long)nxt > B.nnz) set_status(ctl, ST_INTERNAL);
                    else {
                        bs = cur;
                        len = nxt - cur;
                    }
                }
                if (kMode == 0) {
                    // long per-pass segments: padded expansion (no segment search)
                    expand_tile_padded<kNumDenseThreads, float, kD32Unroll>(tile, bs, len, mya, load,
                                                                           apply);
                } else {
                    for (int g0 = 0; g0 < na; g0 += kGroup) {
                        const bool mine = (int)threadIdx.x >= g0 && (int)threadIdx.x < g0 + kGroup;
                        expand_tile<kNumDenseThreads, float, 4>(tile, bs, mine ? len : 0, mya, load,
                                                                apply);
                        flush();
                    }
                }
                cur = nxt;
                nxt = nxt2;
            } else {
                const int T = kMode == 0 ? kNumDenseThreads : kGroup;
                for (int tb = rs; tb < re; tb += T) {
                    const int j = tb + threadIdx.x;
                    int bs = 0, len = 0;
                    float a = 0.f;
                    if ((int)threadIdx.x < T && j < re) {
                        a_entry(A, B, j, bs, len, ctl);
                        a = A.val[j];
                        if (use_tab && len > 0) {
                            const int* tk = tab + (long long)A.col[j] * stride;
                            const int ps = tk[p0], pe = tk[p1];
                            if (ps >= bs && pe >= ps && pe <= bs + len) {
                                bs = ps;
                                len = pe - ps;
                            } else {
                                set_status(ctl, ST_INTERNAL);
                                len = 0;
                            }
                        }
                    }
                    if (kMode == 0)
                        expand_tile_padded<kNumDenseThreads, float, 4>(tile, bs, len, a, load, apply);
                    else
                        expand_tile<kNumDenseThreads, float, 4>(tile, bs, len, a, load, apply);
                    if (kMode == 1) flush();
                }
            }
            // emit this pass in column order
            const int nw = (span + 31) >> 5;
            written += emit_bitmap_lanes<kNumDenseThreads>(
                bm, 0, nw, c0, colC, valC, out, written, nnz_row, scratch, [&](int kk) {
                    float v;
                    if (kMode == 1) {
                        v = (float)acc[kk];
                        acc[kk] = 0.0;
                    } else {
                        v = st[kk];
                        st[kk] = 0.f;
                    }
                    return v;
                });
        }
        if (threadIdx.x == 0 && written != nnz_row) set_status(ctl, ST_INTERNAL);
    }
}

// Word ranks and columns of a thread's bitmap words [wb, wb + wpt) of a pass
// (run: the rank of its first entry; every rank below the value array's
// size). Two words per step, so the two bit-extraction chains interleave
// (fp32 dense tier 212 -> 208 ms; no gain in the fp64-bound tier).
__device__ __forceinline__ void stage_pairs(const unsigned* bm, int* rk, int* stage, int wb,
                                            int wpt, int nw, int run, int c0) {
    for (int q = 0; q < wpt; q += 2) {
        const int w = wb + q;
        if (w >= nw) break;
        const bool two = q + 1 < wpt && w + 1 < nw;
        unsigned x = bm[w];
        unsigned y = two ? bm[w + 1] : 0u;
        rk[w] = run;
        int rx = run;
        run += __popc(x);
        if (two) rk[w + 1] = run;
        int ry = run;
        run += __popc(y);
        const int cx = c0 + w * 32, cy = cx + 32;
        while (x | y) {
            if (x) {
                stage[rx++] = cx + __ffs(x) - 1;
                x &= x - 1;
            }
            if (y) {
                stage[ry++] = cy + __ffs(y) - 1;
                y &= y - 1;
            }
        }
    }
}

// fp32 dense tier with rank-compacted passes (rows whose A entries fit the
// block and whose B rows are sorted; k_num_dense<0> takes the others). A
// pass covers up to kRankPanels table panels; the row's occupancy is
// recorded first (a bitmap expansion: one atomicOr per product), then each
// bitmap word gets the rank of its first entry among the pass's entries and
// the pass's columns are written out (staged at their ranks in the value
// array, then stored coalesced: 8% faster than each thread storing its own
// words' columns, one sector per entry), then a second expansion adds every
// product into a compact value array at its entry's rank (word rank + the
// popcount of the lower bits), which is streamed out with coalesced stores.
// Shared memory per column is a bit and a 1/32 rank instead of a 4-byte
// value, so a pass spans many more columns than a dense value array allows:
// the passes per row, whose fixed cost (block scans, barriers, short
// per-warp work) dominates that tier, drop. The panels per pass are chosen
// per row so that the expected entries of a pass (nnz_row / P per panel)
// stay within 95% of the value array (75 / 85 / 95% measured 198.2 /
// 196.1 / 195.0 ms; on another box 95 / 100 / 110% 193.4 / 193.8 / 226.6
// ms); a pass that still holds more is accumulated in word ranges of at
// most `cap` entries.
// two 512-thread blocks per SM, each with half of the SM's shared memory
// (14 panels per pass, ~13K values), instead of one of 1024 (24 panels,
// ~32K values): one block's barriers and scans overlap the other's walk
// (193.4 -> 181.1 ms at 12 panels)
constexpr int kRankThreads = 512;
constexpr int kRankBlocks = 2;                    // per SM
// panels per pass (each block's share of the SM): 10 / 12 / 14 / 16 -> 182.1 /
// 181.1 / 180.3 / 202.4 ms (16 leaves too few values)
constexpr int kRankPanels = 14;
// products per lane per step of the value expansion: 4 / 5 / 6 -> 186.8 /
// 183.9 / 181.1 ms at 12 panels, 7 -> 189.5 ms at 14
constexpr int kRankUnroll = 6;
constexpr int kRankOccUnroll = 8;     // occupancy expansion items are one int
// A entries a row of this kernel may have (more go to k_num_dense<0>): the
// fp32 rule keeps dense rows to at most fp32_max_terms (167 by default)
// entries, and a tile of 256 entries leaves more shared memory for values
// than one entry per thread
constexpr int kRankTileE = kRankTileEntries;

// With a row bitmap cache, a row that holds a slot reads each pass's bitmap
// words from it (one coalesced copy) instead of the occupancy expansion.
__global__ void __launch_bounds__(kRankThreads, kRankBlocks) k_num_dense_rank(CsrDev A, CsrDev B,
                                                                   const int* map, Ctl* ctl,
                                                                   const int* rptC, int row_begin,
                                                                   int* colC, float* valC,
                                                                   int bin_lo, int bin_hi, int tier,
                                                                   const int* tab, int P, int PW,
                                                                   int pmax, int cap,
                                                                   const int* rc_slot,
                                                                   const unsigned* rc_bits,
                                                                   int rc_nslots, int rc_wpr,
                                                                   const int2* bcv) {
    constexpr int kT = kRankThreads;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int RW = (pmax * PW) >> 5;                  // words of the widest pass
    unsigned* bm = reinterpret_cast<unsigned*>(sm_raw);
    int* rk = reinterpret_cast<int*>(bm + RW);
    float* vals = reinterpret_cast<float*>(rk + RW);
    __shared__ int s_idx, s_hi;
    __shared__ int scratch[33];
    __shared__ ExpandTile<kT, float, kRankTileE> tile;
    const int begin = ctl->bin_off[bin_lo], end = ctl->bin_off[bin_hi];
    if (begin >= end) return;
    if (tab == nullptr || (ctl->b_unsorted & 1) != 0) return;     // fallback kernel's rows
    const int t = threadIdx.x;
    for (int i = t; i < RW; i += kT) bm[i] = 0u;
    for (int i = t; i < cap; i += kT) vals[i] = 0.f;
    const long long stride = P + 1;

    int c0 = 0, span = 0, lo = 0, hi = 0, rbase = 0;
    auto load_key = [&](int q) { return B.col[q]; };
    // [c0, c0 + span) by one unsigned compare; columns outside B never fall
    // in it and are flagged on the slow side
    auto mark = [&](int key, float) {
        const unsigned kk = (unsigned)key - (unsigned)c0;
        if (kk < (unsigned)span) atomicOr(&bm[kk >> 5], 1u << (kk & 31));
        else if (key_in(key, B, ctl)) set_status(ctl, ST_INTERNAL);
    };
    auto load = [&](int q) {
        const int2 v = bcv[q];
        return KeyVal{v.x, __int_as_float(v.y)};
    };
    auto add = [&](KeyVal kv, float a) {
        const unsigned kk = (unsigned)kv.key - (unsigned)c0;
        if (kk >= (unsigned)span) {
            key_in(kv.key, B, ctl);
            return;
        }
        const int w = (int)(kk >> 5);
        if ((unsigned)(w - lo) >= (unsigned)(hi - lo)) return;            // other word range
        const unsigned word = bm[w];
        const int r = rk[w] + __popc(word & ((1u << (kk & 31)) - 1u)) - rbase;
        // the column must be in the pass's bitmap (a cached bitmap that does
        // not match the operands is reported, not used)
        if ((unsigned)r < (unsigned)cap && ((word >> (kk & 31)) & 1u)) atomicAdd(&vals[r], a * kv.v);
        else set_status(ctl, ST_INTERNAL);
    };

    // thread 0 fetches the next row one row ahead (the pending atomic stays
    // in a register until the next row starts), so its latency hides behind
    // the current row
    int nxt_idx = 0;
    if (t == 0) nxt_idx = begin + atomicAdd(&ctl->work[tier], 1);
    bool dirty = false;              // bm holds words of an earlier pass
    for (;;) {
        if (t == 0) s_idx = nxt_idx;
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= end) break;
        if (t == 0) nxt_idx = begin + atomicAdd(&ctl->work[tier], 1);
        const int r = map[idx];
        const int row = row_begin + r;
        const int out = rptC[r];
        const int nnz_row = rptC[r + 1] - out;
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        const int na = re - rs;
        if (na > kRankTileE) continue;                // fallback kernel's row
        int cslot = rc_slot != nullptr ? rc_slot[row] : -1;
        if (cslot >= rc_nslots) {
            set_status(ctl, ST_INTERNAL);
            cslot = -1;
        }
        const unsigned* cbits = cslot >= 0 ? rc_bits + (size_t)cslot * rc_wpr : nullptr;
        const long long per_panel = ((long long)nnz_row + P - 1) / P;
        long long want = per_panel > 0 ? (95ll * cap / 100) / per_panel : pmax;
        const int ppp = (int)(want < 1 ? 1 : (want > pmax ? pmax : want));
        const int npass = (P + ppp - 1) / ppp;
        int myk = -1, cur = 0, nxt = 0;
        float mya = 0.f;
        if (t < na) {
            const int j = rs + t;
            const int k = A.col[j];
            if ((unsigned)k < (unsigned)B.rows) {
                myk = k;
                mya = A.val[j];
                cur = tab[(long long)k * stride];
                nxt = tab[(long long)k * stride + (ppp < P ? ppp : P)];
            } else {
                set_status(ctl, ST_INVALID);
            }
        }
        int written = 0;
        for (int pass = 0; pass < npass; ++pass) {
            const int p0 = pass * ppp;
            const int p1 = p0 + ppp < P ? p0 + ppp : P;
            c0 = p0 * PW;
            span = (int)(B.cols - (long long)c0 < (long long)(p1 - p0) * PW ? B.cols - (long long)c0
                                                                            : (long long)(p1 - p0) * PW);
            int nxt2 = 0;
            if (myk >= 0 && pass + 1 < npass)
                nxt2 = tab[(long long)myk * stride + (p1 + ppp < P ? p1 + ppp : P)];
            int bs = 0, len = 0;
            if (myk >= 0) {
                if (cur < 0 || nxt < cur || (long long)nxt > B.nnz) set_status(ctl, ST_INTERNAL);
                else {
                    bs = cur;
                    len = nxt - cur;
                }
            }
            // 1. occupancy (c0 is a multiple of the panel width, so of 32):
            // thread t holds words [wb, wb + wpt) of the pass in registers,
            // loaded from the cached bitmap or read after the marks
            const int nw = (span + 31) >> 5;
            const int wpt = (nw + kT - 1) / kT;
            const int wb = t * wpt;
            int cnt = 0;
            if (cbits != nullptr) {
                const unsigned* src = cbits + (c0 >> 5);
                for (int q = 0; q < wpt; ++q)
                    if (wb + q < nw) {
                        const unsigned v = src[wb + q];
                        bm[wb + q] = v;
                        cnt += __popc(v);
                    }
            } else {
                if (dirty) {                          // marks need a clear bitmap
                    for (int i = t; i < nw; i += kT) bm[i] = 0u;
                    __syncthreads();
                }
                expand_tile_padded<kT, float, kRankOccUnroll>(tile, bs, len, mya, load_key, mark);
                for (int q = 0; q < wpt; ++q)
                    if (wb + q < nw) cnt += __popc(bm[wb + q]);
            }
            dirty = true;
            // 2. word ranks, and the columns of ranks below cap staged at
            // their ranks in the value array (stored to C coalesced below);
            // a thread reads back only the words it wrote
            int tot;
            int run = block_excl_scan(cnt, scratch, &tot);
            int* stage = reinterpret_cast<int*>(vals);
            if (tot <= cap) {
                stage_pairs(bm, rk, stage, wb, wpt, nw, run, c0);
            } else {                                  // ranks past cap staged per range below
                for (int q = 0; q < wpt; ++q) {
                    const int w = wb + q;
                    if (w >= nw) break;
                    rk[w] = run;
                    unsigned bits = bm[w];
                    while (bits) {
                        if ((unsigned)run < (unsigned)cap) stage[run] = c0 + w * 32 + __ffs(bits) - 1;
                        bits &= bits - 1;
                        ++run;
                    }
                }
            }
            __syncthreads();
            // 3. values, in word ranges of at most cap entries
            for (lo = 0; lo < nw; lo = hi) {
                if (t == 0) {
                    const int base_lo = rk[lo];
                    int h;
                    if (tot - base_lo <= cap) {
                        h = nw;
                    } else {                          // largest h with rank(h) - rank(lo) <= cap
                        int a = lo + 1, b = nw - 1;
                        while (a < b) {
                            const int mid = (a + b + 1) >> 1;
                            if (rk[mid] - base_lo <= cap) a = mid;
                            else b = mid - 1;
                        }
                        h = a;
                    }
                    s_hi = h;
                }
                __syncthreads();
                hi = s_hi;
                rbase = rk[lo];
                const int cnt_sub = (hi < nw ? rk[hi] : tot) - rbase;
                if (lo > 0) {                         // a later range: stage its columns now
                    for (int q = 0; q < wpt; ++q) {
                        const int w = wb + q;
                        if (w >= hi) break;
                        if (w < lo) continue;
                        unsigned bits = bm[w];
                        int rr = rk[w] - rbase;
                        while (bits) {
                            if ((unsigned)rr < (unsigned)cap) stage[rr] = c0 + w * 32 + __ffs(bits) - 1;
                            bits &= bits - 1;
                            ++rr;
                        }
                    }
                    __syncthreads();
                }
                // the range's columns to C, coalesced; every staged slot is
                // cleared for the values (the expansion's block scan orders
                // the clears before any add)
                const int ncl = lo == 0 ? (tot < cap ? tot : cap) : cnt_sub;
                for (int i = t; i < ncl; i += kT) {
                    const int o = written + rbase + i;
                    if (i < cnt_sub && o < nnz_row) colC[out + o] = stage[i];
                    vals[i] = 0.f;
                }
                expand_tile_padded<kT, float, kRankUnroll>(tile, bs, len, mya, load, add);
                for (int i = t; i < cnt_sub; i += kT) {
                    const int o = written + rbase + i;
                    if (o < nnz_row) valC[out + o] = vals[i];
                    vals[i] = 0.f;
                }
                __syncthreads();
            }
            written += tot;
            cur = nxt;
            nxt = nxt2;
        }
        if (t == 0 && written != nnz_row) set_status(ctl, ST_INTERNAL);
    }
}

// Heavy rows whose entries can gather more than fp32_max_terms products
// (the fp64 tier). Products on cold columns of B (see hot.cu) are summed in
// fp32 exactly as in the fp32 tier. Products on hot columns (one slot per
// hot column of the sub-pass) are split over kHotCopies fp32 partial sums
// by the rank of their A entry in the expansion tile (rank mod kHotCopies):
// with at most kHotThreads entries in a tile and each entry adding at most
// one product to a column (B rows sorted, no repeated column), a copy
// gathers at most kHotThreads / kHotCopies = 128 terms per column. A
// product reads B's column word (the column, or sign bit | hot rank for a
// hot column) beside its value. After every tile
// the copies are added, in a fixed order, into a double-float sum per slot
// (an fp32 pair kept exact by TwoSum) and cleared; at the end of the
// sub-pass the pair is rounded once into the pass array. The error stays
// within (gamma_128 + u) * sum|a||b| plus the pair's ~2^-44 relative
// rounding, below the 1e-5 bound, with fp32 arithmetic and shared-memory
// atomics only.
// When B has unsorted or repeated columns (ctl->b_unsorted != 0) the bound
// does not hold and hot-column products go straight to the fp64
// accumulator with fp64 atomics instead.
//
// A pass covers ppp table panels (as many as shared memory holds, set at
// launch); when it holds more hot columns than kHotSlots it is split into
// sub-passes at hot-column boundaries (re-reading its segments).
constexpr int kHotThreads = 1024;
constexpr int kHotUnroll = 4;      // products per warp step batch (2 and 8 measured slower)
constexpr int kHotSlots = 1024;
constexpr int kHotCopies = 8;
static_assert(kHotThreads / kHotCopies <= 160, "a copy must gather at most 160 terms per tile");

__global__ void __launch_bounds__(kHotThreads, 1) k_num_dense_hot(CsrDev A, CsrDev B,
                                                                  const int* map, Ctl* ctl,
                                                                  const int* rptC, int row_begin,
                                                                  int* colC, float* valC,
                                                                  int bin_lo, int bin_hi, int tier,
                                                                  const int* tab, int P, int PW,
                                                                  int ppp, const int* hot_rank,
                                                                  const int* hot_col,
                                                                  const int2* bhv,
                                                                  const int* rc_slot,
                                                                  const unsigned* rc_bits,
                                                                  int rc_nslots, int rc_wpr,
                                                                  int skip_cached) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int W = PW * ppp;                                           // columns per pass
    double* acc = reinterpret_cast<double*>(sm_raw);                  // [kHotSlots]
    float* cp = reinterpret_cast<float*>(acc + kHotSlots);            // [kHotCopies][kHotSlots]
    float* st = cp + kHotCopies * kHotSlots;                          // [W]
    unsigned* bm = reinterpret_cast<unsigned*>(st + W);               // [W / 32]
    __shared__ int s_idx;
    __shared__ int scratch[33];
    __shared__ unsigned touched[kHotSlots / 32];  // hot slots that received a product this sub-pass
    __shared__ ExpandTile<kHotThreads, float> tile;
    const int begin = ctl->bin_off[bin_lo], end = ctl->bin_off[bin_hi];
    if (begin >= end) return;
    // beside k_num_dense_hotr, only rows without a cached bitmap are this
    // kernel's; the grouping flags whether there are any
    if (skip_cached && ctl->dense_uncached == 0) return;
    const int t = threadIdx.x;
    const int nwords = W >> 5;
    for (int i = t; i < kHotSlots / 32; i += kHotThreads) touched[i] = 0u;
    for (int i = t; i < W; i += kHotThreads) st[i] = 0.f;
    for (int i = t; i < nwords; i += kHotThreads) bm[i] = 0u;
    for (int i = t; i < kHotSlots; i += kHotThreads) acc[i] = 0.0;
    for (int i = t; i < kHotCopies * kHotSlots; i += kHotThreads) cp[i] = 0.f;
    const bool use_tab = tab != nullptr && (ctl->b_unsorted & 1) == 0;
    const bool split = ctl->b_unsorted == 0;       // copies bound the terms per column
    const int npass = (P + ppp - 1) / ppp;
    const long long stride = P + 1;

    // pass start, sub-pass columns [lo, hi), its hot ranks [hr0, hr0 + nhs),
    // and the pass's hot ranks [hrp0, hrp1)
    int pc0 = 0, lo = 0, hi = 0, hr0 = 0, nhs = 0, hrp0 = 0, hrp1 = 0;
    // the row's cached column bitmap (allocation phase), or nullptr: with it
    // the sub-pass's bitmap words are copied in and products mark nothing
    const unsigned* cbits = nullptr;
    auto load = [&](int q) {
        const int2 v = bhv[q];
        return KeyVal{v.x, __int_as_float(v.y)};
    };
    // one bitmap OR and one fp32 add per product, hot or cold, on selected
    // addresses (a hot product marks its slot, a cold one its column), so the
    // warp does not diverge into two instruction sequences
    auto apply = [&](KeyVal kv, float a, int seg) {
        const int code = kv.key;
        const bool hot = code < 0;                   // (sign bit | hot rank)
        int x;                                       // hot slot or pass column
        if (hot) {
            const int rank = code & 0x7fffffff;
            x = rank - hr0;
            if ((unsigned)x >= (unsigned)nhs) {      // another sub-pass's column
                if (use_tab && (rank < hrp0 || rank >= hrp1)) set_status(ctl, ST_INTERNAL);
                return;
            }
        } else {
            // [lo, hi) by one unsigned compare; a column outside B never
            // falls in it and is flagged here
            if ((unsigned)code - (unsigned)lo >= (unsigned)(hi - lo)) {
                if (key_in(code, B, ctl) && use_tab && (code < pc0 || code >= pc0 + W))
                    set_status(ctl, ST_INTERNAL);
                return;
            }
            x = code - pc0;
        }
        if (cbits == nullptr) atomicOr((hot ? touched : bm) + (x >> 5), 1u << (x & 31));
        if (hot && !split) atomicAdd(&acc[x], (double)a * (double)kv.v);
        else atomicAdd(hot ? &cp[(seg & (kHotCopies - 1)) * kHotSlots + x] : &st[x], a * kv.v);
    };
    // add the copies of this sub-pass's hot slots into the slot sums: with
    // the copies (split) a double-float pair per slot, each copy added by
    // TwoSum in fp32 (GB300's fp64 pipe is slow; see k_num_dense_hotr);
    // without them the products went straight into the fp64 sum (acc)
    float2* acc2 = reinterpret_cast<float2*>(acc);
    auto fold = [&]() {
        if (split) {
            for (int h = t; h < nhs; h += kHotThreads) {
                float2 v = acc2[h];
#pragma unroll
                for (int c = 0; c < kHotCopies; ++c) {
                    const float x = cp[c * kHotSlots + h];
                    cp[c * kHotSlots + h] = 0.f;
                    const float sum = v.x + x;
                    const float bp = sum - v.x;
                    const float err = (v.x - (sum - bp)) + (x - bp);
                    v.x = sum;
                    v.y += err;
                }
                acc2[h] = v;
            }
        }
        __syncthreads();
    };

    for (;;) {
        if (t == 0) s_idx = begin + atomicAdd(&ctl->work[tier], 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= end) break;
        const int r = map[idx];
        const int row = row_begin + r;
        const int out = rptC[r];
        const int nnz_row = rptC[r + 1] - out;
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        const int na = re - rs;
        const bool cached = use_tab && na <= kHotThreads;
        {
            int cslot = rc_slot != nullptr ? rc_slot[row] : -1;
            if (cslot >= rc_nslots) {
                set_status(ctl, ST_INTERNAL);
                cslot = -1;
            }
            if (skip_cached && cslot >= 0) continue;          // k_num_dense_hotr's row
            cbits = cslot >= 0 ? rc_bits + (size_t)cslot * rc_wpr : nullptr;
        }
        int myk = -1, cur = 0, nxt = 0;
        float mya = 0.f;
        if (cached && t < na) {
            const int j = rs + t;
            const int k = A.col[j];
            if ((unsigned)k < (unsigned)B.rows) {
                myk = k;
                mya = A.val[j];
                cur = tab[(long long)k * stride];
                nxt = tab[(long long)k * stride + (ppp < P ? ppp : P)];
            } else {
                set_status(ctl, ST_INVALID);
            }
        }
        int written = 0;
        for (int pass = 0; pass < npass; ++pass) {
            pc0 = pass * W;
            const int pc1 = (int)(B.cols - (long long)pc0 < W ? B.cols : pc0 + W);
            const int p0 = pass * ppp;
            const int p1 = p0 + ppp < P ? p0 + ppp : P;
            int nxt2 = 0;
            if (cached && myk >= 0 && pass + 1 < npass)
                nxt2 = tab[(long long)myk * stride + (p1 + ppp < P ? p1 + ppp : P)];
            int bs = 0, len = 0;
            if (cached && myk >= 0) {
                if (cur < 0 || nxt < cur || (long long)nxt > B.nnz) set_status(ctl, ST_INTERNAL);
                else {
                    bs = cur;
                    len = nxt - cur;
                }
            }
            hrp0 = hot_rank[pc0];
            hrp1 = hot_rank[pc1];
            // sub-passes of at most kHotSlots hot columns
            for (lo = pc0; lo < pc1; lo = hi) {
                hr0 = hot_rank[lo];
                hi = hrp1 - hr0 <= kHotSlots ? pc1 : hot_col[hr0 + kHotSlots];
                if (hi <= lo || hi > pc1) {              // defensive: malformed hot data
                    set_status(ctl, ST_INTERNAL);
                    hi = pc1;
                }
                nhs = hot_rank[hi] - hr0;
                if (nhs < 0 || nhs > kHotSlots) {        // defensive: malformed hot data
                    set_status(ctl, ST_INTERNAL);
                    nhs = nhs < 0 ? 0 : kHotSlots;
                }
                if (cbits != nullptr) {
                    // the sub-pass's columns [lo, hi) of the cached bitmap (words
                    // outside it stay clear); the expansion's block scan orders
                    // these stores before any product reads them
                    const int w0 = (lo - pc0) >> 5, w1 = (hi - pc0 + 31) >> 5;
                    for (int q = w0 + t; q < w1; q += kHotThreads) {
                        unsigned v = cbits[(pc0 >> 5) + q];
                        if (q == w0) v &= ~0u << ((lo - pc0) & 31);
                        if (q == w1 - 1 && ((hi - pc0) & 31)) v &= (1u << ((hi - pc0) & 31)) - 1u;
                        bm[q] = v;
                    }
                }
                if (cached) {
                    // packed expansion: this tier's per-pass segments are often short
                    expand_tile<kHotThreads, float, kHotUnroll, true>(tile, bs, len, mya, load,
                                                                      apply);
                    fold();
                } else {
                    for (int tb = rs; tb < re; tb += kHotThreads) {
                        const int j = tb + t;
                        int tbs = 0, tlen = 0;
                        float a = 0.f;
                        if (j < re) {
                            a_entry(A, B, j, tbs, tlen, ctl);
                            a = A.val[j];
                            if (use_tab && tlen > 0) {
                                const int* tk = tab + (long long)A.col[j] * stride;
                                const int ps = tk[p0], pe = tk[p1];
                                if (ps >= tbs && pe >= ps && pe <= tbs + tlen) {
                                    tbs = ps;
                                    tlen = pe - ps;
                                } else {
                                    set_status(ctl, ST_INTERNAL);
                                    tlen = 0;
                                }
                            }
                        }
                        expand_tile<kHotThreads, float, kHotUnroll, true>(tile, tbs, tlen, a, load,
                                                                          apply);
                        fold();
                    }
                }
                // round the hot columns' sums once into the pass array and mark
                // the hot columns that received a product in the bitmap
                for (int h = t; h < nhs; h += kHotThreads) {
                    const int kk = hot_col[hr0 + h] - pc0;
                    if ((unsigned)kk < (unsigned)W) {
                        st[kk] = split ? acc2[h].x + acc2[h].y : (float)acc[h];
                        if (cbits == nullptr && ((touched[h >> 5] >> (h & 31)) & 1u))
                            atomicOr(&bm[kk >> 5], 1u << (kk & 31));
                    }
                    acc[h] = 0.0;
                }
                __syncthreads();
                // (emit_bitmap synchronises before the next sub-pass's products)
                if (t < kHotSlots / 32) touched[t] = 0u;
                // emit [lo, hi) in column order (bits outside it are clear)
                written += emit_bitmap<kHotThreads>(
                    bm, (lo - pc0) >> 5, (hi - pc0 + 31) >> 5, pc0, colC, valC, out, written,
                    nnz_row, scratch, [&](int kk) {
                        const float v = st[kk];
                        st[kk] = 0.f;
                        return v;
                    });
            }
            cur = nxt;
            nxt = nxt2;
        }
        if (t == 0 && written != nnz_row) set_status(ctl, ST_INTERNAL);
    }
}

// fp64-bound dense tier with rank-compacted passes, for rows whose column
// bitmap the allocation phase cached (rows without a slot stay with
// k_num_dense_hot). With the row's columns known, a pass no longer needs a
// dense value array over its columns: each bitmap word gets the rank of its
// first entry, every product of a cold column adds into a compact value
// array at its entry's rank (word rank + popcount of the lower bits), and a
// pass is as wide as its entries allow (up to `cap` entries and
// kHotrSlots hot columns; ~4 table panels on R-MAT hub rows instead of 2),
// so a row takes about half as many passes, each with longer B segments.
// Hot columns keep the partial-sum scheme of k_num_dense_hot (kHotCopies
// fp32 copies by the product's A-entry rank, folded into fp64 after every
// tile, rounded once), with kHotrSlots slots and the copies padded apart in
// shared memory. A pass with more hot columns than slots (only where hot
// columns cluster inside one panel) is walked once per slot range, cold
// products being added in the first walk only.
//
// Work items are (row, split): the row's table panels are cut into `splits`
// consecutive column ranges, each taken by whichever block draws it, so one
// heavy row runs on several SMs at once. A range writes its columns and
// values at the row's output offset plus the entries of the earlier ranges
// (popcounts of the cached bitmap), so the pieces need no merge step: they
// are column-disjoint and already in order.
// Column ranges per row when opts.dense_splits is 0: by the row's bin q
// (bins of the fp64 tier hold rows with IP in (2^(45-q), 2^(46-q)]): one
// range per 128K intermediate products, at most 8 and at most one per panel.
// (On the R-MAT scale 20 product, whose tier rows hold 1M-22M products, 8
// ranges for every row measured best: 1 / 4 / 8 / 16 / 32 ranges gave 410 /
// 262 / 249 / 252 / 269 ms; one range per 2M products gave 301 ms.)
__device__ __forceinline__ int auto_splits(int q, int P) {
    const int L = 46 - q;                     // IP <= 2^L
    const int sp = L >= 20 ? 8 : (L > 17 ? 1 << (L - 17) : 1);
    return sp < P ? sp : (P > 0 ? P : 1);
}

// hot-column slots and value slots of a pass: 2048 / 20480, 1792 / 22528,
// 1536 / 24576, 1024 / 28672 -> 211.3 / 206.5 / 204.7 / 222.1 ms (fewer
// slots leave room for more values; too few cut passes at hot columns)
constexpr int kHotrSlots = 1536;
constexpr int kHotrCap = 24576;
constexpr int kHotrStride = kHotrSlots + 1;   // copies of one slot in different banks
// threads per block and products per warp step batch: with 1024 threads
// (64 registers), unroll 2 / 3 / 4 measured 219.2 / 211.7 / 231.0 ms on the
// R-MAT scale 20 product (earlier forms: 254 / 248 / 268 ms); 768 x 4 /
// 512 x 6 / 512 x 8 (more registers, fewer warps) 273 / 316 / 324 ms
#ifndef SPG_HOTR_THREADS
#define SPG_HOTR_THREADS 1024
#endif
#ifndef SPG_HOTR_UNROLL
#define SPG_HOTR_UNROLL 3
#endif
constexpr int kHotrThreads = SPG_HOTR_THREADS;
constexpr int kHotrUnroll = SPG_HOTR_UNROLL;
static_assert(kHotrThreads / kHotCopies <= 160, "a copy must gather at most 160 terms per tile");

__global__ void __launch_bounds__(kHotrThreads, 1) k_num_dense_hotr(
    CsrDev A, CsrDev B, const int* map, Ctl* ctl, const int* rptC, int row_begin, int* colC,
    float* valC, int bin_lo, int bin_hi, int tier, const int* tab, int P, int PW, int pmax,
    int cap, const int* hot_rank, const int* hot_col, const int2* bhv, const int* rc_slot,
    const unsigned* rc_bits, const int* rc_pc, int rc_nslots, int rc_wpr, int splits) {
    constexpr int kT = kHotrThreads;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double* acc = reinterpret_cast<double*>(sm_raw);                  // [kHotrSlots]
    float* cp = reinterpret_cast<float*>(acc + kHotrSlots);           // [kHotCopies][kHotrStride]
    float* vals = cp + kHotCopies * kHotrStride;                      // [cap]
    unsigned* bm = reinterpret_cast<unsigned*>(vals + cap);           // [pmax * PW / 32]
    int* rk = reinterpret_cast<int*>(bm + ((pmax * PW) >> 5));        // [pmax * PW / 32]
    __shared__ int s_idx, s_g, s_S, s_p1;
    __shared__ int scratch[33];
    __shared__ int s_pc[kMaxPanels];    // entries of the item's panels
    __shared__ int s_ph[kMaxPanels];    // hot columns of the item's panels
    __shared__ ExpandTile<kT, float> tile;
    const int begin = ctl->bin_off[bin_lo], end = ctl->bin_off[bin_hi];
    if (begin >= end) return;
    if (tab == nullptr || (ctl->b_unsorted & 1) != 0 || rc_slot == nullptr || rc_pc == nullptr) return;
    const int t = threadIdx.x;
    for (int i = t; i < kHotrSlots; i += kT) acc[i] = 0.0;
    for (int i = t; i < kHotCopies * kHotrStride; i += kT) cp[i] = 0.f;
    for (int i = t; i < cap; i += kT) vals[i] = 0.f;
    const bool split = ctl->b_unsorted == 0;       // copies bound the terms per column
    const long long stride = P + 1;

    // pass start c0 and width span, hot ranks of this walk [hr0, hr0 + nhs),
    // of the pass [hrp0, hrp1); cold: this walk adds cold products
    int c0 = 0, span = 0, hr0 = 0, nhs = 0, hrp0 = 0, hrp1 = 0;
    bool cold = true;
    auto load = [&](int q) {
        const int2 v = bhv[q];
        return KeyVal{v.x, __int_as_float(v.y)};
    };
    // one instruction sequence for hot and cold products: both compute a
    // cold rank (a hot one on word 0) and add once at a selected address
    auto apply = [&](KeyVal kv, float a, int seg) {
        const int code = kv.key;
        const bool hot = code < 0;                             // (sign bit | hot rank)
        const int x = hot ? (code & 0x7fffffff) - hr0 : code - c0;
        const bool ok = hot ? (unsigned)x < (unsigned)nhs : (cold && (unsigned)x < (unsigned)span);
        const unsigned kk = (!hot && ok) ? (unsigned)x : 0u;
        const unsigned word = bm[kk >> 5];
        const int r = rk[kk >> 5] + __popc(word & ((1u << (kk & 31)) - 1u));
        if (ok) {
            if (!hot && (!((word >> (kk & 31)) & 1u) || (unsigned)r >= (unsigned)cap))
                set_status(ctl, ST_INTERNAL);                                  // not in C's row
            else if (hot && !split) atomicAdd(&acc[x], (double)a * (double)kv.v);
            else atomicAdd(hot ? &cp[(seg & (kHotCopies - 1)) * kHotrStride + x] : &vals[r], a * kv.v);
        } else if (hot) {
            const int rank = code & 0x7fffffff;
            if (rank < hrp0 || rank >= hrp1) set_status(ctl, ST_INTERNAL);    // outside the pass
        } else if (cold && key_in(code, B, ctl)) {
            set_status(ctl, ST_INTERNAL);                                      // outside the pass
        }
    };
    // the copies of this walk's slots into the slot sums. With the copies
    // (split), a slot sum is a double-float pair (hi, lo) in the slot's 8
    // bytes, each copy added exactly by Knuth's TwoSum (the rounding error of
    // hi + x recovered in fp32 and carried in lo): fp32 work only, since
    // GB300's fp64 pipe runs at 1/64 of its fp32 rate; the pair holds the sum
    // to about 2^-44 of its terms' magnitude, far inside the bound. Without
    // the copies the products went straight into an fp64 sum (acc).
    float2* acc2 = reinterpret_cast<float2*>(acc);
    auto fold = [&]() {
        if (split) {
            for (int h = t; h < nhs; h += kT) {
                float2 v = acc2[h];
#pragma unroll
                for (int c = 0; c < kHotCopies; ++c) {
                    const float x = cp[c * kHotrStride + h];
                    cp[c * kHotrStride + h] = 0.f;
                    const float sum = v.x + x;
                    const float bp = sum - v.x;
                    const float err = (v.x - (sum - bp)) + (x - bp);
                    v.x = sum;
                    v.y += err;
                }
                acc2[h] = v;
            }
        }
        __syncthreads();
    };

    for (;;) {
        if (t == 0) {
            // item -> (bin, row of the bin, column range); bins are heaviest first
            long long item = atomicAdd(&ctl->work[tier], 1);
            int idx = end, g = 0, S = 1;
            for (int b = bin_lo; b < bin_hi; ++b) {
                const int n = ctl->bin_off[b + 1] - ctl->bin_off[b];
                const int sb = splits > 0 ? splits : auto_splits(b - bin_lo, P);
                if (item < (long long)n * sb) {
                    idx = ctl->bin_off[b] + (int)(item / sb);
                    g = (int)(item % sb);
                    S = sb;
                    break;
                }
                item -= (long long)n * sb;
            }
            s_idx = idx;
            s_g = g;
            s_S = S;
        }
        __syncthreads();
        const int idx = s_idx, g = s_g, splits_row = s_S;
        __syncthreads();
        if (idx >= end) break;
        const int r = map[idx];
        const int row = row_begin + r;
        const int out = rptC[r];
        const int nnz_row = rptC[r + 1] - out;
        const int cslot = rc_slot[row];
        if (cslot < 0 || cslot >= rc_nslots) continue;     // k_num_dense_hot's row
        const unsigned* cbits = rc_bits + (size_t)cslot * rc_wpr;
        const int gp0 = (int)((long long)P * g / splits_row);
        const int gp1 = (int)((long long)P * (g + 1) / splits_row);
        if (gp0 >= gp1) continue;
        int rs, re;
        row_extent(A, row, rs, re, ctl);
        const int na = re - rs;
        const bool cached = na <= kT;
        // entries per panel (counted by the allocation phase beside the
        // cached bitmap) and hot columns per panel for this item's panels;
        // entries before them = its offset
        int before = 0;
        const int* pcr = rc_pc + (size_t)cslot * P;
        for (int p = t; p < gp1; p += kT) {
            const int c = pcr[p];
            if (p >= gp0) {
                const long long cA = (long long)p * PW;
                const long long cB = cA + PW < B.cols ? cA + PW : B.cols;
                s_pc[p - gp0] = c;
                s_ph[p - gp0] = hot_rank[cB] - hot_rank[cA];
            } else {
                before += c;
            }
        }
        int pass_base = block_sum(before, scratch);                   // (barrier: s_pc, s_ph ready)
        int myk = -1, cur = 0;
        float mya = 0.f;
        if (cached && t < na) {
            const int j = rs + t;
            const int k = A.col[j];
            if ((unsigned)k < (unsigned)B.rows) {
                myk = k;
                mya = A.val[j];
                cur = tab[(long long)k * stride + gp0];
            } else {
                set_status(ctl, ST_INVALID);
            }
        }
        const int item_base = pass_base;
        for (int p0 = gp0; p0 < gp1;) {
            if (t == 0) {                    // widest pass within cap entries and the hot slots
                int p1 = p0, ent = 0, hot = 0;
                while (p1 < gp1 && p1 - p0 < pmax) {
                    const int c = s_pc[p1 - gp0], h = s_ph[p1 - gp0];
                    if (p1 > p0 && (ent + c > cap || hot + h > kHotrSlots)) break;
                    ent += c;
                    hot += h;
                    ++p1;
                }
                s_p1 = p1;
            }
            __syncthreads();
            const int p1 = s_p1;
            c0 = p0 * PW;
            span = (int)((long long)p1 * PW < B.cols ? (long long)p1 * PW - c0 : B.cols - (long long)c0);
            const int nw = (span + 31) >> 5;
            int bs = 0, len = 0;
            if (myk >= 0) {
                const int nxt = tab[(long long)myk * stride + p1];
                if (cur < 0 || nxt < cur || (long long)nxt > B.nnz) set_status(ctl, ST_INTERNAL);
                else {
                    bs = cur;
                    len = nxt - cur;
                }
                cur = nxt;
            }
            // the pass's bitmap words, their ranks and the pass's columns
            // (thread t owns words [wb, wb + wpt))
            const unsigned* src = cbits + (c0 >> 5);
            const int wpt = (nw + kT - 1) / kT;
            const int wb = t * wpt;
            int cnt = 0;
            for (int q = 0; q < wpt; ++q)
                if (wb + q < nw) {
                    const unsigned v = src[wb + q];
                    bm[wb + q] = v;
                    cnt += __popc(v);
                }
            int tot;
            int run = block_excl_scan(cnt, scratch, &tot);
            if (tot > cap) set_status(ctl, ST_INTERNAL);          // cannot happen: cap >= panel width
            // the pass's columns go through the value array: each thread
            // writes its words' columns at their ranks, then the block stores
            // them to C coalesced and clears the array
            int* stage = reinterpret_cast<int*>(vals);
            for (int q = 0; q < wpt; ++q) {
                const int w = wb + q;
                if (w >= nw) break;
                rk[w] = run;
                unsigned bits = bm[w];
                while (bits) {
                    if ((unsigned)run < (unsigned)cap) stage[run] = c0 + w * 32 + __ffs(bits) - 1;
                    bits &= bits - 1;
                    ++run;
                }
            }
            __syncthreads();
            for (int i = t; i < tot && i < cap; i += kT) {
                const int o = pass_base + i;
                if (o < nnz_row) colC[out + o] = stage[i];
                vals[i] = 0.f;
            }
            // (the expansion's block scan orders bm / rk before any product)
            hrp0 = hot_rank[c0];
            hrp1 = hot_rank[c0 + span];
            for (int sub = 0, h0 = hrp0; sub == 0 || h0 < hrp1; ++sub, h0 += nhs) {
                hr0 = h0;
                nhs = hrp1 - h0 < kHotrSlots ? hrp1 - h0 : kHotrSlots;
                cold = sub == 0;
                if (cached) {
                    expand_tile<kT, float, kHotrUnroll, true>(tile, bs, len, mya, load, apply);
                    fold();
                } else {
                    for (int tb = rs; tb < re; tb += kT) {
                        const int j = tb + t;
                        int tbs = 0, tlen = 0;
                        float a = 0.f;
                        if (j < re) {
                            // the pass's segment straight from the panel table
                            // (two dependent loads: the entry, then its offsets)
                            const int k = A.col[j];
                            a = A.val[j];
                            if ((unsigned)k < (unsigned)B.rows) {
                                const int* tk = tab + (long long)k * stride;
                                const int ps = tk[p0], pe = tk[p1];
                                if (ps >= 0 && pe >= ps && (long long)pe <= B.nnz) {
                                    tbs = ps;
                                    tlen = pe - ps;
                                } else {
                                    set_status(ctl, ST_INTERNAL);
                                }
                            } else {
                                set_status(ctl, ST_INVALID);
                            }
                        }
                        expand_tile<kT, float, kHotrUnroll, true>(tile, tbs, tlen, a, load, apply);
                        fold();
                    }
                }
                // round the slot range's sums once into the value array
                for (int h = t; h < nhs; h += kT) {
                    const int kk = hot_col[hr0 + h] - c0;
                    float v;
                    if (split) {
                        const float2 p2 = acc2[h];
                        v = p2.x + p2.y;                 // one rounding of the pair
                        acc2[h] = make_float2(0.f, 0.f);
                    } else {
                        v = (float)acc[h];
                        acc[h] = 0.0;
                    }
                    if ((unsigned)kk < (unsigned)span) {
                        const unsigned word = bm[kk >> 5];
                        const int rr = rk[kk >> 5] + __popc(word & ((1u << (kk & 31)) - 1u));
                        if (((word >> (kk & 31)) & 1u) && (unsigned)rr < (unsigned)cap)
                            vals[rr] = v;
                        else if (v != 0.f)
                            set_status(ctl, ST_INTERNAL);
                    } else {
                        set_status(ctl, ST_INTERNAL);
                    }
                }
                __syncthreads();
            }
            for (int i = t; i < tot && i < cap; i += kT) {
                const int o = pass_base + i;
                if (o < nnz_row) valC[out + o] = vals[i];
                vals[i] = 0.f;
            }
            __syncthreads();
            pass_base += tot;
            p0 = p1;
        }
        if (t == 0) {
            int want = 0;
            for (int p = gp0; p < gp1; ++p) want += s_pc[p - gp0];
            if (pass_base - item_base != want || (splits_row == 1 && pass_base != nnz_row))
                set_status(ctl, ST_INTERNAL);
        }
        __syncthreads();
    }
}

// shared memory of the fp64 tier for ppp panels of pw columns per pass
constexpr size_t hot_smem_of(int pw, int ppp) {
    return (sizeof(double) + sizeof(float) * kHotCopies) * kHotSlots + 4 * (size_t)pw * ppp +
           (size_t)pw * ppp / 8;
}

// ---------------------------------------------------------------------------

static size_t num_warp_smem(size_t acc) { return (acc + 4) * kWarpsPerBlockNW * kWarpTableNum; }
static size_t num_block_smem(const spgemm_plan* p, size_t acc) {
    return (acc + 4) * pow2_ceil(2u * (unsigned)p->opts.block_max_nnz);
}
static size_t num_block_smem_small(const spgemm_plan* p, size_t acc) {
    const unsigned n = (unsigned)block_small_nnz(p->opts);
    return (acc + 4) * pow2_ceil(2u * (n > 32 ? n : 32));
}
static size_t num_block_smem_mid(const spgemm_plan* p, size_t acc) {
    const unsigned n = (unsigned)block_mid_nnz(p->opts);
    return (acc + 4) * pow2_ceil(2u * (n > 32 ? n : 32));
}
static int table_max_bits(size_t slots) {
    int b = 0;
    while (((size_t)1 << b) < slots) ++b;
    return b;
}
// rank-compacted fp32 dense kernel: bitmap + word ranks of pmax panels,
// then as many fp32 values as the rest holds (at most 32768, leaving L1
// some room)
static int rank_cap(const spgemm_plan* p, int pmax, int pw) {
    const size_t words = (size_t)pmax * pw / 32 * 8;
    const size_t left = p->rank_budget > words ? (p->rank_budget - words) / 4 : 0;
    return (int)(left > 32768 ? 32768 : left);
}
static size_t rank_smem(const spgemm_plan* p, int pmax, int pw) {
    return (size_t)pmax * pw / 32 * 8 + 4 * (size_t)rank_cap(p, pmax, pw);
}

static size_t num_dense_hot_smem(const spgemm_plan* p) {
    return hot_smem_of(p->opts.panel_cols, p->hot_ppp);
}

// rank-compacted fp64 tier: hot slots and copies, a value array of `cap`
// entries (at least one panel), bitmap words and word ranks of pmax panels
static size_t hotr_fixed() {
    return sizeof(double) * kHotrSlots + sizeof(float) * kHotCopies * kHotrStride;
}
static size_t hotr_smem(int pw, int pmax, int cap) {
    return hotr_fixed() + 4 * (size_t)cap + (size_t)pmax * (pw / 32) * 8;
}

// kMode 0: fp32 values and a bitmap over three table panels; kMode 1: fp64
// values, fp32 group sums and two bitmaps over one panel

static size_t num_dense_smem(const spgemm_plan* p, int mode) {
    const size_t W = (size_t)p->opts.panel_cols * (mode == 0 ? p->d32_ppp : 1);
    return mode == 0 ? 4 * W + W / 8 : 12 * W + W / 4;
}

void occupancy_numeric(spgemm_plan* p) {
    // fp64 dense tier: as many table panels per pass as the shared memory
    // left beside its static arrays holds
    {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, (const void*)k_num_dense_hot);
        const size_t fixed = hot_smem_of(p->opts.panel_cols, 0) + fa.sharedSizeBytes;
        const size_t per = hot_smem_of(p->opts.panel_cols, 1) - hot_smem_of(p->opts.panel_cols, 0);
        p->hot_ppp = p->smem_optin > fixed + per ? (int)((p->smem_optin - fixed) / per) : 1;
        if (p->hot_ppp > 64) p->hot_ppp = 64;
    }
    // fp32 dense tier: as many table panels per pass as a block's share of
    // the SM's shared memory holds beside its static arrays
    {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, (const void*)k_num_dense<0, kD32Threads>);
        int per_sm = 0, reserved = 0;
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, p->device);
        size_t avail = (size_t)per_sm / kD32Blocks;
        avail = avail > (size_t)reserved ? avail - reserved : 0;
        if (avail > p->smem_optin) avail = p->smem_optin;
        avail = avail > fa.sharedSizeBytes ? avail - fa.sharedSizeBytes : 0;
        const size_t per = 4 * (size_t)p->opts.panel_cols + p->opts.panel_cols / 8;
        p->d32_ppp = avail >= per ? (int)(avail / per) : 1;
        if (p->d32_ppp > 64) p->d32_ppp = 64;
    }
    {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, (const void*)k_num_dense_rank);
        int per_sm = 0, reserved = 0;
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device);
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, p->device);
        size_t avail = (size_t)per_sm / kRankBlocks;
        avail = avail > (size_t)reserved ? avail - reserved : 0;
        if (avail > p->smem_optin) avail = p->smem_optin;
        p->rank_budget = avail > fa.sharedSizeBytes ? avail - fa.sharedSizeBytes : 0;
    }
    // rank-compacted fp64 tier: kHotrCap value slots (at least one panel),
    // as many panels per pass as the rest of shared memory holds
    {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, (const void*)k_num_dense_hotr);
        const int pw = p->opts.panel_cols;
        const int cap = pw > kHotrCap ? pw : kHotrCap;
        const size_t budget = p->smem_optin > fa.sharedSizeBytes ? p->smem_optin - fa.sharedSizeBytes : 0;
        const size_t base = hotr_smem(pw, 0, cap), per = (size_t)(pw / 32) * 8;
        p->hotr_cap = cap;
        p->hotr_pmax = budget > base + per ? (int)((budget - base) / per) : 0;
        if (p->hotr_pmax > kMaxPanels) p->hotr_pmax = kMaxPanels;
        allow_max_dynamic_smem((const void*)k_num_dense_hotr, p);
    }
    struct K {
        const void* f;
        int threads;
        size_t smem;
        int* occ;
    } ks[] = {
        {(const void*)k_num_dense_rank, kRankThreads, rank_smem(p, kRankPanels, p->opts.panel_cols),
         &p->occ_num_rank},
        {(const void*)k_num_warp<float>, kWarpsPerBlockNW * 32, num_warp_smem(4), &p->occ_num_warp32},
        {(const void*)k_num_warp<double>, kWarpsPerBlockNW * 32, num_warp_smem(8), &p->occ_num_warp64},
        {(const void*)k_num_block<float, kBlockThreadsFull>, kBlockThreadsFull, num_block_smem(p, 4),
         &p->occ_num_block32},
        {(const void*)k_num_block<double, kBlockThreadsFull>, kBlockThreadsFull, num_block_smem(p, 8),
         &p->occ_num_block64},
        {(const void*)k_num_block<float>, kNumBlockThreads, num_block_smem_small(p, 4), &p->occ_num_block32s},
        {(const void*)k_num_block<double>, kNumBlockThreads, num_block_smem_small(p, 8), &p->occ_num_block64s},
        {(const void*)k_num_block<float>, kNumBlockThreads, num_block_smem_mid(p, 4), &p->occ_num_block32m},
        {(const void*)k_num_block<double>, kNumBlockThreads, num_block_smem_mid(p, 8), &p->occ_num_block64m},
        {(const void*)k_num_dense<0, kD32Threads>, kD32Threads, num_dense_smem(p, 0), &p->occ_num_dense32},
        {(const void*)k_num_dense<1, 1024>, 1024, num_dense_smem(p, 1), &p->occ_num_dense64},
        {(const void*)k_num_dense_hot, kHotThreads, num_dense_hot_smem(p), &p->occ_num_dense_hot},
    };
    allow_max_dynamic_smem((const void*)k_num_narrow<float>, p);
    allow_max_dynamic_smem((const void*)k_num_narrow<double>, p);
    for (auto& k : ks) {
        allow_max_dynamic_smem(k.f, p);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(k.occ, k.f, k.threads, k.smem);
        if (*k.occ < 1) *k.occ = 1;
    }
}

__global__ void k_reset_bflag(Ctl* ctl) { ctl->b_unsorted = 0; }

void launch_bpanel(const spgemm_plan* p, const CsrDev& B, const WsPtrs& w, cudaStream_t s) {
    SPG_LAUNCH(p, K_RESET, s, k_reset_bflag<<<1, 1, 0, s>>>(w.ctl));
    if (w.bpanel == nullptr || B.rows == 0) return;
    const long long warps = B.rows;
    long long blocks = (warps * 32 + 255) / 256;
    if (blocks > (long long)p->num_sms * 16) blocks = (long long)p->num_sms * 16;
    SPG_LAUNCH(p, K_BPANEL, s, k_bpanel<<<(int)blocks, 256, 0, s>>>(B, w.panels, w.panel_cols, w.bpanel, w.ctl));
}

// (column word, value) of every B entry packed into one 8-byte record per
// entry, so the dense tiers read a product's column and value with one
// vector load: bcv holds the column, bhv the column word of the fp64 tier
// (column, or sign bit | hot rank). Rebuilt by every accumulation call, so
// B's values may change between calls.
__global__ void k_pack_b(CsrDev B, const int* bhot, int2* bhv, int2* bcv) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < B.nnz;
         j += (long long)gridDim.x * blockDim.x) {
        const int v = __float_as_int(B.val[j]);
        bcv[j] = make_int2(B.col[j], v);
        bhv[j] = make_int2(bhot[j], v);
    }
}

// Output-capacity guard of the graph-capturable path: empties every bin
// when C does not fit (or its row pointers overflowed), so no tier writes.
__global__ void k_cap_guard(const int* rptC, int n, long long capacity, Ctl* ctl) {
    const bool bad = (ctl->status & ST_OVERFLOW) || (long long)rptC[n] > capacity || rptC[n] < 0;
    if (bad) {
        for (int b = threadIdx.x; b <= kNumBins; b += blockDim.x) ctl->bin_off[b] = 0;
        if (threadIdx.x == 0) set_status(ctl, ST_BUDGET);
    }
}

__global__ void k_copy_total(const Ctl* ctl, int which, long long* dst) { *dst = ctl->totals[which]; }

void launch_copy_total(const spgemm_plan* p, const WsPtrs& w, int which, long long* dst,
                       cudaStream_t s) {
    SPG_LAUNCH(p, K_GUARD, s, k_copy_total<<<1, 1, 0, s>>>(w.ctl, which, dst));
}

// Column ranges per row of the rank-compacted fp64 tier (work items per
// row): opts.dense_splits when set, else 0 (the kernel's per-bin choice).
static int dense_splits(const spgemm_plan* p, int panels) {
    int sp = p->opts.dense_splits;             // 0: chosen per row by the kernel
    if (sp > panels) sp = panels > 0 ? panels : 1;
    return sp;
}

void launch_numeric(const spgemm_plan* p, const CsrDev& A, const CsrDev& B, const long long* ip,
                    int row_begin, int row_end, const int* rptC, const WsPtrs& w, int* colC,
                    float* valC, cudaStream_t s, long long capacity) {
    GroupArgs g{};
    g.phase = 1;
    g.row_begin = row_begin;
    g.n = row_end - row_begin;
    g.ip = ip;
    g.rptA = A.rpt;
    g.rptC = rptC;
    g.bcols = B.cols;
    g.rc_slot = w.rc_slot;
    g.opts = p->opts;
    launch_group(p, g, w, w.map, nullptr, s);
    if (g.n == 0) return;
    if (capacity >= 0)
        SPG_LAUNCH(p, K_GUARD, s, k_cap_guard<<<1, 64, 0, s>>>(rptC, g.n, capacity, w.ctl));
    const int sms = p->num_sms;
    SPG_LAUNCH(p, K_NUM_ESC, s, k_num_esc<<<sms * 8, 256, 0, s>>>(A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_ESC));
    if (B.cols <= kNarrowCols) {
        const int pad = (B.cols + 31) & ~31;
        const int nwp = narrow_warps(p);
        const int grid = sms * (64 / nwp > 1 ? 64 / nwp : 1);
        SPG_LAUNCH(p, K_NUM_NARROW, s,
                   k_num_narrow<float><<<grid, nwp * 32, (size_t)nwp * (pad * 4 + 128), s>>>(
                       A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_NARROW32, pad));
        SPG_LAUNCH(p, K_NUM_NARROW, s,
                   k_num_narrow<double><<<grid, nwp * 32, (size_t)nwp * (pad * 8 + 128), s>>>(
                       A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_NARROW64, pad));
    }
    SPG_LAUNCH(p, K_NUM_WARP32, s,
               k_num_warp<float><<<sms * p->occ_num_warp32, kWarpsPerBlockNW * 32, num_warp_smem(4), s>>>(
                   A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_WARP32, hash_load(p)));
    SPG_LAUNCH(p, K_NUM_WARP64, s,
               k_num_warp<double><<<sms * p->occ_num_warp64, kWarpsPerBlockNW * 32, num_warp_smem(8), s>>>(
                   A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_WARP64, hash_load(p)));
    // block hash tier: rows of more than half of block_max_nnz entries with
    // the full table (one block per SM), the others with a half- or
    // quarter-size table and as many blocks per SM as it leaves room for
    const int max_bits = table_max_bits(num_block_smem(p, 4) / 8);
    const int mid_bits = table_max_bits(num_block_smem_mid(p, 4) / 8);
    const int small_bits = table_max_bits(num_block_smem_small(p, 4) / 8);
    SPG_LAUNCH(p, K_NUM_BLOCK32, s,
               k_num_block<float, kBlockThreadsFull><<<sms * p->occ_num_block32, kBlockThreadsFull,
                                                      num_block_smem(p, 4), s>>>(
                   A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_BLOCK32, 2, max_bits,
                   hash_load(p)));
    SPG_LAUNCH(p, K_NUM_BLOCK32, s,
               k_num_block<float><<<sms * p->occ_num_block32m, kNumBlockThreads, num_block_smem_mid(p, 4), s>>>(
                   A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_BLOCK32M, 10, mid_bits,
                   hash_load(p)));
    SPG_LAUNCH(p, K_NUM_BLOCK32, s,
               k_num_block<float><<<sms * p->occ_num_block32s, kNumBlockThreads, num_block_smem_small(p, 4), s>>>(
                   A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_BLOCK32S, 8, small_bits,
                   hash_load(p)));
    SPG_LAUNCH(p, K_NUM_BLOCK64, s,
               k_num_block<double, kBlockThreadsFull><<<sms * p->occ_num_block64, kBlockThreadsFull,
                                                       num_block_smem(p, 8), s>>>(
                   A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_BLOCK64, 3, max_bits,
                   hash_load(p)));
    SPG_LAUNCH(p, K_NUM_BLOCK64, s,
               k_num_block<double><<<sms * p->occ_num_block64m, kNumBlockThreads, num_block_smem_mid(p, 8), s>>>(
                   A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_BLOCK64M, 11, mid_bits,
                   hash_load(p)));
    SPG_LAUNCH(p, K_NUM_BLOCK64, s,
               k_num_block<double><<<sms * p->occ_num_block64s, kNumBlockThreads, num_block_smem_small(p, 8), s>>>(
                   A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_BLOCK64S, 9, small_bits,
                   hash_load(p)));
    const int PW = w.panel_cols;
    if (w.bhv && w.bpanel && B.nnz > 0)
        SPG_LAUNCH(p, K_HOT, s, k_pack_b<<<sms * 8, 256, 0, s>>>(B, w.bhot, w.bhv, w.bcv));
    const int pmax = w.panels < kRankPanels ? w.panels : kRankPanels;
    const int cap = w.bpanel ? rank_cap(p, pmax, PW) : 0;
    if (w.bpanel && cap >= 1024) {
        // rank-compacted passes for the rows it takes, then the dense-array
        // kernel for the rest (B unsorted, or more A entries than threads)
        SPG_LAUNCH(p, K_NUM_DENSE32, s,
                   k_num_dense_rank<<<sms * p->occ_num_rank, kRankThreads, rank_smem(p, pmax, PW), s>>>(
                       A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_DENSE32_0,
                       NB_DENSE32_0 + NB_DENSE_N, 4, w.bpanel, w.panels, PW, pmax, cap,
                       w.rc_slot, w.rc_bits, w.rc_nslots, w.rc_wpr, w.bcv));
        SPG_LAUNCH(p, K_NUM_DENSE32, s,
                   k_num_dense<0, kD32Threads><<<sms * p->occ_num_dense32, kD32Threads, num_dense_smem(p, 0), s>>>(
                       A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_DENSE32_0,
                       NB_DENSE32_0 + NB_DENSE_N, 6, w.bpanel, w.panels, PW, p->d32_ppp, kRankTileE));
    } else {
        SPG_LAUNCH(p, K_NUM_DENSE32, s,
                   k_num_dense<0, kD32Threads><<<sms * p->occ_num_dense32, kD32Threads, num_dense_smem(p, 0), s>>>(
                       A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_DENSE32_0,
                       NB_DENSE32_0 + NB_DENSE_N, 4, w.bpanel, w.panels, PW, p->d32_ppp, 0));
    }
    if (w.bhot && w.bpanel) {
        // rows with a cached bitmap: rank-compacted passes, split into
        // p->opts-independent column ranges per row (dense_splits)
        const bool hotr = w.rc_slot != nullptr && w.rc_pc != nullptr && p->hotr_pmax >= 1;
        if (hotr) {
            const int pmax_r = p->hotr_pmax < w.panels ? p->hotr_pmax : w.panels;
            const int splits = dense_splits(p, w.panels);
            SPG_LAUNCH(p, K_NUM_DENSE64, s,
                       k_num_dense_hotr<<<sms, kHotrThreads, hotr_smem(PW, pmax_r, p->hotr_cap), s>>>(
                           A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_DENSE64_0,
                           NB_DENSE64_0 + NB_DENSE_N, 7, w.bpanel, w.panels, PW, pmax_r,
                           p->hotr_cap, w.hot_rank, w.hot_col, w.bhv, w.rc_slot, w.rc_bits,
                           w.rc_pc, w.rc_nslots, w.rc_wpr, splits));
        }
        SPG_LAUNCH(p, K_NUM_DENSE64, s,
                   k_num_dense_hot<<<sms * p->occ_num_dense_hot, kHotThreads, num_dense_hot_smem(p), s>>>(
                       A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_DENSE64_0,
                       NB_DENSE64_0 + NB_DENSE_N, 5, w.bpanel, w.panels, PW, p->hot_ppp,
                       w.hot_rank, w.hot_col, w.bhv, w.rc_slot, w.rc_bits, w.rc_nslots,
                       w.rc_wpr, hotr ? 1 : 0));
        return;
    }
    SPG_LAUNCH(p, K_NUM_DENSE64, s,
               k_num_dense<1, 1024><<<sms * p->occ_num_dense64, 1024, num_dense_smem(p, 1), s>>>(
                   A, B, w.map, w.ctl, rptC, row_begin, colC, valC, NB_DENSE64_0,
                   NB_DENSE64_0 + NB_DENSE_N, 5, w.bpanel, w.panels, PW, 1, 0));
}

}  // namespace spg

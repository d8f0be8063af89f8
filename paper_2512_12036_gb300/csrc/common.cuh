// Device-side building blocks shared by the SpGEMM kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spg {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kNumBins = 64;
constexpr int kSkipBin = kNumBins - 1;
constexpr int kMaxTiers = 16;
constexpr int kEmpty = -1;            // empty hash slot (column indices are >= 0)

// Status bits recorded by kernels; the host maps them to SPGEMM_ERR_* codes.
enum : int {
    ST_INVALID = 1,    // an index or row pointer out of range
    ST_INTERNAL = 2,   // a capacity guard tripped (table full, count mismatch)
    ST_OVERFLOW = 4,   // a 32-bit result overflowed
    ST_TIMEOUT = 8,    // a bounded wait gave up
    ST_UNSUPPORTED = 16,
    ST_BUDGET = 32     // the result exceeds the caller's output capacity
};

// Control block at the start of every workspace (256-byte aligned).
struct Ctl {
    int status;
    int b_unsorted;             // bit 0: a row of B is not sorted by column;
                                // bit 1: a sorted row of B repeats a column
    int rc_used;                // row bitmap cache slots handed out
    int dense_wide;             // accumulation grouping: a row of the fp32 dense tier has
                                // more A entries than the rank-compacted kernel takes
    int dense_uncached;         // accumulation grouping: a row of the fp64-bound dense tier
                                // has no cached bitmap
    int pad0;
    long long totals[8];        // 0: IP total, 1: nnz total, 2: scan total
    int work[kMaxTiers];        // dynamic row counters of the block-per-row tiers
    int bin_off[kNumBins + 1];  // start of every bin in the row map
    int pad1[256 - 6 - 16 - kMaxTiers - (kNumBins + 1)];
};
static_assert(sizeof(Ctl) % 256 == 0, "Ctl must keep the following arrays aligned");

__device__ __forceinline__ void set_status(Ctl* c, int bits) { atomicOr(&c->status, bits); }

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

__device__ __forceinline__ long long warp_incl_scan64(long long v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Largest lane s with excl[s] <= p, where excl is non-decreasing across the
// warp and excl[0] = 0 <= p. All 32 lanes must call it.
__device__ __forceinline__ int warp_find_src(int excl, int p) {
    int s = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        int e = __shfl_sync(kFull, excl, s + step);
        if (e <= p) s += step;
    }
    return s;
}

__host__ __device__ __forceinline__ unsigned pow2_ceil(unsigned x) {
    if (x <= 1) return 1;
#ifdef __CUDA_ARCH__
    return 1u << (32 - __clz(x - 1));
#else
    unsigned r = 1;
    while (r < x) r <<= 1;
    return r;
#endif
}

__host__ __device__ __forceinline__ int log2_ceil_ll(long long x) {
    int l = 0;
    while ((1ll << l) < x) ++l;
    return l;
}

// Bits of a hash table for `keys` keys at a target load of load_pct percent:
// the smallest power of two 2^b >= keys * 100 / load_pct, b in [lo, hi].
__host__ __device__ __forceinline__ int table_bits(long long keys, int load_pct, int lo, int hi) {
    int b = lo;
    while (b < hi && (1ll << b) * load_pct < 100 * keys) ++b;
    return b;
}

// Multiplicative (Fibonacci) hashing into a power-of-two table of 2^bits
// slots: the top bits of key * floor(2^32 / golden ratio).
__device__ __forceinline__ unsigned hash_slot(int key, int bits) {
    return ((unsigned)key * 2654435769u) >> (32 - bits);
}

// Block-wide exclusive scan of one int per thread; returns the exclusive
// prefix and writes the block total to *total. `scratch` holds 33 ints.
__device__ __forceinline__ int block_excl_scan(int v, int* scratch, int* total) {
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    int incl = warp_incl_scan(v);
    if (lane == 31) scratch[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nwarps ? scratch[lane] : 0;
        int wi = warp_incl_scan(w);
        scratch[lane] = wi - w;
        if (lane == 31) scratch[32] = wi;
    }
    __syncthreads();
    int r = scratch[warp] + incl - v;
    *total = scratch[32];
    __syncthreads();
    return r;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* scratch) {
    const int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    T r = 0;
    if (warp == 0) {
        r = lane < nwarps ? scratch[lane] : T(0);
        r = warp_sum(r);
        if (lane == 0) scratch[32] = r;
    }
    __syncthreads();
    r = scratch[32];
    __syncthreads();
    return r;
}

// One radix-selection step, called by all 32 lanes of a warp: hist holds
// the 256 bins of the current digit (keys sharing the prefix found so far),
// `above` the keys known to be larger than that prefix. Returns in every
// lane the digit whose bin holds the k-th largest key and the count of keys
// above that bin. Lane l reads bins 8l .. 8l+7; a suffix sum over lanes
// gives each lane the keys above its bins.
__device__ __forceinline__ void radix_digit256(const int* hist, int above, int k, int& dig,
                                                int& run_at) {
    const int lane = lane_id();
    int c[8], tot = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        c[i] = hist[8 * lane + i];
        tot += c[i];
    }
    int hi_sum = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_down_sync(kFull, hi_sum, o);
        if (lane + o < 32) hi_sum += v;
    }
    int run = above + hi_sum - tot;
    int my_dig = -1, my_run = 0;
#pragma unroll
    for (int i = 7; i >= 0; --i) {
        if (my_dig < 0 && run < k && run + c[i] >= k) {
            my_dig = 8 * lane + i;
            my_run = run;
        }
        run += c[i];
    }
    // exactly one lane's bins hold the k-th largest key
    const unsigned who = __ballot_sync(kFull, my_dig >= 0);
    const int src = who ? __ffs(who) - 1 : 0;
    dig = __shfl_sync(kFull, my_dig, src);
    run_at = __shfl_sync(kFull, my_run, src);
    if (dig < 0) dig = 0;
}

// Operand views passed by value to kernels.
struct CsrDev {
    int rows, cols;
    long long nnz;
    const int* rpt;
    const int* col;
    const float* val;
};

// Row extent [s, e) with range checks; returns false (and flags) if broken.
__device__ __forceinline__ bool row_extent(const CsrDev& M, int r, int& s, int& e, Ctl* ctl) {
    s = M.rpt[r];
    e = M.rpt[r + 1];
    if (s < 0 || e < s || (long long)e > M.nnz) {
        set_status(ctl, ST_INVALID);
        s = e = 0;
        return false;
    }
    return true;
}

// For one stored entry j of A: the B row it selects, as [bs, bs+len), and a.
__device__ __forceinline__ void a_entry(const CsrDev& A, const CsrDev& B, int j, int& bs, int& len,
                                        Ctl* ctl) {
    const int k = A.col[j];
    bs = 0;
    len = 0;
    if ((unsigned)k >= (unsigned)B.rows) {
        set_status(ctl, ST_INVALID);
        return;
    }
    const int s = B.rpt[k];
    const int e = B.rpt[k + 1];
    if (s < 0 || e < s || (long long)e > B.nnz) {
        set_status(ctl, ST_INVALID);
        return;
    }
    bs = s;
    len = e - s;
}

// Long B rows: a chunk whose lengths may overflow an int32 prefix sum is
// walked one A entry at a time instead of through the flattened expansion.
constexpr int kLongRow = 1 << 25;

// Warp-cooperative expansion of the products of A entries [j0, j1): every
// lane gets a (product index) and the callback receives (t, a_index) where
// t indexes B's col/val and a_index the A entry. Chunks of 32 A entries are
// spread over all 32 lanes by a prefix sum of the selected B-row lengths, so
// short and long B rows both keep every lane busy and loads coalesce along
// each B row. The callback runs for valid products only, with all lanes of
// the warp converged around it except for the p < total predicate.
template <class F>
__device__ __forceinline__ void warp_expand(const CsrDev& A, const CsrDev& B, int j0, int j1,
                                            int jstride, Ctl* ctl, F&& f) {
    const int lane = lane_id();
    for (int base = j0; base < j1; base += jstride) {
        const int j = base + lane;
        int bs = 0, len = 0;
        if (j < j1) a_entry(A, B, j, bs, len, ctl);
        const bool huge = __any_sync(kFull, len >= kLongRow);
        if (huge) {
            for (int q = 0; q < 32; ++q) {
                const int qbs = __shfl_sync(kFull, bs, q);
                const int qlen = __shfl_sync(kFull, len, q);
                for (int t = lane; t < qlen; t += 32) f(qbs + t, base + q);
            }
            continue;
        }
        const int incl = warp_incl_scan(len);
        const int excl = incl - len;
        const int total = __shfl_sync(kFull, incl, 31);
        for (int p0 = 0; p0 < total; p0 += 32) {
            const int p = p0 + lane;
            const int s = warp_find_src(excl, p);
            const int sbs = __shfl_sync(kFull, bs, s);
            const int sex = __shfl_sync(kFull, excl, s);
            if (p < total) f(sbs + (p - sex), base + s);
        }
    }
}


// Block-wide exclusive scan of one 64-bit value per thread (scratch: 33 slots).
__device__ __forceinline__ unsigned long long block_excl_scan_u64(unsigned long long v,
                                                                  unsigned long long* scratch,
                                                                  unsigned long long* total) {
    const int lane = lane_id(), warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long n = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) scratch[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long wv = lane < nwarps ? scratch[lane] : 0ull;
        unsigned long long wi = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long n = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += n;
        }
        scratch[lane] = wi - wv;
        if (lane == 31) scratch[32] = wi;
    }
    __syncthreads();
    const unsigned long long r = scratch[warp] + incl - v;
    *total = scratch[32];
    __syncthreads();
    return r;
}

// Shared-memory staging for block_expand: one tile of up to kE A entries
// (non-empty segments) expanded by kT threads.
template <int kT, typename Acc, int kE = kT>
struct ExpandTile {
    long long off[kE + 1];        // exclusive prefix of segment lengths (non-empty entries)
    int bs[kE];                   // segment start in B
    int ln[kE];                   // segment length (padded expansion)
    Acc a[kE];                    // a_ik (accumulation phase only)
    unsigned long long scratch[33];
};

// Position (0..31) of the (k+1)-th set bit of w, k < popc(w): a binary
// search on the popcounts of the low halves.
__device__ __forceinline__ int select_bit(unsigned w, int k) {
    int bit = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int c = __popc(w & ((1u << s) - 1u));
        if (k >= c) {
            w >>= s;
            bit += s;
            k -= c;
        }
    }
    return bit;
}

// Block-wide ordered emit of an occupancy bitmap: the set bits of words
// [w0, w1) of bm (bit b of word w = column c0 + 32*w + b; bits outside the
// range to emit must be clear) become entries (column, take(32*w + b)) at
// positions written, written+1, ... of a row
// that starts at colC/valC + out and holds nnz_row entries. Each warp owns a
// contiguous run of words; a block scan of the warps' counts places the
// runs; inside a run, 32 words at a time, entry s of the group goes to lane
// s mod 32, which finds its word by a search on the warp prefix of the
// popcounts and its bit by select_bit, so the column and value stores of a
// warp are contiguous. take(kk) returns the value and clears its slot; the
// words are cleared. Returns the number of entries. scratch holds 33 ints;
// ends with a block barrier.
template <int kT, class Take>
__device__ __forceinline__ int emit_bitmap(unsigned* bm, int w0, int w1, int c0, int* colC,
                                           float* valC, long long out, int written,
                                           int nnz_row, int* scratch, Take&& take) {
    constexpr int kWarps = kT / 32;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const int nw = w1 - w0;
    const int per = (nw + kWarps - 1) / kWarps;
    const int ws = w0 + warp * per;
    const int we = ws + per < w1 ? ws + per : w1;
    int cnt = 0;
    for (int g = ws; g < we; g += 32) cnt += g + lane < we ? __popc(bm[g + lane]) : 0;
    cnt = warp_sum(cnt);
    if (lane == 0) scratch[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        const int v = lane < kWarps ? scratch[lane] : 0;
        const int inc = warp_incl_scan(v);
        __syncwarp();
        scratch[lane] = inc - v;
        if (lane == 31) scratch[32] = inc;
    }
    __syncthreads();
    int pos = written + scratch[warp];
    const int total = scratch[32];
    for (int g = ws; g < we; g += 32) {
        const unsigned word = g + lane < we ? bm[g + lane] : 0u;
        const int c = __popc(word);
        const int inc = warp_incl_scan(c);
        const int excl = inc - c;
        const int T = __shfl_sync(kFull, inc, 31);
        for (int r = 0; r < T; r += 32) {
            const int p = r + lane;
            const int src = warp_find_src(excl, p < T ? p : T - 1);
            const unsigned sw = __shfl_sync(kFull, word, src);
            const int se = __shfl_sync(kFull, excl, src);
            if (p < T) {
                const int kk = (g + src) * 32 + select_bit(sw, p - se);
                const float v = take(kk);
                const int o = pos + p;
                if (o < nnz_row) {
                    colC[out + o] = c0 + kk;
                    valC[out + o] = v;
                }
            }
        }
        if (g + lane < we) bm[g + lane] = 0u;
        pos += T;
    }
    __syncthreads();
    return total;
}

// Per-thread form of emit_bitmap for sparse bitmaps (a few bits per word):
// thread t owns consecutive words, a block scan of the popcounts places its
// entries and it writes them in column order. Fewer instructions than the
// warp-cooperative form when words hold few bits, at the price of scattered
// stores. Same arguments and result; ends with a block barrier.
template <int kT, class Take>
__device__ __forceinline__ int emit_bitmap_lanes(unsigned* bm, int w0, int w1, int c0, int* colC,
                                                 float* valC, long long out, int written,
                                                 int nnz_row, int* scratch, Take&& take) {
    const int wpt = (w1 - w0 + kT - 1) / kT;
    const int wb = w0 + (int)threadIdx.x * wpt;
    int cnt = 0;
    for (int q = 0; q < wpt; ++q)
        if (wb + q < w1) cnt += __popc(bm[wb + q]);
    int tot;
    int pos = written + block_excl_scan(cnt, scratch, &tot);
    for (int q = 0; q < wpt; ++q) {
        const int w = wb + q;
        if (w >= w1) break;
        unsigned bits = bm[w];
        while (bits) {
            const int kk = w * 32 + __ffs(bits) - 1;
            bits &= bits - 1;
            const float v = take(kk);
            if (pos < nnz_row) {
                colC[out + pos] = c0 + kk;
                valC[out + pos] = v;
            }
            ++pos;
        }
        bm[w] = 0u;
    }
    __syncthreads();
    return tot;
}

// The per-warp walk of expand_tile over the compacted segments (offsets
// off[0..nE], starts sbs[], multipliers sa[]). Off is int when the tile's
// total fits 31 bits (the common case; fewer instructions per step), else
// long long.
template <typename Off, int kWarps, typename Acc, int kUnroll, bool kSeg, class Load, class Apply>
__device__ __forceinline__ void expand_walk(const Off* off, const int* sbsv, const Acc* sav, int nE,
                                            Off P, Load& load, Apply& apply) {
    using Item = decltype(load(0));
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const Off per = ((P + Off(32) * kWarps - 1) / (Off(32) * kWarps)) * Off(32);
    Off base = (Off)warp * per;
    const Off wend = base + per < P ? base + per : P;
    if (base >= wend) return;
    // segment holding product `base`: largest e with off[e] <= base
    int lo = 0, hi = nE - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= base) lo = mid;
        else hi = mid - 1;
    }
    int s = lo;
    Off so = off[s], se = off[s + 1];
    int sbs = sbsv[s];
    Acc sa = sav[s];
    while (base < wend) {
        int tq[kUnroll];
        Acc aq[kUnroll];
        bool vq[kUnroll];
        int sq[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            vq[u] = false;
            tq[u] = 0;
            aq[u] = Acc(0);
            sq[u] = 0;
            if (base < wend) {                       // warp-uniform
                if (base + 32 <= se) {               // the 32 products lie in segment s
                    tq[u] = sbs + (int)(base - so) + lane;
                    aq[u] = sa;
                    sq[u] = s;
                    vq[u] = base + lane < wend;
                    base += 32;
                    if (base == se && s + 1 < nE) {
                        ++s;
                        so = se;
                        se = off[s + 1];
                        sbs = sbsv[s];
                        sa = sav[s];
                    }
                } else {
                    const int e = s + lane;
                    Off d = e <= nE ? off[e] - base : Off(1 << 30);
                    if (d > Off(1 << 30)) d = Off(1 << 30);
                    const int rel = (int)d;      // lane 0: <= 0, then non-decreasing
                    const int wbs = e < nE ? sbsv[e] : 0;
                    const Acc wa = e < nE ? sav[e] : Acc(0);
                    // segments are non-empty, so their starts inside the
                    // window are distinct: lane l's segment is the number
                    // of starts at or before position l
                    const unsigned starts =
                        __reduce_or_sync(kFull, rel > 0 && rel < 32 ? 1u << rel : 0u);
                    const int src = __popc(starts & ((2u << lane) - 1u));
                    tq[u] = __shfl_sync(kFull, wbs - rel, src) + lane;
                    aq[u] = __shfl_sync(kFull, wa, src);
                    sq[u] = s + src;
                    vq[u] = base + lane < wend;
                    // segment of base + 32
                    const int cnt = __popc(__ballot_sync(kFull, rel <= 32));
                    int ns = s + cnt - 1;
                    if (cnt == 32 && s + 32 <= nE && off[s + 32] <= base + 32) ns = s + 32;
                    s = ns < nE - 1 ? ns : nE - 1;
                    base += 32;
                    so = off[s];
                    se = off[s + 1];
                    sbs = sbsv[s];
                    sa = sav[s];
                }
            }
        }
        Item it[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (vq[u]) it[u] = load(tq[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (vq[u]) {
                if constexpr (kSeg) apply(it[u], aq[u], sq[u]);
                else apply(it[u], aq[u]);
            }
        }
    }
}

// Block-wide, load-balanced expansion of the products of one tile of A
// entries. Every thread of the block calls it with the B segment
// [bs, bs+len) and multiplier a of its own entry (len = 0: none). Empty
// segments are compacted away by a block scan and an exclusive prefix of
// the lengths is kept in shared memory. The tile's products are then cut
// into equal, 32-aligned ranges, one per warp, so every warp does the same
// work whatever the B-row lengths. A warp walks its range 32 products at a
// time: when the 32 fall inside one segment (the common case for long B
// rows) lane l simply takes position bs + offset + l; otherwise lanes find
// their segment in a 32-entry window of the prefix (segments are non-empty,
// so 32 products never span more than 32 of them). Loads coalesce along
// each segment. Products are handled kUnroll steps at a time: load(t) for
// all of them first (independent loads in flight), then apply(item, a) in
// order. With kSeg, apply(item, a, seg) also gets the product's segment
// index (its entry's rank among the tile's non-empty entries). Ends with a
// block barrier.
template <int kT, typename Acc, int kUnroll, bool kSeg = false, class Load, class Apply>
__device__ __forceinline__ void expand_tile(ExpandTile<kT, Acc>& sm, int bs, int len, Acc a,
                                            Load&& load, Apply&& apply) {
    const int tid = threadIdx.x;
    constexpr int kWarps = kT / 32;
    constexpr unsigned long long kMask48 = (1ull << 48) - 1ull;
    const unsigned long long v = len > 0 ? ((1ull << 48) | (unsigned long long)len) : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan_u64(v, sm.scratch, &tot);
    const int nE = (int)(tot >> 48);
    const long long P = (long long)(tot & kMask48);
    const bool narrow = P < (1ll << 30);             // block-uniform
    int* off32 = reinterpret_cast<int*>(sm.off);     // same storage, int view
    if (len > 0) {
        const int ci = (int)(ex >> 48);
        if (narrow) off32[ci] = (int)(ex & kMask48);
        else sm.off[ci] = (long long)(ex & kMask48);
        sm.bs[ci] = bs;
        sm.a[ci] = a;
    }
    if (tid == 0) {
        if (narrow) off32[nE] = (int)P;
        else sm.off[nE] = P;
    }
    __syncthreads();
    if (narrow)
        expand_walk<int, kWarps, Acc, kUnroll, kSeg>(off32, sm.bs, sm.a, nE, (int)P, load, apply);
    else
        expand_walk<long long, kWarps, Acc, kUnroll, kSeg>(sm.off, sm.bs, sm.a, nE, P, load, apply);
    __syncthreads();
}

// expand_tile with every segment padded to a multiple of 32 products in the
// flattened order: the warps' equal ranges are 32-aligned, so each 32-product
// step of a warp lies inside one segment and lane l takes position
// bs + offset + l when that is below the segment's length (lanes in the
// padding idle). Moving on to the next segment is a constant-time step and
// no step needs a segment search, which suits tiles whose segments are
// mostly long (in R-MAT heavy rows about 9 in 10 lanes stay busy). Same
// contract as expand_tile, including kSeg.
template <typename Off, int kWarps, typename Acc, int kUnroll, bool kSeg, class Load, class Apply>
__device__ __forceinline__ void expand_walk_padded(const Off* off, const int* sbsv, const int* slnv,
                                                   const Acc* sav, int nE, Off P, Load& load,
                                                   Apply& apply) {
    using Item = decltype(load(0));
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    const Off per = ((P / 32 + kWarps - 1) / kWarps) * 32;
    Off base = (Off)warp * per;
    const Off wend = base + per < P ? base + per : P;
    if (base >= wend) return;
    int lo = 0, hi = nE - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= base) lo = mid;
        else hi = mid - 1;
    }
    int s = lo;
    Off so = off[s], se = off[s + 1];
    int sbs = sbsv[s], sln = slnv[s];
    Acc sa = sav[s];
    while (base < wend) {
        int tq[kUnroll];
        Acc aq[kUnroll];
        bool vq[kUnroll];
        int sq[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            vq[u] = false;
            tq[u] = 0;
            aq[u] = Acc(0);
            sq[u] = 0;
            if (base < wend) {                       // warp-uniform
                if (base >= se) {                    // next segment (padded length >= 32)
                    ++s;
                    so = se;
                    se = off[s + 1];
                    sbs = sbsv[s];
                    sln = slnv[s];
                    sa = sav[s];
                }
                const int o = (int)(base - so) + lane;
                tq[u] = sbs + o;
                aq[u] = sa;
                sq[u] = s;
                vq[u] = o < sln;
                base += 32;
            }
        }
        Item it[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (vq[u]) it[u] = load(tq[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (vq[u]) {
                if constexpr (kSeg) apply(it[u], aq[u], sq[u]);
                else apply(it[u], aq[u]);
            }
        }
    }
}

// (A tile of kE < kT entries takes at most kE threads with len > 0; a
// caller that passes more gets no expansion.)
template <int kT, typename Acc, int kUnroll, bool kSeg = false, int kE, class Load, class Apply>
__device__ __forceinline__ void expand_tile_padded(ExpandTile<kT, Acc, kE>& sm, int bs, int len, Acc a,
                                                   Load&& load, Apply&& apply) {
    const int tid = threadIdx.x;
    constexpr int kWarps = kT / 32;
    constexpr unsigned long long kMask48 = (1ull << 48) - 1ull;
    const unsigned long long plen = (unsigned long long)(((long long)len + 31) & ~31ll);
    const unsigned long long v = len > 0 ? ((1ull << 48) | plen) : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan_u64(v, sm.scratch, &tot);
    const int nE = (int)(tot >> 48);
    const long long P = (long long)(tot & kMask48);    // a multiple of 32
    if (kE < kT && nE > kE) {                           // block-uniform
        __syncthreads();
        return;
    }
    if (len > 0) {
        const int ci = (int)(ex >> 48);
        sm.off[ci] = (long long)(ex & kMask48);
        sm.bs[ci] = bs;
        sm.ln[ci] = len;
        sm.a[ci] = a;
    }
    if (tid == 0) sm.off[nE] = P;
    __syncthreads();
    // one 64-bit walk: a second, 32-bit instantiation here pushed the fp32
    // dense kernel past 64 registers (spills, 16% slower)
    expand_walk_padded<long long, kWarps, Acc, kUnroll, kSeg>(sm.off, sm.bs, sm.ln, sm.a, nE, P,
                                                              load, apply);
    __syncthreads();
}

// expand_tile over A entries [j0, j1) in tiles of kT; seg(j, bs, len, a)
// gives the segment and multiplier of entry j.
template <int kT, typename Acc, int kUnroll, class Seg, class Load, class Apply>
__device__ __forceinline__ void block_expand(int j0, int j1, ExpandTile<kT, Acc>& sm, Seg&& seg,
                                             Load&& load, Apply&& apply) {
    for (int tb = j0; tb < j1; tb += kT) {
        const int j = tb + threadIdx.x;
        int bs = 0, len = 0;
        Acc a = Acc(0);
        if (j < j1) seg(j, bs, len, a);
        expand_tile<kT, Acc, kUnroll>(sm, bs, len, a, load, apply);
    }
}

}  // namespace spg

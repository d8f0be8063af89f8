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
    int pad0[2];
    long long totals[8];        // 0: IP total, 1: nnz total, 2: scan total
    int work[kMaxTiers];        // dynamic row counters of the block-per-row tiers
    int bin_off[kNumBins + 1];  // start of every bin in the row map
    int pad1[256 - 4 - 16 - kMaxTiers - (kNumBins + 1)];
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

// Shared-memory staging for block_expand: one tile of kT A entries.
template <int kT, typename Acc>
struct ExpandTile {
    long long off[kT + 1];        // exclusive prefix of segment lengths (non-empty entries)
    int bs[kT];                   // segment start in B
    Acc a[kT];                    // a_ik (accumulation phase only)
    unsigned long long scratch[33];
};

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
    using Item = decltype(load(0));
    const int tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    constexpr int kWarps = kT / 32;
    constexpr unsigned long long kMask48 = (1ull << 48) - 1ull;
    const unsigned long long v = len > 0 ? ((1ull << 48) | (unsigned long long)len) : 0ull;
    unsigned long long tot;
    const unsigned long long ex = block_excl_scan_u64(v, sm.scratch, &tot);
    if (len > 0) {
        const int ci = (int)(ex >> 48);
        sm.off[ci] = (long long)(ex & kMask48);
        sm.bs[ci] = bs;
        sm.a[ci] = a;
    }
    const int nE = (int)(tot >> 48);
    const long long P = (long long)(tot & kMask48);
    if (tid == 0) sm.off[nE] = P;
    __syncthreads();
    const long long per = ((P + 32ll * kWarps - 1) / (32ll * kWarps)) * 32ll;
    long long base = (long long)warp * per;
    const long long wend = base + per < P ? base + per : P;
    if (base < wend) {
        // segment holding product `base`: largest e with off[e] <= base
        int lo = 0, hi = nE - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sm.off[mid] <= base) lo = mid;
            else hi = mid - 1;
        }
        int s = lo;
        long long so = sm.off[s], se = sm.off[s + 1];
        int sbs = sm.bs[s];
        Acc sa = sm.a[s];
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
                            se = sm.off[s + 1];
                            sbs = sm.bs[s];
                            sa = sm.a[s];
                        }
                    } else {
                        const int e = s + lane;
                        long long d = e <= nE ? sm.off[e] - base : (1ll << 30);
                        if (d > (1ll << 30)) d = 1ll << 30;
                        const int rel = (int)d;      // lane 0: <= 0, then non-decreasing
                        const int wbs = e < nE ? sm.bs[e] : 0;
                        const Acc wa = e < nE ? sm.a[e] : Acc(0);
                        const int src = warp_find_src(rel, lane);
                        tq[u] = __shfl_sync(kFull, wbs, src) + (lane - __shfl_sync(kFull, rel, src));
                        aq[u] = __shfl_sync(kFull, wa, src);
                        sq[u] = s + src;
                        vq[u] = base + lane < wend;
                        // segment of base + 32
                        const int cnt = __popc(__ballot_sync(kFull, rel <= 32));
                        int ns = s + cnt - 1;
                        if (cnt == 32 && s + 32 <= nE && sm.off[s + 32] <= base + 32) ns = s + 32;
                        s = ns < nE - 1 ? ns : nE - 1;
                        base += 32;
                        so = sm.off[s];
                        se = sm.off[s + 1];
                        sbs = sm.bs[s];
                        sa = sm.a[s];
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

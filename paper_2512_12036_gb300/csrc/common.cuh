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
    ST_UNSUPPORTED = 16
};

// Control block at the start of every workspace (256-byte aligned).
struct Ctl {
    int status;
    int b_unsorted;             // set when some row of B is not sorted by column
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

}  // namespace spg

// Markov-clustering matrix step (Algorithm 6) on the rows of M^T: after the
// expansion E = M^T * M^T (= (M*M)^T), each row of E (a column of M) is
// pruned (entries below theta dropped), cut to its k largest entries (ties
// to the smaller column), inflated (v^r) and normalised to sum 1.
//
// Keep/drop decisions are taken in fp32 on the value (order 0: prune and
// top-k first, then inflate) or on the fp32-rounded inflated value (order 1:
// inflate first). The k-th largest decision value is found by a radix
// selection over order-preserving 32-bit keys (four 8-bit digits, a
// 256-bin histogram each), so no sort is needed; kept entries keep their
// column order.
// Weights and the row sum are fp64; each output is rounded once to fp32.
// k < 0 keeps every entry that passes the threshold (a plain normalisation
// when theta <= 0 and r = 1).
#include "internal.h"

namespace spg {

constexpr int kMclWarpMax = 1024;     // rows up to this length: one warp, 32 entries per lane
constexpr int kMclThreads = 256;
constexpr int kMclBlockThreads = 1024;
constexpr int kMclStage = 32768;      // decision keys of a block row kept in shared memory (128 KB)
constexpr int kMclChunk = 128;        // rows the block kernel looks at together

struct MclParams {
    float theta;
    int k;
    double r;
    int order;
};

__device__ __forceinline__ unsigned ord_key(float x) {
    const unsigned b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ double mcl_weight(float v, double r) {
    const double d = (double)v;
    if (r == 2.0) return d * d;
    if (r == 1.0) return d;
    return pow(d, r);
}

__device__ __forceinline__ float mcl_decide(float v, const MclParams& p) {
    return p.order == 0 ? v : (float)mcl_weight(v, p.r);
}

// ---------------------------------------------------------------------------
// One warp per row of length <= kMclWarpMax. kWrite = false: count the kept
// entries into counts[row]; true: write them at rpt_out[row].
template <bool kWrite>
__global__ void __launch_bounds__(kMclThreads) k_mcl_warp(CsrDev E, MclParams prm, int* counts,
                                                          const int* rpt_out, int* col_out,
                                                          float* val_out, Ctl* ctl) {
    constexpr int kPer = kMclWarpMax / 32;
    __shared__ int whist[kMclThreads / 32][256];
    const int lane = lane_id();
    int* hist = whist[threadIdx.x >> 5];
    const long long gw = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = gw; row < E.rows; row += nw) {
        int s, e;
        row_extent(E, (int)row, s, e, ctl);
        const int n = e - s;
        if (n > kMclWarpMax) continue;                       // block kernel's row
        unsigned key[kPer];
        int cnt = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int q = s + lane + 32 * i;
            key[i] = 0u;
            if (q < e) {
                const float d = mcl_decide(E.val[q], prm);
                if (d >= prm.theta) {
                    key[i] = ord_key(d);
                    ++cnt;
                }
            }
        }
        cnt = warp_sum(cnt);
        const bool cut = prm.k >= 0 && cnt > prm.k;
        unsigned K = 1u;
        int need_eq = 0;
        if (cut) {
            // the k-th largest key by radix selection, 8 bits a pass from the
            // top, on a per-warp 256-bin histogram (see mcl_radix_digit)
            unsigned prefix = 0u, pmask = 0u;
            int above = 0;
            for (int sh = 24; sh >= 0; sh -= 8) {
#pragma unroll
                for (int b = 0; b < 8; ++b) hist[8 * lane + b] = 0;
                __syncwarp();
#pragma unroll
                for (int i = 0; i < kPer; ++i)
                    if (key[i] != 0u && (key[i] & pmask) == prefix)
                        atomicAdd(&hist[(key[i] >> sh) & 255u], 1);
                __syncwarp();
                int dig, run_at;
                radix_digit256(hist, above, prm.k, dig, run_at);
                prefix |= (unsigned)dig << sh;
                pmask |= 255u << sh;
                above = run_at;
                __syncwarp();
            }
            K = prefix;
            need_eq = prm.k - above;
        }
        const int keep_n = cut ? prm.k : cnt;
        if (!kWrite) {
            if (lane == 0) counts[row] = keep_n;
            continue;
        }
        // pass 1: kept flags in column order, weight sum
        unsigned keepmask = 0u;
        int eq_seen = 0;
        double wsum = 0.0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const bool cand = key[i] != 0u;
            bool kp = cand;
            if (cut) {                               // warp-uniform branch
                const bool eq = cand && key[i] == K;
                const unsigned eqb = __ballot_sync(kFull, eq);
                const int rank = eq_seen + __popc(eqb & lanemask_lt());
                kp = cand && (key[i] > K || (eq && rank < need_eq));
                eq_seen += __popc(eqb);
            }
            if (kp) {
                keepmask |= 1u << i;
                wsum += mcl_weight(E.val[s + lane + 32 * i], prm.r);
            }
        }
        wsum = warp_sum(wsum);
        // pass 2: write in column order
        int pos = rpt_out[row];
        const int pend = rpt_out[row + 1];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const bool kp = (keepmask >> i) & 1u;
            const unsigned b = __ballot_sync(kFull, kp);
            if (kp) {
                const int q = s + lane + 32 * i;
                const int o = pos + __popc(b & lanemask_lt());
                if (o < pend) {
                    col_out[o] = E.col[q];
                    const double w = mcl_weight(E.val[q], prm.r);
                    val_out[o] = wsum > 0.0 ? (float)(w / wsum) : 0.f;
                } else {
                    set_status(ctl, ST_INTERNAL);
                }
            }
            pos += __popc(b);
        }
        if (lane == 0 && pos != pend) set_status(ctl, ST_INTERNAL);
    }
}

// ---------------------------------------------------------------------------
// One block per row of length > kMclWarpMax (picked from chunks of rows). The
// row's decision keys are computed once into shared memory (rows up to
// kMclStage entries; longer rows recompute them per pass) and the k-th
// largest is found by a 4-pass radix selection (8 bits a pass).
template <bool kWrite>
__global__ void __launch_bounds__(kMclBlockThreads) k_mcl_block(CsrDev E, MclParams prm,
                                                                int* counts, const int* rpt_out,
                                                                int* col_out, float* val_out,
                                                                Ctl* ctl) {
    __shared__ int red[33];
    __shared__ double redd[33];
    __shared__ int scratch[33];
    __shared__ int hist[256];
    __shared__ int s_dig, s_above;
    extern __shared__ unsigned skey[];             // kMclStage decision keys
    __shared__ int s_long[kMclBlockThreads];       // this chunk's rows above kMclWarpMax
    __shared__ int s_nlong;
    // chunks of kMclChunk consecutive rows: one parallel look at their
    // lengths picks this kernel's rows, which the block then takes one at a
    // time (small chunks keep the blocks' shares of long rows even)
    for (long long base = (long long)blockIdx.x * kMclChunk; base < E.rows;
         base += (long long)gridDim.x * kMclChunk) {
    {
        const long long r0 = base + threadIdx.x;
        bool is_long = false;
        if ((int)threadIdx.x < kMclChunk && r0 < E.rows) {
            const int rs0 = E.rpt[r0], re0 = E.rpt[r0 + 1];
            is_long = re0 - rs0 > kMclWarpMax;
        }
        int nl;
        const int slot = block_excl_scan(is_long ? 1 : 0, scratch, &nl);
        if (is_long) s_long[slot] = (int)r0;
        if (threadIdx.x == 0) s_nlong = nl;
        __syncthreads();
    }
    const int nlong = s_nlong;
    for (int li = 0; li < nlong; ++li) {
        const long long row = s_long[li];
        int s, e;
        row_extent(E, (int)row, s, e, ctl);
        if (e - s <= kMclWarpMax) continue;
        auto key_of = [&](int q) -> unsigned {
            const float d = mcl_decide(E.val[q], prm);
            return d >= prm.theta ? ord_key(d) : 0u;
        };
        // decision keys, staged in shared memory when the row fits
        const int n = e - s;
        const bool staged = n <= kMclStage;
        int c0 = 0;
        for (int q = s + threadIdx.x; q < e; q += blockDim.x) {
            const unsigned kq = key_of(q);
            if (staged) skey[q - s] = kq;
            c0 += kq != 0u;
        }
        const int cnt = block_sum(c0, red);       // (barrier: skey ready)
        auto key_at = [&](int q) -> unsigned { return staged ? skey[q - s] : key_of(q); };
        const bool cut = prm.k >= 0 && cnt > prm.k;
        unsigned K = 1u;
        int need_eq = 0;
        if (cut) {
            // the k-th largest key by radix selection, 8 bits a pass from the
            // top: a 256-bin histogram of the keys that share the prefix found
            // so far, then the digit whose bin holds the k-th largest
            unsigned prefix = 0u, pmask = 0u;
            int above = 0;                          // keys known to be larger than the prefix
            for (int sh = 24; sh >= 0; sh -= 8) {
                for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
                __syncthreads();
                for (int q = s + threadIdx.x; q < e; q += blockDim.x) {
                    const unsigned kq = key_at(q);
                    if (kq != 0u && (kq & pmask) == prefix) atomicAdd(&hist[(kq >> sh) & 255u], 1);
                }
                __syncthreads();
                if (threadIdx.x < 32) {
                    int dig, run_at;
                    radix_digit256(hist, above, prm.k, dig, run_at);
                    if (threadIdx.x == 0) {
                        s_dig = dig;
                        s_above = run_at;
                    }
                }
                __syncthreads();
                prefix |= (unsigned)s_dig << sh;
                pmask |= 255u << sh;
                above = s_above;
                __syncthreads();
            }
            K = prefix;
            need_eq = prm.k - above;
        }
        const int keep_n = cut ? prm.k : cnt;
        if (!kWrite) {
            if (threadIdx.x == 0) counts[row] = keep_n;
            continue;
        }
        // chunks of blockDim entries in column order: kept flags, then writes
        auto kept = [&](int q, unsigned kq, int eq_rank) {
            if (kq == 0u) return false;
            if (!cut) return true;
            if (kq > K) return true;
            return kq == K && eq_rank < need_eq;
        };
        double wpart = 0.0;
        int eq_seen = 0;
        for (int base = s; base < e; base += blockDim.x) {
            const int q = base + threadIdx.x;
            const unsigned kq = q < e ? key_of(q) : 0u;
            int eq_tot;
            const int eq_rank = eq_seen + block_excl_scan((cut && kq == K) ? 1 : 0, scratch, &eq_tot);
            if (q < e && kept(q, kq, eq_rank)) wpart += mcl_weight(E.val[q], prm.r);
            eq_seen += eq_tot;
        }
        const double wsum = block_sum(wpart, redd);
        int pos = rpt_out[row];
        const int pend = rpt_out[row + 1];
        eq_seen = 0;
        for (int base = s; base < e; base += blockDim.x) {
            const int q = base + threadIdx.x;
            const unsigned kq = q < e ? key_of(q) : 0u;
            int eq_tot;
            const int eq_rank = eq_seen + block_excl_scan((cut && kq == K) ? 1 : 0, scratch, &eq_tot);
            eq_seen += eq_tot;
            const bool kp = q < e && kept(q, kq, eq_rank);
            int ktot;
            const int o = pos + block_excl_scan(kp ? 1 : 0, scratch, &ktot);
            if (kp) {
                if (o < pend) {
                    col_out[o] = E.col[q];
                    const double w = mcl_weight(E.val[q], prm.r);
                    val_out[o] = wsum > 0.0 ? (float)(w / wsum) : 0.f;
                } else {
                    set_status(ctl, ST_INTERNAL);
                }
            }
            pos += ktot;
        }
        if (threadIdx.x == 0 && pos != pend) set_status(ctl, ST_INTERNAL);
        __syncthreads();
    }
    __syncthreads();                               // s_long is rewritten by the next chunk
    }
}

void occupancy_mcl(spgemm_plan* p) {
    allow_max_dynamic_smem((const void*)k_mcl_block<false>, p);
    allow_max_dynamic_smem((const void*)k_mcl_block<true>, p);
}

void launch_mcl_step(const spgemm_plan* p, const CsrDev& E, float theta, int k, double r,
                     int order, const WsPtrs& w, int* rpt_out, int* col_out, float* val_out,
                     cudaStream_t s) {
    if (E.rows == 0) {
        launch_row_ptr(p, w.map, 0, w, rpt_out, s);
        return;
    }
    const MclParams prm{theta, k, r, order};
    const int sms = p->num_sms;
    int* counts = w.map;                       // E.rows ints of the workspace
    SPG_LAUNCH(p, K_MCL, s, k_mcl_warp<false><<<sms * 8, kMclThreads, 0, s>>>(E, prm, counts, nullptr, nullptr, nullptr, w.ctl));
    SPG_LAUNCH(p, K_MCL, s, k_mcl_block<false><<<sms, kMclBlockThreads, kMclStage * 4, s>>>(E, prm, counts, nullptr, nullptr, nullptr, w.ctl));
    launch_row_ptr(p, counts, E.rows, w, rpt_out, s);
    SPG_LAUNCH(p, K_MCL, s, k_mcl_warp<true><<<sms * 8, kMclThreads, 0, s>>>(E, prm, counts, rpt_out, col_out, val_out, w.ctl));
    SPG_LAUNCH(p, K_MCL, s, k_mcl_block<true><<<sms, kMclBlockThreads, kMclStage * 4, s>>>(E, prm, counts, rpt_out, col_out, val_out, w.ctl));
}

}  // namespace spg

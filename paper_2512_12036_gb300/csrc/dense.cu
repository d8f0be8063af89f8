// Dense fp32 products of the pruned GNN layer (Section IV-C, Eqs. 1-3):
// Y = C_d * W in the forward (C_d the aggregated features A*TopK(X) laid
// out dense), G = dY * W^T and dW = C_d^T * dY in the backward. These are
// the layer's only dense contractions; they run here on the CUDA cores in
// fp32 (fused multiply-add, the same arithmetic as the rest of the layer)
// as register-tiled GEMMs:
//   a 128 x 128 output tile per block of 256 threads, 8 x 8 outputs per
//   thread (rows ty*8.., columns tx*4.. and 64+tx*4..), k-steps of 16
//   staged through shared memory in two buffers (the
//   next step's tile is fetched into registers while the current one is
//   multiplied). Either operand may be read transposed. A long reduction
//   (dW sums over every row of the graph) is split over blocks along K:
//   each block adds its fp32 partial tile into an fp64 accumulator with
//   fp64 atomics, converted to fp32 once at the end.
#include "internal.h"

namespace spg {

constexpr int kGemmBM = 128, kGemmBN = 128, kGemmBK = 16, kGemmThreads = 256;
constexpr int kGemmPad = 4;   // row padding of the shared tiles (spreads banks)

// op(A) is M x K, op(B) is K x N, all row-major with leading dimensions.
// TA: A is stored K x M; TB: B is stored N x K.
template <bool TA, bool TB>
__global__ void __launch_bounds__(kGemmThreads, 2)
    k_sgemm(int M, int N, int K, const float* __restrict__ A, long long lda,
            const float* __restrict__ B, long long ldb, float* __restrict__ C, long long ldc,
            double* __restrict__ Cacc, int kchunk, bool vec) {
    __shared__ __align__(16) float As[2][kGemmBK][kGemmBM + kGemmPad];
    __shared__ __align__(16) float Bs[2][kGemmBK][kGemmBN + kGemmPad];
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    const int m0 = blockIdx.y * kGemmBM, n0 = blockIdx.x * kGemmBN;
    const int kb = blockIdx.z * kchunk;
    const int ke = kb + kchunk < K ? kb + kchunk : K;

    // this thread's share of a tile: 8 consecutive elements along a stored
    // row of the operand (two 16-byte loads when they are all inside and
    // the operand is 16-byte aligned with a leading dimension of 4k floats)
    float ra[8], rb[8];
    auto load8 = [&](float* r, const float* src, int valid) {
        if (vec && valid >= 8) {
            const float4 x = __ldg(reinterpret_cast<const float4*>(src));
            const float4 y = __ldg(reinterpret_cast<const float4*>(src + 4));
            r[0] = x.x; r[1] = x.y; r[2] = x.z; r[3] = x.w;
            r[4] = y.x; r[5] = y.y; r[6] = y.z; r[7] = y.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) r[q] = q < valid ? __ldg(src + q) : 0.f;
        }
    };
    auto fetch = [&](int k0) {
        if (!TA) {                              // A[m][k]: row m = t/2, k = (t&1)*8 ..
            const int m = m0 + (t >> 1), k = k0 + (t & 1) * 8;
            load8(ra, A + (long long)m * lda + k, m < M ? ke - k : 0);
        } else {                                // A[k][m]: row k = t/16, m = (t&15)*8 ..
            const int k = k0 + (t >> 4), m = m0 + (t & 15) * 8;
            load8(ra, A + (long long)k * lda + m, k < ke ? M - m : 0);
        }
        if (!TB) {                              // B[k][n]: row k = t/16, n = (t&15)*8 ..
            const int k = k0 + (t >> 4), n = n0 + (t & 15) * 8;
            load8(rb, B + (long long)k * ldb + n, k < ke ? N - n : 0);
        } else {                                // B[n][k]: row n = t/2, k = (t&1)*8 ..
            const int n = n0 + (t >> 1), k = k0 + (t & 1) * 8;
            load8(rb, B + (long long)n * ldb + k, n < N ? ke - k : 0);
        }
    };
    auto stash = [&](int buf) {
        if (!TA) {
#pragma unroll
            for (int q = 0; q < 8; ++q) As[buf][(t & 1) * 8 + q][t >> 1] = ra[q];
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) As[buf][t >> 4][(t & 15) * 8 + q] = ra[q];
        }
        if (!TB) {
#pragma unroll
            for (int q = 0; q < 8; ++q) Bs[buf][t >> 4][(t & 15) * 8 + q] = rb[q];
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) Bs[buf][(t & 1) * 8 + q][t >> 1] = rb[q];
        }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    int buf = 0;
    if (kb < ke) {
        fetch(kb);
        stash(0);
    }
    __syncthreads();
    for (int k0 = kb; k0 < ke; k0 += kGemmBK) {
        const bool more = k0 + kGemmBK < ke;
        if (more) fetch(k0 + kGemmBK);          // in flight while this step multiplies
#pragma unroll
        for (int k = 0; k < kGemmBK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 8 + 4]);
            // columns tx*4 .. +3 and 64 + tx*4 .. +3: a warp's 16 column
            // groups read 256 contiguous bytes per load (two wavefronts)
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            stash(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + ty * 8 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
            if (n >= N) continue;
            if (Cacc) atomicAdd(&Cacc[(long long)m * N + n], (double)acc[i][j]);
            else C[(long long)m * ldc + n] = acc[i][j];
        }
    }
}

__global__ void k_gemm_zero(double* p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

__global__ void k_gemm_round(const double* acc, int M, int N, float* C, long long ldc) {
    const long long n = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        C[(i / N) * ldc + i % N] = (float)acc[i];
}

// Blocks along K for a reduction of length K over an M x N output: enough
// to fill the GPU twice, each block at least 4096 deep.
int gemm_ksplit(const spgemm_plan* p, int M, int N, int K) {
    const long long tiles = (long long)((M + kGemmBM - 1) / kGemmBM) * ((N + kGemmBN - 1) / kGemmBN);
    long long want = (2ll * p->num_sms + tiles - 1) / tiles;
    const long long maxk = (K + 4095) / 4096;
    if (want > maxk) want = maxk;
    if (want > 65535) want = 65535;
    return want < 1 ? 1 : (int)want;
}

void launch_sgemm(const spgemm_plan* p, int M, int N, int K, const float* A, long long lda,
                  bool ta, const float* B, long long ldb, bool tb, float* C, long long ldc,
                  double* acc, int ksplit, cudaStream_t s) {
    if (M <= 0 || N <= 0) return;
    if (acc == nullptr) ksplit = 1;
    const int kchunk = ksplit > 1 ? (((K + ksplit - 1) / ksplit + kGemmBK - 1) / kGemmBK) * kGemmBK
                                  : (K > 0 ? K : 1);
    const dim3 grid((N + kGemmBN - 1) / kGemmBN, (M + kGemmBM - 1) / kGemmBM,
                    ksplit > 1 ? (K + kchunk - 1) / kchunk : 1);
    const bool vec = ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0 && (lda & 3) == 0 &&
                     (ldb & 3) == 0;
    if (acc)
        SPG_LAUNCH(p, K_GEMM, s, k_gemm_zero<<<p->num_sms * 4, 256, 0, s>>>(acc, (long long)M * N));
#define SPG_SGEMM(TA_, TB_)                                                                       \
    SPG_LAUNCH(p, K_GEMM, s,                                                                      \
               (k_sgemm<TA_, TB_><<<grid, kGemmThreads, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, \
                                                                 acc, kchunk, vec)))
    if (!ta && !tb) SPG_SGEMM(false, false);
    else if (!ta && tb) SPG_SGEMM(false, true);
    else if (ta && !tb) SPG_SGEMM(true, false);
    else SPG_SGEMM(true, true);
#undef SPG_SGEMM
    if (acc)
        SPG_LAUNCH(p, K_GEMM, s, k_gemm_round<<<p->num_sms * 4, 256, 0, s>>>(acc, M, N, C, ldc));
}

}  // namespace spg

using namespace spg;

extern "C" int spgemm_dense_gemm_workspace_bytes(const spgemm_plan* plan, int32_t M, int32_t N,
                                                 int32_t K, size_t* bytes) {
    if (!plan || !bytes || M < 0 || N < 0 || K < 0) return SPGEMM_ERR_INVALID;
    *bytes = gemm_ksplit(plan, M, N, K) > 1 ? sizeof(double) * (size_t)M * (size_t)N + 256 : 0;
    return SPGEMM_OK;
}

extern "C" int spgemm_dense_gemm(const spgemm_plan* plan, int32_t M, int32_t N, int32_t K,
                                 const float* A, int64_t lda, int32_t trans_a, const float* B,
                                 int64_t ldb, int32_t trans_b, float* C, int64_t ldc, void* ws,
                                 size_t ws_bytes, void* stream) {
    if (!plan || M < 0 || N < 0 || K < 0) return SPGEMM_ERR_INVALID;
    if ((trans_a != 0 && trans_a != 1) || (trans_b != 0 && trans_b != 1)) return SPGEMM_ERR_INVALID;
    if (M == 0 || N == 0) return SPGEMM_OK;
    if (!C || ldc < N) return SPGEMM_ERR_INVALID;
    if (K > 0) {
        if (!A || !B) return SPGEMM_ERR_INVALID;
        if (lda < (trans_a ? M : K) || ldb < (trans_b ? K : N)) return SPGEMM_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (K == 0) {                                   // an empty sum
        if (ldc == N)
            return cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * N, s) == cudaSuccess
                       ? SPGEMM_OK : SPGEMM_ERR_CUDA;
        for (int32_t m = 0; m < M; ++m)
            if (cudaMemsetAsync(C + (size_t)m * ldc, 0, sizeof(float) * (size_t)N, s) != cudaSuccess)
                return SPGEMM_ERR_CUDA;
        return SPGEMM_OK;
    }
    int ksplit = gemm_ksplit(plan, M, N, K);
    double* acc = nullptr;
    if (ksplit > 1) {
        const size_t need = sizeof(double) * (size_t)M * (size_t)N;
        if (ws && ws_bytes >= need && ((uintptr_t)ws & 255) == 0) acc = (double*)ws;
        else ksplit = 1;                            // no workspace: one block per tile along K
    }
    launch_sgemm(plan, M, N, K, A, lda, trans_a != 0, B, ldb, trans_b != 0, C, ldc, acc, ksplit, s);
    return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

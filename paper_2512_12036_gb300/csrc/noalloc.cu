// Row-pointer scan for callers that cannot allocate device memory.
//
// spgemm_row_ptr needs a workspace from the caller for its scratch (block
// partial sums and a status/total word). Some callers have no way to get
// one: a plugin inside a host framework that owns every device allocation,
// a real-time or fixed-budget service that forbids allocation after start-up,
// or code that runs where cudaMalloc is not allowed or would synchronise the
// device. spgemm_row_ptr_static runs the same scan kernels with that scratch
// in a fixed array compiled into this library instead (kStaticScratchBytes,
// resident on every GPU that loads the library until the process exits).
#include <mutex>

#include "internal.h"

namespace spg {

// Largest n the static scratch can scan: 2^26 rows -> 16384 block partials.
constexpr int kStaticMaxRows = 1 << 26;
constexpr int kStaticMaxParts = (kStaticMaxRows + kScanItems - 1) / kScanItems + 1;
constexpr size_t kStaticScratchBytes = sizeof(Ctl) + sizeof(long long) * kStaticMaxParts;

// The scratch itself. In host code this name is only a stand-in for the
// symbol: its device address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (looked up once per
// device; the lookup must not happen inside a stream capture).
int scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return SPGEMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || ptr == nullptr)
            return SPGEMM_ERR_CUDA;
        g_scratch_addr[device] = ptr;
    }
    *out = g_scratch_addr[device];
    return SPGEMM_OK;
}
}  // namespace

}  // namespace spg

using namespace spg;

extern "C" int spgemm_row_ptr_static(const spgemm_plan* plan, const int32_t* row_nnz, int32_t n,
                                     int32_t* row_ptr, int64_t* total, void* stream) {
    if (!plan || n < 0 || !row_ptr || (n > 0 && !row_nnz)) return SPGEMM_ERR_INVALID;
    if (n > kStaticMaxRows) return SPGEMM_ERR_UNSUPPORTED;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (device != plan->device) return SPGEMM_ERR_INVALID;
    void* base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    WsPtrs w{};
    w.ctl = (Ctl*)base;
    w.scan_part = (long long*)((unsigned char*)base + sizeof(Ctl));
    w.nscan = (n + kScanItems - 1) / kScanItems;
    // the status word and totals must start at zero; the partials are always
    // written before they are read
    if (cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), s) != cudaSuccess) return SPGEMM_ERR_CUDA;
    launch_row_ptr(plan, row_nnz, n, w, row_ptr, s);
    if (cudaGetLastError() != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (!total) return SPGEMM_OK;
    long long tot = 0;
    int status = 0;
    if (cudaMemcpyAsync(&tot, &w.ctl->totals[2], sizeof(tot), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(&status, &w.ctl->status, sizeof(status), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SPGEMM_ERR_CUDA;
    *total = tot;
    if (status & ST_OVERFLOW) return SPGEMM_ERR_OVERFLOW;
    if (status & ST_INVALID) return SPGEMM_ERR_INVALID;
    return status ? SPGEMM_ERR_INTERNAL : SPGEMM_OK;
}

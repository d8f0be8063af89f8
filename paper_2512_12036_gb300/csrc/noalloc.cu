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
// Per device: the scratch's device address and the id of the context it was
// looked up in. A device reset (cudaDeviceReset) or a new primary context
// reloads the module, and the symbol may then sit at another address, so the
// address is looked up again whenever the current context's id changes.
void* g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};

typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Id of the calling thread's current context (unique for the life of the
// process, unlike the context handle, which a new context may reuse);
// 0 when the driver cannot say.
unsigned long long current_context_id() {
    if (!g_ctx_get_current || !g_ctx_get_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) !=
                cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess)
            return 0;
        g_ctx_get_current = (CtxGetCurrentFn)f1;
        g_ctx_get_id = (CtxGetIdFn)f2;
    }
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != 0 || ctx == nullptr || g_ctx_get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch on the current device, looked up on the
// first call in each context (the lookup must not happen inside a stream
// capture).
int scratch_address(int device, void** out) {
    if (device < 0 || device >= kMaxDevices) return SPGEMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[device] || ctx == 0 || ctx != g_scratch_ctx[device]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || ptr == nullptr)
            return SPGEMM_ERR_CUDA;
        g_scratch_addr[device] = ptr;
        g_scratch_ctx[device] = ctx;
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

// C ABI of libspgemm: argument checks, workspace layout and phase order.
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include "internal.h"

namespace spg {
void occupancy_symbolic(spgemm_plan* p);
void occupancy_numeric(spgemm_plan* p);
void occupancy_backward(spgemm_plan* p);
void occupancy_mcl(spgemm_plan* p);
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout ws_layout(const spgemm_plan* p, long long m, long long b_rows, long long b_cols,
                   long long b_nnz) {
    WsLayout L;
    L.m = (int)m;
    L.nblk = (int)((m + kBinRows - 1) / kBinRows);
    const long long nscan_rows = m > b_cols ? m : b_cols;
    L.nscan = (int)((nscan_rows + kScanItems - 1) / kScanItems);
    const long long pw = p->opts.panel_cols;
    L.panels = (int)((b_cols + pw - 1) / pw);
    size_t off = 0;
    L.ctl = off;
    off = align256(off + sizeof(Ctl));
    L.map = off;
    off = align256(off + sizeof(int) * (size_t)(m > 0 ? m : 1));
    L.blk_counts = off;
    off = align256(off + sizeof(int) * (size_t)kNumBins * (size_t)(L.nblk > 0 ? L.nblk : 1));
    L.scan_part = off;
    off = align256(off + sizeof(long long) * (size_t)(L.nscan + 1));
    L.bpanel = off;
    if (L.panels > 0 && L.panels <= kMaxPanels && b_rows > 0)
        off = align256(off + sizeof(int) * (size_t)b_rows * (size_t)(L.panels + 1));
    if (b_cols > 0 && b_nnz > 0) {
        L.has_hot = true;
        L.colcnt = off;
        off = align256(off + sizeof(int) * (size_t)(b_cols + 1));
        L.hot_rank = off;
        off = align256(off + sizeof(int) * (size_t)(b_cols + 1));
        L.hot_col = off;
        off = align256(off + sizeof(int) * (size_t)b_cols);
        L.bhot = off;
        off = align256(off + sizeof(int) * (size_t)b_nnz);
        L.bhv = off;
        off = align256(off + 8 * (size_t)b_nnz);
        L.bcv = off;
        off = align256(off + 8 * (size_t)b_nnz);
    }
    const long long wpr = (b_cols + 31) / 32;
    if (p->opts.row_cache_mb > 0 && m > 0 && wpr > 0 && wpr <= kRowCacheMaxWords) {
        const size_t bytes = (size_t)p->opts.row_cache_mb << 20;
        // per slot: the bitmap, and the entry count of each table panel
        const bool counts = L.panels > 0 && L.panels <= kMaxPanels;
        const size_t slot_bytes = align256(sizeof(int) * (size_t)m) + (counts ? 256 : 0);
        const size_t row_bytes = sizeof(unsigned) * (size_t)wpr + (counts ? sizeof(int) * (size_t)L.panels : 0);
        long long n = bytes > slot_bytes ? (long long)((bytes - slot_bytes) / row_bytes) : 0;
        if (n > m) n = m;
        if (n > 0) {
            L.rc_nslots = (int)n;
            L.rc_wpr = (int)wpr;
            L.rc_slot = off;
            off += align256(sizeof(int) * (size_t)m);
            L.rc_bits = off;
            off = align256(off + sizeof(unsigned) * (size_t)wpr * (size_t)n);
            if (counts) {
                L.rc_pc = off;
                off = align256(off + sizeof(int) * (size_t)L.panels * (size_t)n);
            }
        }
    }
    L.total = off;
    return L;
}

WsPtrs ws_ptrs(const WsLayout& L, void* ws, int panel_cols) {
    char* b = (char*)ws;
    WsPtrs w;
    w.ctl = (Ctl*)(b + L.ctl);
    w.map = (int*)(b + L.map);
    w.blk_counts = (int*)(b + L.blk_counts);
    w.scan_part = (long long*)(b + L.scan_part);
    w.bpanel = (L.panels > 0 && L.panels <= kMaxPanels && (L.has_hot ? L.colcnt : L.total) > L.bpanel)
                   ? (int*)(b + L.bpanel) : nullptr;
    w.colcnt = L.has_hot ? (int*)(b + L.colcnt) : nullptr;
    w.hot_rank = L.has_hot ? (int*)(b + L.hot_rank) : nullptr;
    w.hot_col = L.has_hot ? (int*)(b + L.hot_col) : nullptr;
    w.bhot = L.has_hot ? (int*)(b + L.bhot) : nullptr;
    w.bhv = L.has_hot ? (int2*)(b + L.bhv) : nullptr;
    w.bcv = L.has_hot ? (int2*)(b + L.bcv) : nullptr;
    w.rc_slot = L.rc_nslots > 0 ? (int*)(b + L.rc_slot) : nullptr;
    w.rc_bits = L.rc_nslots > 0 ? (unsigned*)(b + L.rc_bits) : nullptr;
    w.rc_pc = L.rc_nslots > 0 && L.rc_pc > 0 ? (int*)(b + L.rc_pc) : nullptr;
    w.rc_nslots = L.rc_nslots;
    w.rc_wpr = L.rc_wpr;
    w.nblk = L.nblk;
    w.nscan = L.nscan;
    w.panels = L.panels;
    w.panel_cols = panel_cols;
    return w;
}

void allow_max_dynamic_smem(const void* f, const spgemm_plan* p) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) return;
    const size_t st = fa.sharedSizeBytes;
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         p->smem_optin > st ? (int)(p->smem_optin - st) : 0);
}

void init_occupancy(spgemm_plan* p) {
    occupancy_symbolic(p);
    occupancy_numeric(p);
    occupancy_backward(p);
    occupancy_mcl(p);
}

const char* const kKernelNames[K_NUM_KERNELS] = {
    "fill", "check_rpt", "zero_total", "ip_count", "sum", "group_hist", "group_scan",
    "group_scatter", "scan_part", "scan_top", "scan_final", "reset_flag", "bpanel", "sym_esc",
    "sym_warp", "sym_block", "sym_dense", "num_esc", "num_warp32", "num_warp64", "num_block32",
    "num_block64", "num_dense32", "num_dense64", "backward", "guard", "mcl", "hot", "layer",
    "sym_narrow", "num_narrow", "gemm"};

void prof_begin(const spgemm_plan* p, int kid, cudaStream_t s) {
    (void)kid;
    ProfState* st = p->prof;
    __atomic_fetch_add(&st->launches, 1ull, __ATOMIC_RELAXED);
    if (st->on && st->n < st->cap) cudaEventRecord(st->ev[2 * st->n], s);
}

void prof_end(const spgemm_plan* p, int kid, cudaStream_t s) {
    ProfState* st = p->prof;
    if (st->on && st->n < st->cap) {
        cudaEventRecord(st->ev[2 * st->n + 1], s);
        st->kid[st->n] = kid;
        ++st->n;
    }
}

static void prof_free(ProfState* st) {
    if (st->ev) {
        for (int i = 0; i < 2 * st->cap; ++i) cudaEventDestroy(st->ev[i]);
        free(st->ev);
        free(st->kid);
    }
    st->ev = nullptr;
    st->kid = nullptr;
    st->cap = 0;
    st->n = 0;
    st->on = 0;
}

}  // namespace spg

using namespace spg;

static int cuda_err(cudaError_t e) { return e == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA; }

static int check_csr(const spgemm_csr* M, bool need_vals) {
    if (!M) return SPGEMM_ERR_INVALID;
    if (M->rows < 0 || M->cols < 0 || M->nnz < 0 || M->nnz > 2147483647ll) return SPGEMM_ERR_INVALID;
    if (!M->row_ptr) return SPGEMM_ERR_INVALID;
    if (M->nnz > 0 && !M->col_idx) return SPGEMM_ERR_INVALID;
    if (need_vals && M->nnz > 0 && !M->vals) return SPGEMM_ERR_INVALID;
    return SPGEMM_OK;
}

static CsrDev dev_view(const spgemm_csr* M) {
    CsrDev d;
    d.rows = M->rows;
    d.cols = M->cols;
    d.nnz = M->nnz;
    d.rpt = M->row_ptr;
    d.col = M->col_idx;
    d.val = M->vals;
    return d;
}

static int check_pair(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B,
                      bool need_vals) {
    if (!plan) return SPGEMM_ERR_INVALID;
    int rc = check_csr(A, need_vals);
    if (rc) return rc;
    rc = check_csr(B, need_vals);
    if (rc) return rc;
    if (A->cols != B->rows) return SPGEMM_ERR_INVALID;
    return SPGEMM_OK;
}

static int check_ws(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B, void* ws,
                    size_t ws_bytes, WsLayout* L) {
    *L = ws_layout(plan, A->rows, B->rows, B->cols, B->nnz);
    if (!ws || ws_bytes < L->total) return SPGEMM_ERR_WORKSPACE;
    if (((uintptr_t)ws & 255) != 0) return SPGEMM_ERR_WORKSPACE;
    return SPGEMM_OK;
}

static int map_status(int bits) {
    if (bits & ST_INVALID) return SPGEMM_ERR_INVALID;
    if (bits & ST_BUDGET) return SPGEMM_ERR_BUDGET;
    if (bits & ST_OVERFLOW) return SPGEMM_ERR_OVERFLOW;
    if (bits & ST_TIMEOUT) return SPGEMM_ERR_TIMEOUT;
    if (bits & ST_UNSUPPORTED) return SPGEMM_ERR_UNSUPPORTED;
    if (bits & ST_INTERNAL) return SPGEMM_ERR_INTERNAL;
    return SPGEMM_OK;
}

// Synchronise, fetch totals[which] (if out) and the status word, clear it.
static int sync_read(Ctl* ctl, int which, int64_t* out, cudaStream_t s) {
    Ctl h;                                   // its head, up to and including the totals
    cudaError_t e = cudaMemcpyAsync(&h, ctl, offsetof(Ctl, totals) + sizeof(h.totals),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (out && which >= 0) *out = h.totals[which];
    if (h.status) {
        int zero = 0;
        cudaMemcpyAsync(&ctl->status, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
    }
    return map_status(h.status);
}

extern "C" {

int spgemm_opts_default(spgemm_opts* o) {
    if (!o) return SPGEMM_ERR_INVALID;
    memset(o, 0, sizeof(*o));
    o->fp32_max_terms = 167;
    o->esc_max = 32;
    o->warp_max_ip = 1024;
    o->block_max_ip = 16384;
    o->warp_max_nnz = 512;
    o->block_max_nnz = 8192;
    o->panel_cols = 16384;
    return SPGEMM_OK;
}

int spgemm_plan_create(spgemm_plan** out, const spgemm_opts* opts, int device) {
    if (!out) return SPGEMM_ERR_INVALID;
    *out = nullptr;
    spgemm_opts o;
    if (opts) o = *opts;
    else spgemm_opts_default(&o);
    // limits of the kernels: in-register tier is one warp, tables are powers
    // of two in shared memory, a dense panel is at most 32 columns per thread
    if (o.esc_max < 1 || o.esc_max > 32) return SPGEMM_ERR_INVALID;
    if (o.warp_max_ip < o.esc_max || o.warp_max_ip > kWarpTableSym / 2) return SPGEMM_ERR_INVALID;
    if (o.block_max_ip < o.warp_max_ip || o.block_max_ip > 32768) return SPGEMM_ERR_INVALID;
    if (o.warp_max_nnz < 1 || o.warp_max_nnz > kWarpTableNum / 2) return SPGEMM_ERR_INVALID;
    if (o.block_max_nnz < o.warp_max_nnz || o.block_max_nnz > 8192) return SPGEMM_ERR_INVALID;
    if (o.panel_cols < 1024 || o.panel_cols > 16384 || (o.panel_cols & (o.panel_cols - 1)))
        return SPGEMM_ERR_INVALID;
    if (o.fp32_max_terms < 0) return SPGEMM_ERR_INVALID;
    if (o.row_cache_mb < 0 || o.dense_splits < 0 || o.dense_splits > 64) return SPGEMM_ERR_INVALID;
    if (o.stage_b != 0 && o.stage_b != 1) return SPGEMM_ERR_INVALID;
    if (o.narrow_warps < 0 || o.narrow_warps > kNarrowMaxWarps || o.narrow_max_ip < 0)
        return SPGEMM_ERR_INVALID;
    if (o.hash_load_pct != 0 && (o.hash_load_pct < 25 || o.hash_load_pct > 90))
        return SPGEMM_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return SPGEMM_ERR_CUDA;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    spgemm_plan* p = (spgemm_plan*)calloc(1, sizeof(spgemm_plan));
    if (!p) return SPGEMM_ERR_INTERNAL;
    p->prof = new ProfState();
    p->device = device;
    p->opts = o;
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    p->num_sms = v > 0 ? v : 1;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    p->smem_optin = (size_t)v;
    init_occupancy(p);
    cudaError_t e = cudaGetLastError();
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        delete p->prof;
        free(p);
        return SPGEMM_ERR_CUDA;
    }
    *out = p;
    return SPGEMM_OK;
}

int spgemm_plan_destroy(spgemm_plan* p) {
    if (!p) return SPGEMM_OK;
    prof_free(p->prof);
    delete p->prof;
    free(p);
    return SPGEMM_OK;
}

int spgemm_profile_enable(spgemm_plan* plan, int on) {
    if (!plan) return SPGEMM_ERR_INVALID;
    ProfState* st = plan->prof;
    if (!on) {
        prof_free(st);
        return SPGEMM_OK;
    }
    if (st->cap == 0) {
        const int cap = 8192;
        st->ev = (cudaEvent_t*)calloc(2 * cap, sizeof(cudaEvent_t));
        st->kid = (int*)calloc(cap, sizeof(int));
        if (!st->ev || !st->kid) {
            prof_free(st);
            return SPGEMM_ERR_INTERNAL;
        }
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(plan->device);
        for (int i = 0; i < 2 * cap; ++i) {
            if (cudaEventCreate(&st->ev[i]) != cudaSuccess) {
                st->cap = i / 2;
                cudaSetDevice(prev);
                prof_free(st);
                return SPGEMM_ERR_CUDA;
            }
            st->cap = (i + 1) / 2;
        }
        cudaSetDevice(prev);
        st->cap = cap;
    }
    st->n = 0;
    st->on = 1;
    return SPGEMM_OK;
}

int spgemm_profile_read(spgemm_plan* plan, double* ms, int64_t* launches, int n) {
    if (!plan || n < 0 || (n > 0 && (!ms || !launches))) return SPGEMM_ERR_INVALID;
    ProfState* st = plan->prof;
    for (int k = 0; k < n; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (int i = 0; i < st->n; ++i) {
        if (cudaEventSynchronize(st->ev[2 * i + 1]) != cudaSuccess) return SPGEMM_ERR_CUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, st->ev[2 * i], st->ev[2 * i + 1]) != cudaSuccess)
            return SPGEMM_ERR_CUDA;
        const int k = st->kid[i];
        if (k < n) {
            ms[k] += t;
            launches[k] += 1;
        }
    }
    st->n = 0;
    return SPGEMM_OK;
}

int spgemm_kernel_count(void) { return K_NUM_KERNELS; }

const char* spgemm_kernel_name(int kid) {
    return (kid >= 0 && kid < K_NUM_KERNELS) ? kKernelNames[kid] : "unknown";
}

int64_t spgemm_launch_total(const spgemm_plan* plan) {
    return plan ? (int64_t)__atomic_load_n(&plan->prof->launches, __ATOMIC_RELAXED) : 0;
}

int spgemm_workspace_bytes(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B,
                           size_t* bytes) {
    if (!plan || !A || !B || !bytes) return SPGEMM_ERR_INVALID;
    if (A->rows < 0 || B->rows < 0 || B->cols < 0) return SPGEMM_ERR_INVALID;
    *bytes = ws_layout(plan, A->rows, B->rows, B->cols, B->nnz).total;
    return SPGEMM_OK;
}

int spgemm_workspace_init(const spgemm_plan* plan, void* ws, size_t ws_bytes, void* stream) {
    if (!plan) return SPGEMM_ERR_INVALID;
    if (!ws || ws_bytes < sizeof(Ctl) || ((uintptr_t)ws & 255)) return SPGEMM_ERR_WORKSPACE;
    return cuda_err(cudaMemsetAsync(ws, 0, sizeof(Ctl), (cudaStream_t)stream));
}

int spgemm_count(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B, void* ws,
                 size_t ws_bytes, int64_t* ip_row, int64_t* ip_total, void* stream) {
    int rc = check_pair(plan, A, B, false);
    if (rc) return rc;
    if (A->rows > 0 && !ip_row) return SPGEMM_ERR_INVALID;
    WsLayout L;
    rc = check_ws(plan, A, B, ws, ws_bytes, &L);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(L, ws, plan->opts.panel_cols);
    launch_ip_count(plan, dev_view(A), dev_view(B), (long long*)ip_row, w, s);
    rc = cuda_err(cudaGetLastError());
    if (rc) return rc;
    if (ip_total) return sync_read(w.ctl, 0, ip_total, s);
    return SPGEMM_OK;
}

int spgemm_group(const spgemm_plan* plan, const int64_t* key, int32_t n, const int64_t* thr,
                 int32_t nthr, void* ws, size_t ws_bytes, int32_t* map, int32_t* offsets,
                 void* stream) {
    if (!plan || n < 0 || nthr < 0 || nthr > 32 || !offsets) return SPGEMM_ERR_INVALID;
    if (n > 0 && (!key || !map)) return SPGEMM_ERR_INVALID;
    if (nthr > 0 && !thr) return SPGEMM_ERR_INVALID;
    WsLayout L = ws_layout(plan, n, 0, 0);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws & 255)) return SPGEMM_ERR_WORKSPACE;
    WsPtrs w = ws_ptrs(L, ws, plan->opts.panel_cols);
    GroupArgs g{};
    g.phase = 2;
    g.n = n;
    g.key = (const long long*)key;
    g.thr = (const long long*)thr;
    g.nthr = nthr;
    g.opts = plan->opts;
    launch_group(plan, g, w, map, offsets, (cudaStream_t)stream);
    return cuda_err(cudaGetLastError());
}

int spgemm_symbolic(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B,
                    const int64_t* ip_row, void* ws, size_t ws_bytes, int32_t* row_nnz,
                    int64_t* nnz_total, void* stream) {
    int rc = check_pair(plan, A, B, false);
    if (rc) return rc;
    if (A->rows > 0 && (!ip_row || !row_nnz)) return SPGEMM_ERR_INVALID;
    WsLayout L;
    rc = check_ws(plan, A, B, ws, ws_bytes, &L);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(L, ws, plan->opts.panel_cols);
    CsrDev dA = dev_view(A), dB = dev_view(B);
    launch_symbolic(plan, dA, dB, (const long long*)ip_row, w, row_nnz, s);
    launch_bpanel(plan, dB, w, s);
    launch_hot(plan, dB, w, s);
    launch_nnz_total(plan, row_nnz, A->rows, w, s);
    rc = cuda_err(cudaGetLastError());
    if (rc) return rc;
    if (nnz_total) return sync_read(w.ctl, 1, nnz_total, s);
    return SPGEMM_OK;
}

int spgemm_row_ptr(const spgemm_plan* plan, const int32_t* row_nnz, int32_t n, void* ws,
                   size_t ws_bytes, int32_t* row_ptr, int64_t* total, void* stream) {
    if (!plan || n < 0 || !row_ptr || (n > 0 && !row_nnz)) return SPGEMM_ERR_INVALID;
    WsLayout L = ws_layout(plan, n, 0, 0);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws & 255)) return SPGEMM_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(L, ws, plan->opts.panel_cols);
    launch_row_ptr(plan, row_nnz, n, w, row_ptr, s);
    int rc = cuda_err(cudaGetLastError());
    if (rc) return rc;
    if (total) return sync_read(w.ctl, 2, total, s);
    return SPGEMM_OK;
}

int spgemm_numeric(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B,
                   const int64_t* ip_row, int32_t row_begin, int32_t row_end,
                   const int32_t* row_ptr_C, void* ws, size_t ws_bytes, int32_t* col_C,
                   float* val_C, void* stream) {
    int rc = check_pair(plan, A, B, true);
    if (rc) return rc;
    if (row_begin < 0 || row_end < row_begin || row_end > A->rows) return SPGEMM_ERR_INVALID;
    if (row_end > row_begin && (!ip_row || !row_ptr_C)) return SPGEMM_ERR_INVALID;
    WsLayout L;
    rc = check_ws(plan, A, B, ws, ws_bytes, &L);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(L, ws, plan->opts.panel_cols);
    launch_numeric(plan, dev_view(A), dev_view(B), (const long long*)ip_row, row_begin, row_end,
                   row_ptr_C, w, col_C, val_C, s);
    return cuda_err(cudaGetLastError());
}

int spgemm(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B, void* ws,
           size_t ws_bytes, int64_t* ip_row, int32_t* row_nnz, int32_t* row_ptr_C,
           spgemm_alloc_fn alloc, void* alloc_ctx, int64_t* nnz_C, void* stream) {
    int rc = check_pair(plan, A, B, true);
    if (rc) return rc;
    if (!alloc || !nnz_C || !row_ptr_C) return SPGEMM_ERR_INVALID;
    rc = spgemm_workspace_init(plan, ws, ws_bytes, stream);
    if (rc) return rc;
    rc = spgemm_count(plan, A, B, ws, ws_bytes, ip_row, nullptr, stream);
    if (rc) return rc;
    int64_t total = 0;
    rc = spgemm_symbolic(plan, A, B, ip_row, ws, ws_bytes, row_nnz, &total, stream);
    if (rc) return rc;
    *nnz_C = total;
    if (total > 2147483647ll) return SPGEMM_ERR_OVERFLOW;
    rc = spgemm_row_ptr(plan, row_nnz, A->rows, ws, ws_bytes, row_ptr_C, nullptr, stream);
    if (rc) return rc;
    int32_t* col = nullptr;
    float* val = nullptr;
    if (alloc(alloc_ctx, total, &col, &val) != 0) return SPGEMM_ERR_BUDGET;
    if (total > 0 && (!col || !val)) return SPGEMM_ERR_BUDGET;
    rc = spgemm_numeric(plan, A, B, ip_row, 0, A->rows, row_ptr_C, ws, ws_bytes, col, val, stream);
    if (rc) return rc;
    WsLayout L = ws_layout(plan, A->rows, B->rows, B->cols, B->nnz);
    return sync_read(ws_ptrs(L, ws, plan->opts.panel_cols).ctl, -1, nullptr, (cudaStream_t)stream);
}

int spgemm_batched(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B, void* ws,
                   size_t ws_bytes, int64_t* ip_row, int32_t* row_nnz, int32_t* row_ptr_C,
                   int32_t* col_C, float* val_C, int64_t capacity, int64_t* nnz_C, void* stream) {
    int rc = check_pair(plan, A, B, true);
    if (rc) return rc;
    if (capacity < 0 || capacity > 2147483647ll) return SPGEMM_ERR_INVALID;
    if (!nnz_C || !row_ptr_C) return SPGEMM_ERR_INVALID;
    if (A->rows > 0 && (!ip_row || !row_nnz)) return SPGEMM_ERR_INVALID;
    if (capacity > 0 && (!col_C || !val_C)) return SPGEMM_ERR_INVALID;
    WsLayout L;
    rc = check_ws(plan, A, B, ws, ws_bytes, &L);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(L, ws, plan->opts.panel_cols);
    CsrDev dA = dev_view(A), dB = dev_view(B);
    launch_ip_count(plan, dA, dB, (long long*)ip_row, w, s);
    launch_symbolic(plan, dA, dB, (const long long*)ip_row, w, row_nnz, s);
    launch_bpanel(plan, dB, w, s);
    launch_hot(plan, dB, w, s);
    launch_row_ptr(plan, row_nnz, A->rows, w, row_ptr_C, s);
    launch_copy_total(plan, w, 2, (long long*)nnz_C, s);
    launch_numeric(plan, dA, dB, (const long long*)ip_row, 0, A->rows, row_ptr_C, w, col_C, val_C,
                   s, capacity);
    return cuda_err(cudaGetLastError());
}

static size_t backward_ws_bytes(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B,
                                WsLayout* L) {
    *L = ws_layout(plan, A->rows, B->rows, B->cols);
    return L->total + backward_extra_bytes(A->nnz, B->nnz);
}

int spgemm_backward_workspace_bytes(const spgemm_plan* plan, const spgemm_csr* A,
                                    const spgemm_csr* B, size_t* bytes) {
    if (!plan || !A || !B || !bytes) return SPGEMM_ERR_INVALID;
    if (A->rows < 0 || B->rows < 0 || B->cols < 0 || A->nnz < 0 || B->nnz < 0)
        return SPGEMM_ERR_INVALID;
    WsLayout L;
    *bytes = backward_ws_bytes(plan, A, B, &L);
    return SPGEMM_OK;
}

int spgemm_backward(const spgemm_plan* plan, const spgemm_csr* A, const spgemm_csr* B,
                    const int32_t* row_ptr_C, const int32_t* col_C, int64_t nnz_C,
                    const float* dC, float* dA, float* dB, void* ws, size_t ws_bytes,
                    void* stream) {
    int rc = check_pair(plan, A, B, true);
    if (rc) return rc;
    if (nnz_C < 0 || nnz_C > 2147483647ll) return SPGEMM_ERR_INVALID;
    if (A->rows > 0 && !row_ptr_C) return SPGEMM_ERR_INVALID;
    if (nnz_C > 0 && (!col_C || !dC)) return SPGEMM_ERR_INVALID;
    if (A->nnz > 0 && dA == nullptr && dB == nullptr) return SPGEMM_OK;
    WsLayout L;
    const size_t need = backward_ws_bytes(plan, A, B, &L);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) return SPGEMM_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(L, ws, plan->opts.panel_cols);
    double* dB64 = (double*)((char*)ws + L.total);
    double* dA64 = dB64 + (B->nnz > 0 ? B->nnz : 1);
    launch_backward(plan, dev_view(A), dev_view(B), row_ptr_C, col_C, dC, dA, dB, w, dB64, dA64, s);
    return cuda_err(cudaGetLastError());
}

int spgemm_mcl_step(const spgemm_plan* plan, const spgemm_csr* E, float theta, int32_t k, float r,
                    int32_t order, void* ws, size_t ws_bytes, int32_t* row_ptr_out,
                    int32_t* col_out, float* val_out, int64_t* nnz_out, void* stream) {
    if (!plan) return SPGEMM_ERR_INVALID;
    int rc = check_csr(E, true);
    if (rc) return rc;
    if (!row_ptr_out || (order != 0 && order != 1) || !(r > 0.f)) return SPGEMM_ERR_INVALID;
    if (E->nnz > 0 && (!col_out || !val_out)) return SPGEMM_ERR_INVALID;
    WsLayout L = ws_layout(plan, E->rows, 0, 0);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws & 255)) return SPGEMM_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(L, ws, plan->opts.panel_cols);
    launch_mcl_step(plan, dev_view(E), theta, k, (double)r, order, w, row_ptr_out, col_out, val_out,
                    s);
    rc = cuda_err(cudaGetLastError());
    if (rc) return rc;
    if (nnz_out) return sync_read(w.ctl, 2, nnz_out, s);
    return SPGEMM_OK;
}

int spgemm_topk_dense(const spgemm_plan* plan, const float* X, int32_t n, int32_t d, int64_t ldx,
                      int32_t k, int32_t* row_ptr, int32_t* col, float* val, void* stream) {
    if (!plan || n < 0 || d < 0 || k < 0 || ldx < d || !row_ptr) return SPGEMM_ERR_INVALID;
    if (n > 0 && d > 0 && !X) return SPGEMM_ERR_INVALID;
    const long long kk = k < d ? k : d;
    if ((long long)n * kk > 2147483647ll) return SPGEMM_ERR_OVERFLOW;
    if ((long long)n * kk > 0 && (!col || !val)) return SPGEMM_ERR_INVALID;
    launch_topk(plan, X, n, d, (long long)ldx, k, row_ptr, col, val, (cudaStream_t)stream);
    return cuda_err(cudaGetLastError());
}

int spgemm_csr_scatter_dense(const spgemm_plan* plan, const spgemm_csr* M, const float* vals,
                             float* X, int64_t ldx, void* ws, size_t ws_bytes, void* stream) {
    if (!plan) return SPGEMM_ERR_INVALID;
    int rc = check_csr(M, vals == nullptr);
    if (rc) return rc;
    if (ldx < M->cols || (M->rows > 0 && M->cols > 0 && !X)) return SPGEMM_ERR_INVALID;
    if (!ws || ws_bytes < sizeof(Ctl) || ((uintptr_t)ws & 255)) return SPGEMM_ERR_WORKSPACE;
    launch_scatter_dense(plan, dev_view(M), vals ? vals : M->vals, X, (long long)ldx, (Ctl*)ws,
                         (cudaStream_t)stream);
    return cuda_err(cudaGetLastError());
}

int spgemm_csr_gather_dense(const spgemm_plan* plan, const spgemm_csr* M, const float* D,
                            int64_t ldd, float* out, void* ws, size_t ws_bytes, void* stream) {
    if (!plan) return SPGEMM_ERR_INVALID;
    int rc = check_csr(M, false);
    if (rc) return rc;
    if (ldd < M->cols || (M->rows > 0 && M->cols > 0 && !D) || (M->nnz > 0 && !out))
        return SPGEMM_ERR_INVALID;
    if (!ws || ws_bytes < sizeof(Ctl) || ((uintptr_t)ws & 255)) return SPGEMM_ERR_WORKSPACE;
    launch_gather_dense(plan, dev_view(M), D, (long long)ldd, out, (Ctl*)ws, (cudaStream_t)stream);
    return cuda_err(cudaGetLastError());
}

int spgemm_sample_rows(const spgemm_plan* plan, const spgemm_csr* P, int32_t s, const float* u,
                       int32_t mode, void* ws, size_t ws_bytes, int32_t* row_ptr_Q,
                       int32_t* col_Q, float* val_Q, int64_t* nnz_Q, void* stream) {
    if (!plan) return SPGEMM_ERR_INVALID;
    int rc = check_csr(P, mode != 0);
    if (rc) return rc;
    if (s < 1 || s > 32) return SPGEMM_ERR_UNSUPPORTED;
    if (mode < 0 || mode > 2 || !row_ptr_Q) return SPGEMM_ERR_INVALID;
    if (P->rows > 0 && (!u || !col_Q || !val_Q)) return SPGEMM_ERR_INVALID;
    WsLayout L = ws_layout(plan, P->rows, 0, 0);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws & 255)) return SPGEMM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(L, ws, plan->opts.panel_cols);
    launch_sample_rows(plan, dev_view(P), s, u, mode, w, row_ptr_Q, col_Q, val_Q, st);
    rc = cuda_err(cudaGetLastError());
    if (rc) return rc;
    if (nnz_Q) return sync_read(w.ctl, 2, nnz_Q, st);
    return SPGEMM_OK;
}

int spgemm_select_columns(const spgemm_plan* plan, const spgemm_csr* Q, void* ws, size_t ws_bytes,
                          int32_t* S_row_ptr, int32_t* S_col, float* S_val, int32_t* F_row_ptr,
                          int32_t* F_col, float* F_val, int64_t* m, void* stream) {
    if (!plan) return SPGEMM_ERR_INVALID;
    int rc = check_csr(Q, false);
    if (rc) return rc;
    if (!S_row_ptr || !F_row_ptr) return SPGEMM_ERR_INVALID;
    if (Q->cols > 0 && (!S_col || !S_val || !F_col || !F_val)) return SPGEMM_ERR_INVALID;
    WsLayout L = ws_layout(plan, Q->cols, 0, 0);
    if (!ws || ws_bytes < L.total || ((uintptr_t)ws & 255)) return SPGEMM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(L, ws, plan->opts.panel_cols);
    launch_select_columns(plan, dev_view(Q), w, S_row_ptr, S_col, S_val, F_row_ptr, F_col, F_val,
                          st);
    rc = cuda_err(cudaGetLastError());
    if (rc) return rc;
    if (m) return sync_read(w.ctl, 2, m, st);
    return SPGEMM_OK;
}

int spgemm_status(const spgemm_plan* plan, void* ws, void* stream, int* status) {
    if (!plan || !ws || !status) return SPGEMM_ERR_INVALID;
    *status = sync_read((Ctl*)ws, -1, nullptr, (cudaStream_t)stream);
    return *status == SPGEMM_ERR_CUDA ? SPGEMM_ERR_CUDA : SPGEMM_OK;
}

const char* spgemm_status_string(int st) {
    switch (st) {
        case SPGEMM_OK: return "ok";
        case SPGEMM_ERR_INVALID: return "invalid argument or malformed CSR input";
        case SPGEMM_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case SPGEMM_ERR_OVERFLOW: return "result exceeds int32 row pointers; split A into row blocks";
        case SPGEMM_ERR_BUDGET: return "memory budget exceeded or allocation refused";
        case SPGEMM_ERR_TIMEOUT: return "bounded device wait gave up";
        case SPGEMM_ERR_CUDA: return "CUDA runtime error";
        case SPGEMM_ERR_INTERNAL: return "internal capacity guard tripped";
        case SPGEMM_ERR_UNSUPPORTED: return "unsupported shape";
        default: return "unknown status";
    }
}

}  // extern "C"

// Status strings, per-thread error detail and small shared host utilities of the C ABI.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace cst {

namespace {
thread_local char g_detail[512] = "";
std::atomic<long long> g_launches{0};
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int fail(int status, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
    va_end(ap);
    return status;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(CSTONE_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

int sm_count() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 152;
    static thread_local int cached_dev = -1, cached = 0;
    if (dev != cached_dev) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
        cached = v;
        cached_dev = dev;
    }
    return cached;
}

int cooperative_grid(const void* kernel, int threads, size_t smem, int cap_per_sm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    if (per_sm > cap_per_sm) per_sm = cap_per_sm;
    return sm_count() * per_sm;
}

int check_ws(void* ws, size_t have, size_t need, const char* who) {
    if (ws == nullptr || have < need)
        return fail(CSTONE_ERR_INVALID_ARG, "%s: workspace of %zu bytes given, %zu needed", who, have, need);
    if (!aligned256(ws)) return fail(CSTONE_ERR_INVALID_ARG, "%s: workspace must be 256-byte aligned", who);
    return CSTONE_OK;
}

}  // namespace cst

extern "C" {

const char* cstone_status_string(int status) {
    switch (status) {
        case CSTONE_OK: return "ok";
        case CSTONE_ERR_INVALID_ARG: return "invalid argument";
        case CSTONE_ERR_CUDA: return "CUDA error";
        case CSTONE_ERR_CAPACITY: return "output capacity exceeded";
        case CSTONE_ERR_TIMEOUT: return "device wait timed out";
        case CSTONE_ERR_NOT_CONVERGED: return "rebalance loop did not converge";
        default: return "unknown status";
    }
}

int cstone_last_error_detail(char* buf, size_t len) {
    if (buf && len) {
        strncpy(buf, cst::g_detail, len - 1);
        buf[len - 1] = '\0';
    }
    return CSTONE_OK;
}

int cstone_version(void) { return 100; }

int64_t cstone_kernel_launches(void) { return cst::g_launches.load(std::memory_order_relaxed); }

int cstone_workspace_status(const void* ws, void* stream, int* status) {
    if (!ws || !status) return cst::fail(CSTONE_ERR_INVALID_ARG, "cstone_workspace_status: NULL argument");
    cst::WsHeader h;
    CST_CUDA(cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, cst::as_stream(stream)));
    CST_CUDA(cudaStreamSynchronize(cst::as_stream(stream)));
    *status = static_cast<int>(h.err);
    if (h.err) cst::fail(static_cast<int>(h.err), "device error word %u (info %u)", h.err, h.err_info);
    return CSTONE_OK;
}

}  // extern "C"

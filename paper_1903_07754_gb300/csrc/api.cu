// Error reporting, pointer classification and small ABI helpers.
#include <atomic>
#include <cstdio>
#include <string>

#include "common.cuh"

namespace wedge {

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_launches{0};

wedge_status set_error(wedge_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

wedge_status cuda_error(cudaError_t e, const char* what) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s failed: %s (%d)", what, cudaGetErrorString(e), (int)e);
    g_last_error = buf;
    if (e == cudaErrorMemoryAllocation) return WEDGE_ERR_OUT_OF_MEMORY;
    return WEDGE_ERR_CUDA;
}

void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

wedge_status dev_alloc(wedge_graph* g, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_error(e, "cudaMalloc");
    }
    if (g) g->device_bytes += bytes;
    return WEDGE_OK;
}

void dev_free(void* p) {
    if (p) cudaFree(p);
}

PtrKind classify(const void* p) {
    if (!p) return PtrKind::Invalid;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PtrKind::Host;
    }
    switch (a.type) {
        case cudaMemoryTypeDevice:
        case cudaMemoryTypeManaged:
            return PtrKind::Device;
        default:
            return PtrKind::Host;
    }
}

}  // namespace wedge

extern "C" {

const char* wedge_last_error(void) { return wedge::g_last_error.c_str(); }

const char* wedge_version(void) { return WEDGE_VERSION_STRING; }

uint64_t wedge_kernel_launches(void) { return wedge::g_launches.load(); }

void wedge_default_opts(wedge_app app, wedge_opts* out) {
    if (!out) return;
    *out = wedge_opts{};
    out->switch_mode = WEDGE_SWITCH_THRESHOLD;
    if (app == WEDGE_BFS) {
        out->tau_bp = 100;     // 1% of edges
        out->log2_coarsen = 3; // 256 edges per Wedge bit
    } else {
        out->tau_bp = 2000;    // 20%
        out->log2_coarsen = 2; // 128 edges per Wedge bit
    }
    out->max_iters = 0;
    out->trace = 0;
}

}  // extern "C"

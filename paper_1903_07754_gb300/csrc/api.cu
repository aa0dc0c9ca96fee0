// Error reporting, pointer classification and small ABI helpers.
#include <atomic>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

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

// Device memory comes from one library-owned memory pool per GPU that keeps
// what graphs release (release threshold: never), so creating a graph after
// destroying one maps no new memory.  Allocation and release are ordered on
// a private stream and completed before returning: callers see ordinary
// cudaMalloc / cudaFree semantics, including release only after all device
// work has finished.
namespace {
constexpr int kMaxDevices = 64;
struct DevPool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream = nullptr;
};
std::mutex g_pool_mu;
DevPool g_pools[kMaxDevices];

cudaError_t device_pool(int dev, DevPool** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    DevPool& d = g_pools[dev];
    if (!d.pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&d.pool, &props);
        if (e != cudaSuccess) {
            d.pool = nullptr;
            return e;
        }
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(d.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&d.stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(d.pool);
            d.pool = nullptr;
            return e;
        }
    }
    *out = &d;
    return cudaSuccess;
}
}  // namespace

wedge_status dev_alloc(wedge_graph* g, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    *p = nullptr;
    int dev = 0;
    DevPool* d = nullptr;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = device_pool(dev, &d);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, d->pool, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_error(e, "device allocation");
    }
    if (g) g->device_bytes += bytes;
    return WEDGE_OK;
}

// Stream-ordered free of scratch whose last use was enqueued on s: no
// device-wide wait, so work on other streams keeps running.
void dev_free_async(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

void dev_free(void* p) {
    if (!p) return;
    int dev = 0;
    DevPool* d = nullptr;
    if (cudaGetDevice(&dev) != cudaSuccess || device_pool(dev, &d) != cudaSuccess) return;
    cudaDeviceSynchronize();  // as cudaFree: nothing may still use p
    cudaFreeAsync(p, d->stream);
    cudaStreamSynchronize(d->stream);
}

// Small pinned host blocks (the control-block mirrors that runs read back)
// come from 16 KiB slabs kept for the life of the process: page-locking
// memory per graph would cost more than the rest of a small graph's setup.
namespace {
constexpr size_t kPinnedBlock = 256;
constexpr int kPinnedPerSlab = 64;
std::mutex g_pin_mu;
std::vector<void*> g_pin_free;
}  // namespace

void* pinned_small_alloc(size_t bytes) {
    if (bytes > kPinnedBlock) return nullptr;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        void* slab = nullptr;
        if (cudaMallocHost(&slab, kPinnedBlock * kPinnedPerSlab) != cudaSuccess) return nullptr;
        for (int i = kPinnedPerSlab - 1; i >= 0; --i) g_pin_free.push_back(static_cast<char*>(slab) + kPinnedBlock * i);
    }
    void* p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}

void pinned_small_free(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

wedge_status trim_pools(int device) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (int i = 0; i < kMaxDevices; ++i) {
        if (device >= 0 && i != device) continue;
        if (!g_pools[i].pool) continue;
        cudaError_t e = cudaStreamSynchronize(g_pools[i].stream);
        if (e == cudaSuccess) e = cudaMemPoolTrimTo(g_pools[i].pool, 0);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemPoolTrimTo");
    }
    return WEDGE_OK;
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

wedge_status wedge_trim_memory(int device) {
    if (device < -1) return wedge::set_error(WEDGE_ERR_INVALID_ARG, "device must be >= -1");
    return wedge::trim_pools(device);
}

void wedge_default_opts(wedge_app app, wedge_opts* out) {
    if (!out) return;
    *out = wedge_opts{};
    out->switch_mode = WEDGE_SWITCH_THRESHOLD;
    if (app == WEDGE_BFS) {
        out->tau_bp = 100;     // 1% of edges
        out->log2_coarsen = 0; // 8 edge vectors of <= 4 edges: one 32-edge chunk
    } else {
        out->tau_bp = 2000;    // 20%
        out->log2_coarsen = 0xFFFFFFFFu; // -1: 4 vectors of <= 4 edges, 16-edge entries
    }
    out->max_iters = 0;
    out->trace = 0;
}

}  // extern "C"

// Frontier transformation that allocates no memory.
//
// Some callers cannot call cudaMalloc: a host framework that owns every byte
// of device memory through its own pool and forbids outside allocations,
// latency-critical loops where an allocation (and the device
// synchronisation it can imply) is not acceptable, and deployments whose
// device footprint must be fixed when the library is loaded.  For them this
// entry point runs the transformation of Sections 3.3 and 4 on arrays the
// caller already owns (edge index, vertex bitmap, output list and count) and
// keeps its only scratch, the Wedge Frontier bitmap that removes duplicate
// entries, in a fixed file-scope device array.
//
// The array holds kNoAllocWords 32-bit words (4 MiB) on every GPU that loads
// the library, for as long as the process runs.  Every call on a device uses
// the same array: calls whose work overlaps on the GPU (different streams
// without ordering) race on it.  Each call clears the words it will use
// before using them.
#include <mutex>

#include "common.cuh"

namespace wedge {

constexpr uint32_t kNoAllocWords = 1u << 20;  // 4 MiB: up to 2^25 Wedge Frontier entries
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint32_t g_noalloc_bitmap[kNoAllocWords];

static std::mutex g_noalloc_mutex;
static uint32_t* g_noalloc_ptr[kMaxDevices];

// Device address of the scratch array on the current device, looked up once
// per device (in host code the symbol itself is only a host-side stand-in).
static wedge_status noalloc_scratch(uint32_t** out) {
    int dev = 0;
    WEDGE_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(WEDGE_ERR_NOT_SUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_bitmap);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return WEDGE_OK;
}

__global__ void k_noalloc_clear(uint32_t* __restrict__ bits, uint32_t words, uint32_t* __restrict__ count) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x) bits[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = 0u;
}

// One warp per group of 32 bitmap words: the warp walks the edge-index row
// of every active vertex in its words, 32 entries at a time, sets the entry's
// bit and appends the entries it set first.  Entries >= nbits are skipped.
__global__ void k_noalloc_transform(const uint32_t* __restrict__ eidx_off, const uint32_t* __restrict__ eidx,
                                    const uint32_t* __restrict__ vbm, uint32_t V, uint32_t k, uint32_t nbits,
                                    uint32_t* __restrict__ bits, uint32_t* __restrict__ list,
                                    uint32_t* __restrict__ count) {
    const unsigned full = 0xFFFFFFFFu;
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const uint64_t words = ((uint64_t)V + 31) / 32;
    const uint64_t gw = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t base = gw * 32; base < words; base += nw * 32) {
        const uint64_t wi = base + lane;
        uint32_t word = wi < words ? vbm[wi] : 0u;
        if (wi == words - 1 && (V & 31)) word &= (1u << (V & 31)) - 1u;
        // visit the set bits of the 32 words one vertex at a time
        for (unsigned pending = __ballot_sync(full, word != 0); pending; pending = __ballot_sync(full, word != 0)) {
            const unsigned src_lane = __ffs(pending) - 1;
            const uint32_t w = __shfl_sync(full, word, src_lane);
            const uint32_t u = (uint32_t)((base + src_lane) * 32 + (__ffs(w) - 1));
            if (lane == src_lane) word &= word - 1;
            const uint32_t rb = eidx_off[u], re = eidx_off[u + 1];
            for (uint32_t j0 = rb; j0 < re; j0 += 32) {
                const uint32_t j = j0 + lane;
                bool fresh = false;
                uint32_t b = 0;
                if (j < re) {
                    b = eidx[j] >> k;
                    if (b < nbits) {
                        const uint32_t bit = 1u << (b & 31);
                        fresh = (atomicOr(bits + (b >> 5), bit) & bit) == 0;
                    }
                }
                const unsigned m = __ballot_sync(full, fresh);
                if (m) {
                    const unsigned leader = __ffs(m) - 1;
                    uint32_t slot = 0;
                    if (lane == leader) slot = atomicAdd(count, (uint32_t)__popc(m));
                    slot = __shfl_sync(full, slot, leader);
                    if (fresh) list[slot + __popc(m & lt)] = b;
                }
            }
        }
    }
}

}  // namespace wedge

using namespace wedge;

extern "C" wedge_status wedge_frontier_transform_noalloc(uint32_t V, uint64_t E, const uint32_t* d_eidx_off,
                                                         const uint32_t* d_eidx, const uint32_t* d_vertex_bitmap,
                                                         uint32_t log2_coarsen, uint32_t* d_chunk_list,
                                                         uint32_t* d_chunk_count, wedge_stream_t stream) {
    if (!d_eidx_off || !d_vertex_bitmap || !d_chunk_list || !d_chunk_count)
        return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (V == 0) return set_error(WEDGE_ERR_INVALID_ARG, "V must be >= 1");
    if (log2_coarsen > kMaxCoarsen) return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be <= 7");
    const uint64_t nc = (E + kChunk - 1) / kChunk;
    const uint64_t nbits = (nc + (1ull << log2_coarsen) - 1) >> log2_coarsen;
    const uint64_t words = (nbits + 31) / 32;
    if (words > kNoAllocWords)
        return set_error(WEDGE_ERR_INVALID_ARG,
                         "graph too large for the fixed scratch: ceil(ceil(E/32) / 2^log2_coarsen) must be <= 2^25");
    if (nbits && !d_eidx) return set_error(WEDGE_ERR_INVALID_ARG, "eidx is NULL");
    uint32_t* bits = nullptr;
    WEDGE_TRY(noalloc_scratch(&bits));
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0, dev = 0;
    WEDGE_TRY_CUDA(cudaGetDevice(&dev));
    WEDGE_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    k_noalloc_clear<<<sms * 2, 256, 0, s>>>(bits, (uint32_t)words, d_chunk_count);
    k_noalloc_transform<<<sms * 4, 256, 0, s>>>(d_eidx_off, d_eidx, d_vertex_bitmap, V, log2_coarsen,
                                                 (uint32_t)nbits, bits, d_chunk_list, d_chunk_count);
    count_launch(2);
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

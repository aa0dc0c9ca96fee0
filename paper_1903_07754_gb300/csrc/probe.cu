// A diagnostic kernel beside the engine: the dense pull's memory access
// pattern without its arithmetic, to measure the ceiling that pattern sets
// on this GPU (declared in include/wedge.h).
#include "common.cuh"
#include "tma.cuh"

namespace wedge {

constexpr unsigned kFullMask = 0xFFFFFFFFu;

// Diagnostic: the dense pull's stream and gathers alone.  Warp slices of
// 256 sources, lane = 8 consecutive sources (two 16-byte loads, the next
// slice in flight), one 4-byte gather per source, summed per warp into
// *sink (the sum only keeps the loads alive).
__global__ void __launch_bounds__(kCW * 32, 4)
    k_gather_probe(const uint32_t* __restrict__ src, unsigned long long E, const float* __restrict__ vals,
                   float* sink) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long nw = (unsigned long long)gridDim.x * kCW;
    const unsigned long long nslices = (E + kSliceE - 1) / kSliceE;
    float acc = 0.f;
    uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a;
    auto load = [&](unsigned long long sl) {
        const unsigned long long e = sl * kSliceE + lane * kEPL;
        a = make_uint4(0u, 0u, 0u, 0u);
        b = a;
        if (e + kEPL <= E) {
            a = ld_stream(src + e);
            b = ld_stream(src + e + 4);
        }
    };
    unsigned long long sl = (unsigned long long)blockIdx.x * kCW + (threadIdx.x >> 5);
    if (sl < nslices) load(sl);
    for (; sl < nslices; sl += nw) {
        const uint32_t u[kEPL] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        const unsigned long long e = sl * kSliceE + lane * kEPL;
        const int nv = e + kEPL <= E ? kEPL : (e < E ? (int)(E - e) : 0);
        uint32_t tail[kEPL];
#pragma unroll
        for (int i = 0; i < kEPL; ++i) tail[i] = (nv < kEPL && i < nv) ? src[e + i] : 0u;
        if (sl + nw < nslices) load(sl + nw);
#pragma unroll
        for (int i = 0; i < kEPL; ++i)
            if (i < nv) acc += __ldg(vals + (nv == kEPL ? u[i] : tail[i]));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(kFullMask, acc, d);
    if (lane == 0) atomicAdd(sink, acc);
}

}  // namespace wedge

using namespace wedge;

extern "C" {

wedge_status wedge_gather_probe(wedge_graph_t g, const float* d_vals, float* d_sink, wedge_stream_t stream) {
    if (!g || !d_vals || !d_sink) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    // the PageRank pull's launch shape: 4 resident 256-thread blocks per SM
    k_gather_probe<<<g->num_sms * 4, kCW * 32, 0, s>>>(g->src, g->E, d_vals, d_sink);
    count_launch();
    WEDGE_TRY_CUDA(cudaGetLastError());
    g->last_stream = s;
    return WEDGE_OK;
}

}  // extern "C"

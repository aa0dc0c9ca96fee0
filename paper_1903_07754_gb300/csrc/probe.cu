// A measurement tool beside the engine, built into its own library
// (libwedge_probe.so, declared in include/wedge_probe.h), not into
// libwedge.so: the dense pull's memory access pattern without its
// arithmetic, to measure the ceiling that pattern sets on this GPU.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wedge_probe.h"
#include "tma.cuh"

namespace {

// The dense pull's launch shape: 8 warps per block, a warp slice of 256
// sources, 8 consecutive sources per lane.
constexpr int kWarps = 8;
constexpr int kPerLane = 8;
constexpr int kSlice = 32 * kPerLane;
constexpr unsigned kFullMask = 0xFFFFFFFFu;

// The stream and the gathers alone: lane = 8 consecutive sources (two
// 16-byte loads, the next slice in flight), one 4-byte gather per source,
// summed per warp into *sink (the sum only keeps the loads alive).
__global__ void __launch_bounds__(kWarps * 32, 4)
    k_gather_probe(const uint32_t* __restrict__ src, unsigned long long E, const float* __restrict__ vals,
                   float* sink) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long nw = (unsigned long long)gridDim.x * kWarps;
    const unsigned long long nslices = (E + kSlice - 1) / kSlice;
    float acc = 0.f;
    uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a;
    auto load = [&](unsigned long long sl) {
        const unsigned long long e = sl * kSlice + lane * kPerLane;
        a = make_uint4(0u, 0u, 0u, 0u);
        b = a;
        if (e + kPerLane <= E) {
            a = wedge::ld_stream(src + e);
            b = wedge::ld_stream(src + e + 4);
        }
    };
    unsigned long long sl = (unsigned long long)blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (sl < nslices) load(sl);
    for (; sl < nslices; sl += nw) {
        const uint32_t u[kPerLane] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        const unsigned long long e = sl * kSlice + lane * kPerLane;
        const int nv = e + kPerLane <= E ? kPerLane : (e < E ? (int)(E - e) : 0);
        uint32_t tail[kPerLane];
#pragma unroll
        for (int i = 0; i < kPerLane; ++i) tail[i] = (nv < kPerLane && i < nv) ? src[e + i] : 0u;
        if (sl + nw < nslices) load(sl + nw);
#pragma unroll
        for (int i = 0; i < kPerLane; ++i)
            if (i < nv) acc += __ldg(vals + (nv == kPerLane ? u[i] : tail[i]));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(kFullMask, acc, d);
    if (lane == 0) atomicAdd(sink, acc);
}

}  // namespace

extern "C" {

int wedge_probe_gather(const uint32_t* d_src, uint64_t E, const float* d_vals, float* d_sink,
                       uint32_t blocks_per_sm, void* stream) {
    if (!d_vals || !d_sink || (E && !d_src) || blocks_per_sm == 0 || blocks_per_sm > 32 ||
        (reinterpret_cast<uintptr_t>(d_src) & 15u))
        return (int)cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    if (E == 0) return 0;
    k_gather_probe<<<sms * blocks_per_sm, kWarps * 32, 0, (cudaStream_t)stream>>>(d_src, E, d_vals, d_sink);
    return (int)cudaGetLastError();
}

}  // extern "C"

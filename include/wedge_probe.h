/*
 * wedge_probe.h - a measurement tool beside the Wedge engine
 * (libwedge_probe.so), not part of the engine's ABI (wedge.h) and not a
 * step of the method.
 *
 * The dense pull of Sections 2.1 and 3.2 streams the destination-sorted
 * in-edge sources and gathers one source value per edge.  This probe does
 * exactly that access pattern and nothing else: timed, it measures how fast
 * this GPU streams a given source order with one random 4-byte gather per
 * edge, the ceiling of a pull over that order without its per-destination
 * reduction.
 */
#ifndef WEDGE_PROBE_H
#define WEDGE_PROBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Streams d_src[0 .. E) (device, 16-byte aligned) the way a dense pull does
 * -- blocks of 8 warps, warp slices of 256 sources, lane = 8 consecutive
 * sources in two 16-byte loads with the next slice in flight, a grid of
 * blocks_per_sm (1..32) blocks per SM of the current device -- and adds
 * d_vals[d_src[e]] for every e into *d_sink (one float, device, atomically;
 * only the loads matter).  d_vals: max(d_src) + 1 floats (device); not
 * checked.  Asynchronous on stream (a cudaStream_t; NULL = legacy default).
 * Returns 0 (cudaSuccess) or a cudaError_t code: cudaErrorInvalidValue
 * (NULL pointer, unaligned d_src, blocks_per_sm out of range), or the
 * launch's error. */
int wedge_probe_gather(const uint32_t* d_src, uint64_t E, const float* d_vals, float* d_sink,
                       uint32_t blocks_per_sm, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* WEDGE_PROBE_H */

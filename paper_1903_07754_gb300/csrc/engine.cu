// The Wedge hot path on the device:
//   pull (dense over all chunks, or over the listed Wedge Frontier chunks)
//   with the frontier-fullness epilogue and the fullness decision taken by
//   its last block (Sections 3.2, 3.4, Fig. 5), the frontier transformation
//   (Sections 3.3, 4), PageRank, the run drivers for BFS, CC, SSSP and
//   PageRank (Section 5), and -- beyond the paper -- the learned switch's
//   in-loop inference, batched BFS/SSSP in one persistent launch, the
//   push/pull hybrid the paper compares against, synchronous CC/SSSP and a
//   self-test of the bounded waits.  The iteration loop runs on the device
//   inside a CUDA graph with a conditional while node (traced and
//   synchronous runs drive it from the host).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "common.cuh"
#include "mlp.cuh"
#include "pull.cuh"
#include "tma.cuh"
#include "xform.cuh"

namespace wedge {

// ------------------------------------------------------------------------
// The push/pull hybrid (a comparison engine, not Wedge): iterations the
// fullness test finds sparse push over the frontier's out-edges instead of
// pulling over a Wedge Frontier; dense ones are the same pull.  The loop
// body is k_xform_scan over the out-edge rows (it also prepares the
// iteration: clears the bitmap and record it fills), k_push_expand,
// k_hybrid_prepare (a dense iteration the push chose), k_pull: each kernel
// serves only its own kind of iteration, and the deciding blocks of the push
// and of the pull advance the iteration.
// ------------------------------------------------------------------------

// A dense iteration that follows a push in the same loop body: its
// preparation (k_xform_scan prepared the push's iteration).
__global__ void __launch_bounds__(kXformThreads) k_hybrid_prepare(const XformParams X) {
    const RunCtl* C = X.ctl;
    if (C->done) return;
    const unsigned it = C->it;
    if (X.rec[it].mode != 0) return;
    prepare_iteration(X, it, blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x,
                      (unsigned long long)gridDim.x * blockDim.x);
}

// Relaxes destination v over edge j (source Q.src[j]) in place; true if v
// joins the next frontier (its bit was not yet set).
template <int APP>
__device__ __forceinline__ bool push_relax(const PullParams& P, const PushParams& Q, uint32_t j, uint32_t v,
                                           unsigned it, uint32_t* next) {
    if constexpr (APP == kBFS) {
        if (*reinterpret_cast<volatile uint32_t*>(P.vals + v) != kInf) return false;
        if (atomicCAS(P.vals + v, kInf, it + 1) != kInf) return false;
        if (P.visk) {
            const uint32_t kid = __ldg(Q.kid_of + v);
            atomicOr(P.visk + (kid >> 5), 1u << (kid & 31));
        }
        return set_bit(next, v);
    } else {
        const uint32_t du = P.vals[__ldg(Q.src + j)];
        uint32_t c = du;
        if constexpr (APP == kSSSP) {
            if (du == kInf) return false;
            const unsigned long long sum = (unsigned long long)du + __ldg(Q.w + j);
            c = sum > kSat ? kSat : (uint32_t)sum;
        }
        if (c >= *reinterpret_cast<volatile uint32_t*>(P.vals + v)) return false;
        return c < atomicMin(P.vals + v, c) && set_bit(next, v);
    }
}

// One push iteration: the pieces are expanded like the transformation's
// (a warp task of up to 32 pieces, fewer when there are too few to give
// every warp a task), one out-edge per lane and round.
template <int APP>
__global__ void __launch_bounds__(kXformThreads) k_push_expand(const PullParams P, const PushParams Q) {
    __shared__ uint32_t s_list[kListCap];
    __shared__ unsigned long long s_F;
    __shared__ unsigned s_n, s_row, s_rmax, s_lcnt;
    RunCtl* C = P.ctl;
    if (C->done) return;
    const unsigned it = C->it;
    if (P.rec[it].mode == 0) return;  // a dense iteration: the pull serves it
    const unsigned n = P.rec[it].npieces;
    if (threadIdx.x == 0) {
        s_F = 0;
        s_n = 0;
        s_row = 0;
        s_rmax = 0;
        s_lcnt = 0;
        if (P.trace && blockIdx.x == 0) P.rec[it].t_pull0 = global_timer();
    }
    __syncthreads();
    uint32_t* next = P.bm[(it + 1) & 1];
    Stats st{0ull, 0u, 0u, 0u};
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long gw = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long per = (unsigned long long)n / nw;
    const unsigned ppt = per >= 32 ? 32u : (per < 1 ? 1u : (unsigned)per);
    for (unsigned long long base = gw * ppt; base < n; base += nw * ppt) {
        const unsigned long long idx = base + lane;
        const uint2 pc = (lane < ppt && idx < n) ? __ldcg(Q.pieces + idx) : make_uint2(0u, 0u);
        unsigned incl = pc.y;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, d);
            if (lane >= (unsigned)d) incl += y;
        }
        const unsigned total = __shfl_sync(kFull, incl, 31);
        const unsigned excl = incl - pc.y;
        for (unsigned e0 = 0; e0 < total; e0 += 32) {
            const unsigned e = e0 + lane;
            unsigned jx = 0;
#pragma unroll
            for (unsigned stp = 16; stp >= 1; stp >>= 1) {
                const unsigned cj = jx + stp;
                if (__shfl_sync(kFull, excl, cj) <= e) jx = cj;
            }
            const uint32_t j = __shfl_sync(kFull, pc.x, jx) + (e - __shfl_sync(kFull, excl, jx));
            bool act = false;
            uint32_t v = 0;
            if (e < total) {
                v = __ldg(Q.dst + j);
                act = push_relax<APP>(P, Q, j, v, it, next);
                if (act) count_active(P, v, st);
            }
            stage_list(act, v, &s_lcnt, s_list);
        }
    }
    finish_block<true>(P, it, st, &s_F, &s_n, &s_row, &s_rmax, &s_lcnt, s_list, reinterpret_cast<float*>(s_list));
}

// Initial frontier: size, fullness and edge-index work (the transformation
// derives its pieces from the bitmap), then the decision for pull 0.
__global__ void k_frontier_stats(const uint32_t* __restrict__ bm, uint32_t V, const uint32_t* __restrict__ outdeg,
                                 const uint32_t* __restrict__ eidx_off, IterRec* rec, RunCtl* C,
                                 const __nv_bfloat16* mlp, GraphFeat gf) {
    __shared__ __align__(16) unsigned char dsm_bytes[kDecideSmemBytes];
    float* dsm = reinterpret_cast<float*>(dsm_bytes);
    __shared__ unsigned long long s_F;
    __shared__ unsigned s_n, s_row, s_rmax, s_last;
    if (threadIdx.x == 0) {
        s_F = 0;
        s_n = 0;
        s_row = 0;
        s_rmax = 0;
    }
    __syncthreads();
    unsigned long long F = 0;
    unsigned n = 0, row = 0, rmax = 0;
    const unsigned long long words = ((unsigned long long)V + 31) / 32;
    for (unsigned long long wi = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; wi < words;
         wi += (unsigned long long)gridDim.x * blockDim.x) {
        uint32_t word = bm[wi];
        if (wi == words - 1 && (V & 31)) word &= (1u << (V & 31)) - 1u;
        for (; word; word &= word - 1) {
            const uint32_t u = (uint32_t)(wi * 32 + __ffs(word) - 1);
            F += outdeg[u];
            n += 1;
            const uint32_t len = eidx_off[u + 1] - eidx_off[u];
            row += len;
            rmax = max(rmax, len);
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        F += __shfl_down_sync(kFull, F, d);
        n += __shfl_down_sync(kFull, n, d);
        row += __shfl_down_sync(kFull, row, d);
        rmax = max(rmax, __shfl_down_sync(kFull, rmax, d));
    }
    if ((threadIdx.x & 31) == 0 && n) {
        atomicAdd(&s_F, F);
        atomicAdd(&s_n, n);
        atomicAdd(&s_row, row);
        atomicMax(&s_rmax, rmax);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_n) {
            atomicAdd(&rec->fullness, s_F);
            atomicAdd(&rec->nfront, s_n);
            atomicAdd(&rec->rowsum, s_row);
            atomicMax(&rec->rowmax, s_rmax);
        }
        __threadfence();
        s_last = atomicAdd(&C->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        decide_block(rec, C, 0, mlp, gf, dsm);
        if (threadIdx.x == 0) C->ticket = 0;
    }
}

// Run start: values, initial frontier F_0, records 0 and 1, control block.
__global__ void k_run_init(int app, uint32_t V, uint32_t root, uint32_t* vals, uint32_t* bm0, uint32_t* bm1,
                           uint32_t* wb, unsigned long long wb_words, IterRec* rec, RunCtl* C, RunCtl init,
                           uint32_t* list0, uint32_t* visk, unsigned long long visk_words) {
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
    if (app == kBFS)  // nothing visited: the root's own in-edges are pulled and find it set
        for (unsigned long long i = tid; i < visk_words; i += nth) visk[i] = 0u;
    for (unsigned long long v = tid; v < V; v += nth)
        vals[v] = (app == kCC) ? (uint32_t)v : ((uint32_t)v == root ? 0u : kInf);
    const unsigned long long words = ((unsigned long long)V + 31) / 32;
    for (unsigned long long i = tid; i < words; i += nth) {
        uint32_t w0 = 0;
        if (app == kCC) {
            w0 = kFull;
            if (i == words - 1 && (V & 31)) w0 = (1u << (V & 31)) - 1u;
        } else if ((root >> 5) == i) {
            w0 = 1u << (root & 31);
        }
        bm0[i] = w0;
        bm1[i] = 0u;
    }
    for (unsigned long long i = tid; i < wb_words; i += nth) wb[i] = 0u;
    if (blockIdx.x == 0) {
        if (threadIdx.x < 2 * sizeof(IterRec) / 4) reinterpret_cast<unsigned*>(rec)[threadIdx.x] = 0u;
        if (threadIdx.x == 0) *C = init;
        __syncthreads();
        if (threadIdx.x == 0 && app != kCC) {  // F_0 = {root} as a list as well
            list0[0] = root;
            rec[0].nlist = 1;
        }
    }
}


// ------------------------------------------------------------------------
// Batched BFS (not in the paper): up to 64 traversals at once with a 64-bit
// query mask per vertex (multi-source BFS: a source's frontier mask is the
// set of queries that reached it in the previous iteration).  The union of
// the queries' frontiers drives the fullness decision and the Wedge
// Frontier, so one pull serves all queries.  The whole loop runs in one
// persistent cooperative launch; phases are separated by a bounded grid
// barrier.
// ------------------------------------------------------------------------

// Data that blocks of this one launch write and later read back (frontier
// and seen masks, bitmaps, the Wedge list, work pieces) is read with
// ld.global.cg: L1 is not coherent across SMs inside a launch.
//
// Grid-wide barrier, two levels: blocks arrive on their group's counter (32
// blocks per group, counters 128 bytes apart), the last of each group on the
// top counter, and the last of all bumps the generation the others wait on.
// Layout of bar: [0] top count, [1] generation, [32*(1+g)] group g's count.
// Returns false (and records kStatusTimeout) if the generation does not
// move within kWaitNs.
constexpr unsigned kBarGroup = 32;
constexpr unsigned kBarWords = 32 * (1 + kMaxPullBlocks / kBarGroup);

__device__ bool grid_sync(unsigned* bar, unsigned* status) {
    __shared__ unsigned s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ok = 1;
        volatile unsigned* vgen = bar + 1;
        const unsigned g = *vgen;
        __threadfence();
        const unsigned grp = blockIdx.x / kBarGroup;
        const unsigned ngroups = (gridDim.x + kBarGroup - 1) / kBarGroup;
        const unsigned gsize = min(kBarGroup, gridDim.x - grp * kBarGroup);
        bool released = false;
        unsigned* gc = bar + 32 * (1 + grp);
        if (atomicAdd(gc, 1u) == gsize - 1) {
            atomicExch(gc, 0u);
            if (atomicAdd(bar, 1u) == ngroups - 1) {
                atomicExch(bar, 0u);
                __threadfence();
                atomicAdd(bar + 1, 1u);
                released = true;
            }
        }
        if (!released) {
            const unsigned long long t0 = gtimer();
            for (unsigned n = 1; *vgen == g; ++n) {
                if ((n & 127u) == 0 && gtimer() - t0 > kWaitNs) {
                    atomicOr(status, kStatusTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (*(volatile unsigned*)status & kStatusTimeout) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Self-test of the bounded waits: each kernel waits for something that
// never happens and must come back with kStatusTimeout.
//  kind 0: an mbarrier expecting two arrivals receives one.
//  kind 1: a grid barrier of two blocks where block 1 leaves without
//          arriving (an ordinary launch: block 1 simply exits).
__global__ void k_selftest_wait(int kind, unsigned* bar, unsigned* status) {
    if (kind == 0) {
        __shared__ __align__(8) uint64_t mb;
        if (threadIdx.x == 0) {
            mbar_init(&mb, 2);
            fence_mbar_init();
            mbar_arrive(&mb);
            mbar_wait(&mb, 0, status);
        }
    } else {
        if (blockIdx.x == 1) return;
        grid_sync(bar, status);
    }
}

__global__ void k_msbfs_clear(uint32_t V, unsigned long long* fb0, unsigned long long* fb1, unsigned long long* seen,
                              uint32_t* bm0, uint32_t* bm1, uint32_t* wb, unsigned long long wb_words, IterRec* rec,
                              RunCtl* C, RunCtl init, unsigned* bar) {
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long v = tid; v < V; v += nth) {
        fb0[v] = 0ull;
        fb1[v] = 0ull;
        seen[v] = 0ull;
    }
    const unsigned long long words = ((unsigned long long)V + 31) / 32;
    for (unsigned long long i = tid; i < words; i += nth) {
        bm0[i] = 0u;
        bm1[i] = 0u;
    }
    for (unsigned long long i = tid; i < wb_words; i += nth) wb[i] = 0u;
    for (unsigned long long i = tid; i < kBarWords; i += nth) bar[i] = 0u;
    if (blockIdx.x == 0) {
        if (threadIdx.x < 2 * sizeof(IterRec) / 4) reinterpret_cast<unsigned*>(rec)[threadIdx.x] = 0u;
        if (threadIdx.x == 0) *C = init;
    }
}

__global__ void k_msbfs_roots(const uint32_t* __restrict__ roots, const uint32_t* __restrict__ rq, uint32_t nroots,
                              uint32_t Q, unsigned long long* fb0, unsigned long long* seen, uint32_t* levels,
                              uint8_t* levels8, uint32_t* bm0) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nroots; i += gridDim.x * blockDim.x) {
        const uint32_t v = roots[i], q = rq[i];
        const unsigned long long bit = 1ull << q;
        atomicOr(fb0 + v, bit);
        atomicOr(seen + v, bit);
        if (levels8) levels8[(size_t)v * Q + q] = 0u;
        else levels[(size_t)v * Q + q] = 0u;
        atomicOr(bm0 + (v >> 5), 1u << (v & 31));
    }
}

// ---- Batched SSSP pull (multi-source Bellman-Ford; not in the paper) ----
// A warp takes one 32-edge chunk at a time and lane L holds query L (and
// L + 32 when there are more than 32 queries): distances are vertex-major,
// dist[v * Q + q], so a source's distances for all queries are one or two
// coalesced lines.  The chunk's edges are visited in order, eight at a time
// with their distance loads issued together; each destination's running
// minima are applied (atomicMin, only where they improve) when the chunk
// passes its last edge, and the queries that improved join the
// destination's next-frontier mask.
__device__ __forceinline__ void mssp_flush(const PullParams& P, uint32_t kid, uint32_t acc0, uint32_t acc1,
                                           unsigned long long* fnext, uint32_t* next, Stats& st, unsigned* s_lcnt,
                                           uint32_t* s_list) {
    const unsigned lane = threadIdx.x & 31;
    const bool a = acc0 != kInf, b = acc1 != kInf;
    if (!__any_sync(kFull, a || b)) return;
    const uint32_t dv = __ldg(P.vid + kid);
    uint32_t* row = P.levels + (size_t)dv * P.Q;
    bool i0 = false, i1 = false;
    if (a && acc0 < __ldcg(row + lane)) i0 = acc0 < atomicMin(row + lane, acc0);
    if (b && acc1 < __ldcg(row + lane + 32)) i1 = acc1 < atomicMin(row + lane + 32, acc1);
    const unsigned long long ch =
        (unsigned long long)__ballot_sync(kFull, i0) | ((unsigned long long)__ballot_sync(kFull, i1) << 32);
    if (ch && lane == 0) {
        const unsigned long long prev = atomicOr(fnext + dv, ch);
        if (prev == 0ull && set_bit(next, dv)) {
            st.F += __ldg(P.outdeg + dv);
            st.n += 1;
            st.row += __ldg(P.eidx_off + dv + 1) - __ldg(P.eidx_off + dv);
            if (*reinterpret_cast<volatile unsigned*>(s_lcnt) <= (unsigned)kListCap) {
                const unsigned slot = atomicAdd(s_lcnt, 1u);
                if (slot < (unsigned)kListCap) s_list[slot] = dv;
            }
        }
    }
}

__device__ __forceinline__ void mssp_chunk(const PullParams& P, unsigned long long c, const unsigned long long* fcur,
                           unsigned long long* fnext, uint32_t* next, Stats& st, unsigned* s_lcnt, uint32_t* s_list) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long e0 = c * 32;
    const unsigned nv = (unsigned)(P.E - e0 < 32ull ? P.E - e0 : 32ull);
    uint32_t su = 0, sw = 0;
    unsigned long long sm = 0;
    if (lane < nv) {
        su = P.src[e0 + lane];
        sw = P.w[e0 + lane];
        sm = __ldcg(fcur + su);
    }
    if (!__any_sync(kFull, sm != 0ull)) return;
    const uint2 meta = __ldg(P.cmeta + c);
    uint32_t kid = meta.y;
    const unsigned Q = P.Q;
    const bool q0 = lane < Q, q1 = lane + 32 < Q;
    uint32_t acc0 = kInf, acc1 = kInf;
    for (unsigned g8 = 0; g8 < nv; g8 += 8) {
        uint32_t d0[8], d1[8], wv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const unsigned i = g8 + j;  // < 32
            const unsigned long long m = i < nv ? __shfl_sync(kFull, sm, i) : 0ull;
            const uint32_t u = __shfl_sync(kFull, su, i);
            wv[j] = __shfl_sync(kFull, sw, i);
            const uint32_t* row = P.levels + (size_t)u * Q;
            d0[j] = (q0 && ((m >> lane) & 1ull)) ? __ldcg(row + lane) : kInf;
            d1[j] = (q1 && ((m >> (lane + 32)) & 1ull)) ? __ldcg(row + lane + 32) : kInf;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const unsigned i = g8 + j;
            if (i > 0 && i < nv && ((meta.x >> i) & 1u)) {  // a new destination starts at position i
                mssp_flush(P, kid, acc0, acc1, fnext, next, st, s_lcnt, s_list);
                acc0 = kInf;
                acc1 = kInf;
                ++kid;
            }
            if (d0[j] != kInf) {
                const unsigned long long x = (unsigned long long)d0[j] + wv[j];
                acc0 = min(acc0, x > kSat ? kSat : (uint32_t)x);
            }
            if (d1[j] != kInf) {
                const unsigned long long x = (unsigned long long)d1[j] + wv[j];
                acc1 = min(acc1, x > kSat ? kSat : (uint32_t)x);
            }
        }
    }
    mssp_flush(P, kid, acc0, acc1, fnext, next, st, s_lcnt, s_list);
}

// Dense (every chunk) or sparse (the listed Wedge Frontier entries, whose
// bitmap words are zeroed as consumed) batched SSSP pull of iteration it.
__device__ __forceinline__ void mssp_pull(const PullParams& P, unsigned it, unsigned mode, unsigned k, unsigned nchunks,
                          uint32_t* next, Stats& st, unsigned long long gw, unsigned long long nw, unsigned* s_lcnt,
                          uint32_t* s_list) {
    const unsigned long long* fcur = (it & 1) ? P.fb[1] : P.fb[0];
    unsigned long long* fnext = (it & 1) ? P.fb[0] : P.fb[1];
    if (mode == 0) {
        for (unsigned long long c = gw; c < P.NC; c += nw) mssp_chunk(P, c, fcur, fnext, next, st, s_lcnt, s_list);
        return;
    }
    const unsigned long long nunits = (unsigned long long)nchunks << k;
    const unsigned long long kmask = (1ull << k) - 1;
    for (unsigned long long j = gw; j < nunits; j += nw) {
        const uint32_t b = __ldcg(P.clist + (j >> k));
        const unsigned long long c = ((unsigned long long)b << k) | (j & kmask);
        if ((j & kmask) == 0 && (threadIdx.x & 31) == 0) P.wb[b >> 5] = 0u;
        if (c < P.NC) mssp_chunk(P, c, fcur, fnext, next, st, s_lcnt, s_list);
    }
}

template <bool SSSP>
// Four resident blocks per SM (64 registers, a few spilled): the batched
// pulls are bound by latency and atomics, and the extra warps hide more of
// it than the spills cost (R-MAT s24, 64 queries: SSSP 235 -> 169 ms, BFS
// 12.6 -> 12.4 ms against three blocks per SM at 80 registers).
__global__ void __launch_bounds__(kCW * 32, 4) k_msbfs(const PullParams P, const XformParams X, unsigned* bar) {
    using T = unsigned long long;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned long long s_F;
    __shared__ unsigned s_n, s_row, s_lcnt, s_lbase;
    RunCtl* C = P.ctl;
    if (C->done) return;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T* s_val = reinterpret_cast<T*>(smem);
    uint32_t* s_kid = reinterpret_cast<uint32_t*>(s_val + kCW * kRecCap);
    uint32_t* s_list = reinterpret_cast<uint32_t*>(smem + pull_records_bytes<kMSBFS>());
    uint32_t* my_kid = s_kid + warp * kRecCap;
    T* my_val = s_val + warp * kRecCap;
    const unsigned long long gw = (unsigned long long)blockIdx.x * kCW + warp;
    const unsigned long long nw = (unsigned long long)gridDim.x * kCW;
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long words = ((unsigned long long)X.V + 31) / 32;
    unsigned it = C->it;
    unsigned mode = P.rec[it].mode, k = P.rec[it].k;
    for (;;) {
        // ---- pull it ----
        if (threadIdx.x == 0) {
            s_F = 0;
            s_n = 0;
            s_row = 0;
            s_lcnt = 0;
        }
        __syncthreads();
        Stats st{0ull, 0u, 0u, 0u};
        const uint32_t* cur = (it & 1) ? P.bm[1] : P.bm[0];
        uint32_t* next = (it & 1) ? P.bm[0] : P.bm[1];
        if constexpr (SSSP)
            mssp_pull(P, it, mode, k, __ldcg(&P.rec[it].nchunks), next, st, gw, nw, &s_lcnt, s_list);
        else if (mode == 0)
            pull_dense_direct<kMSBFS>(P, it, cur, next, my_kid, my_val, st, gw, nw, &s_lcnt, s_list);
        else
            pull_sparse<kMSBFS>(P, it, k, __ldcg(&P.rec[it].nchunks), cur, next, my_kid, my_val, st, gw, nw,
                                &s_lcnt, s_list);
        for (int d = 16; d > 0; d >>= 1) {
            st.F += __shfl_down_sync(kFull, st.F, d);
            st.n += __shfl_down_sync(kFull, st.n, d);
            st.row += __shfl_down_sync(kFull, st.row, d);
        }
        if (lane == 0 && st.n) {
            atomicAdd(&s_F, st.F);
            atomicAdd(&s_n, st.n);
            atomicAdd(&s_row, st.row);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_n) {
                atomicAdd(&P.rec[it + 1].fullness, s_F);
                atomicAdd(&P.rec[it + 1].nfront, s_n);
                atomicAdd(&P.rec[it + 1].rowsum, s_row);
            }
            s_lbase = (s_lcnt && s_lcnt <= (unsigned)kListCap) ? atomicAdd(&P.rec[it + 1].nlist, s_lcnt) : ~0u;
        }
        __syncthreads();
        publish_list(P.flist[(it + 1) & 1], s_list, s_lcnt, s_lbase);
        if (!grid_sync(bar, &C->status)) break;
        // ---- decision: every block computes it from the same sums ----
        const unsigned nit = it + 1;
        const unsigned long long F = __ldcg(&P.rec[nit].fullness);
        const unsigned nf = __ldcg(&P.rec[nit].nfront);
        unsigned sparse;
        if (C->switch_mode == WEDGE_SWITCH_ALWAYS_DENSE) sparse = 0;
        else if (C->switch_mode == WEDGE_SWITCH_ALWAYS_SPARSE) sparse = 1;
        else sparse = (F * 10000ull < (unsigned long long)C->tau_bp * C->E) ? 1u : 0u;
        // 8-bit levels: the pull found a vertex at level 255 or more
        const bool overflow = P.levels8 != nullptr && (__ldcg(&C->status) & kStatusLevelOverflow) != 0;
        const bool done = nf == 0 || nit >= C->max_iters || overflow;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            P.rec[nit].mode = sparse;
            P.rec[nit].k = C->k;
            C->it = nit;
            if (done) {
                C->done = 1;
                if (nf && !overflow) C->status |= kStatusMaxIters;
            }
        }
        if (done) break;
        // ---- retire frontier it (masks and bitmap), prepare the next ----
        const unsigned nl_t = __ldcg(&P.rec[it].nlist), nf_t = __ldcg(&P.rec[it].nfront);
        clear_frontier((it & 1) ? P.bm[1] : P.bm[0], words, (it & 1) ? P.flist[1] : P.flist[0], nl_t == nf_t, nf_t,
                       (it & 1) ? P.fb[1] : P.fb[0], tid, nth);
        if (blockIdx.x == 0 && threadIdx.x < sizeof(IterRec) / 4)
            reinterpret_cast<unsigned*>(P.rec + nit + 1)[threadIdx.x] = 0u;
        if (sparse) {
            if (__ldcg(&P.rec[nit].nlist) == nf)
                xform_scan_list((nit & 1) ? P.flist[1] : P.flist[0], nf, X.eidx_off, PieceOut{X.pieces, nullptr, nullptr, nullptr, nullptr, nullptr}, &P.rec[nit].npieces,
                                gw, nw);
            else
                xform_scan_words(next, X.V, words, X.eidx_off, PieceOut{X.pieces, nullptr, nullptr, nullptr, nullptr, nullptr}, &P.rec[nit].npieces, gw, nw);
        }
        if (!grid_sync(bar, &C->status)) break;
        if (sparse)
            xform_expand_pieces<kSrcPieces>(X.pieces, __ldcg(&P.rec[nit].npieces), C->k, X.eidx, X.wb, X.clist,
                                &P.rec[nit].nchunks, gw, nw);
        if (!grid_sync(bar, &C->status)) break;
        it = nit;
        mode = sparse;
        k = C->k;
    }
}

// ------------------------------------------------------------------------
// PageRank vertex step (K6): pr = (1-d)/V + d*(acc + D/V); then either the
// next iteration's fixed-point contributions and dangling mass, or the
// final FP32 ranks.
// ------------------------------------------------------------------------
// Block-wide sum of x, added to *dst with one atomic per block (blockDim
// a multiple of 32, at most 1024).
__device__ __forceinline__ void block_add_u64(unsigned long long x, unsigned long long* dst) {
    __shared__ unsigned long long part[32];
    for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(kFull, x, d);
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) part[warp] = x;
    __syncthreads();
    if (warp == 0) {
        x = lane < (blockDim.x >> 5) ? part[lane] : 0ull;
        for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(kFull, x, d);
        if (lane == 0 && x) atomicAdd(dst, x);
    }
}

// Contributions live in PageRank's gather order: u's at contrib[perm[u]].
__global__ void k_pr_init(uint32_t V, const uint32_t* __restrict__ outdeg, const uint32_t* __restrict__ perm,
                          float* __restrict__ contrib, unsigned long long* __restrict__ acc, RunCtl* C) {
    const float pr0 = 1.0f / (float)V;
    unsigned long long dang = 0;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t od = outdeg[v];
        contrib[perm[v]] = od ? pr0 / (float)od : 0.0f;
        acc[v] = 0ull;
        if (!od) dang += __float2ull_rn(pr0 * 0x1p62f);
    }
    block_add_u64(dang, &C->dangling[0]);
}

// One vertex of the PageRank step: rank from the fixed-point in-edge sum,
// the next contribution, and the dangling mass it adds.
__device__ __forceinline__ void pr_vertex(unsigned long long a, uint32_t od, float dv, float base, float d, int last,
                                          float& out, float& contrib, unsigned long long& dang) {
    const float pr = fmaf(d, __ull2float_rn(a) * 0x1p-62f + dv, base);
    if (last) {
        out = pr;
    } else {
        contrib = od ? pr / (float)od : 0.0f;
        if (!od) dang += __float2ull_rn(pr * 0x1p62f);
    }
}

// The vertex step, four consecutive vertices per thread and iteration with
// 16- and 32-byte accesses (a grid-stride scalar loop kept too few bytes in
// flight to reach HBM rates).  Sums of destinations split across pull
// slices are zeroed for the next pull's atomics.
__global__ void k_pr_apply(uint32_t V, const uint32_t* __restrict__ outdeg, const uint32_t* __restrict__ split_bm,
                           const uint32_t* __restrict__ perm, unsigned long long* __restrict__ acc,
                           float* __restrict__ contrib, float* __restrict__ out, RunCtl* C, unsigned t, int last,
                           float base, float d) {
    const float dv = __ull2float_rn(__ldcg(&C->dangling[t & 1])) * 0x1p-62f / (float)V;
    unsigned long long dang = 0;
    const unsigned long long nq = V / 4;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < nq; q += stride) {
        const unsigned long long v = 4 * q;
        const ulonglong2 a01 = reinterpret_cast<const ulonglong2*>(acc)[2 * q];
        const ulonglong2 a23 = reinterpret_cast<const ulonglong2*>(acc)[2 * q + 1];
        const uint4 od = last ? make_uint4(0u, 0u, 0u, 0u) : reinterpret_cast<const uint4*>(outdeg)[q];
        const uint32_t split = (__ldg(split_bm + (v >> 5)) >> (v & 31)) & 0xFu;
        if (split) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((split >> i) & 1u) acc[v + i] = 0ull;
        }
        float4 o, c;
        pr_vertex(a01.x, od.x, dv, base, d, last, o.x, c.x, dang);
        pr_vertex(a01.y, od.y, dv, base, d, last, o.y, c.y, dang);
        pr_vertex(a23.x, od.z, dv, base, d, last, o.z, c.z, dang);
        pr_vertex(a23.y, od.w, dv, base, d, last, o.w, c.w, dang);
        if (last) {
            reinterpret_cast<float4*>(out)[q] = o;
        } else {  // into the gather order
            const uint4 pp = reinterpret_cast<const uint4*>(perm)[q];
            contrib[pp.x] = c.x;
            contrib[pp.y] = c.y;
            contrib[pp.z] = c.z;
            contrib[pp.w] = c.w;
        }
    }
    // the tail of V mod 4 vertices
    for (unsigned long long v = 4 * nq + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V; v += stride) {
        const unsigned long long a = acc[v];
        if ((__ldg(split_bm + (v >> 5)) >> (v & 31)) & 1u) acc[v] = 0ull;
        float o = 0.f, c = 0.f;
        pr_vertex(a, last ? 0u : outdeg[v], dv, base, d, last, o, c, dang);
        if (last) out[v] = o;
        else contrib[perm[v]] = c;
    }
    if (!last) block_add_u64(dang, &C->dangling[(t + 1) & 1]);
}

// A caller's contributions (by vertex) into PageRank's gather order.
__global__ void k_pr_scatter(uint32_t V, const uint32_t* __restrict__ perm, const float* __restrict__ in,
                             float* __restrict__ out) {
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += (unsigned long long)gridDim.x * blockDim.x)
        out[perm[v]] = in[v];
}

__global__ void k_ctl_init(RunCtl* C, RunCtl init) {
    if (threadIdx.x == 0) *C = init;
}

// Leaves the Wedge bitmap clear after a standalone transformation: the
// words of the listed entries, or, for a long list, every word the
// precision uses (`used_words`, 16-byte stores; the bitmap is allocated in
// whole 16-byte units).
__global__ void k_clear_listed(const uint32_t* __restrict__ list, const uint32_t* __restrict__ count,
                               uint32_t* __restrict__ wb, unsigned long long used_words) {
    const unsigned n = *count;
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
    if ((unsigned long long)n * 8 >= used_words) {
        uint4* w4 = reinterpret_cast<uint4*>(wb);
        const unsigned long long n4 = (used_words + 3) / 4;
        for (unsigned long long i = tid; i < n4; i += nth) w4[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
        for (unsigned long long i = tid; i < n; i += nth) wb[list[i] >> 5] = 0u;
    }
}

__global__ void k_standalone_prep(IterRec* rec, RunCtl* C, unsigned iter, unsigned sparse, unsigned k,
                                  const uint32_t* count_in, unsigned cap) {
    if (threadIdx.x == 0) {
        RunCtl c{};
        c.it = iter;
        c.max_iters = 0xFFFFFFFFu;
        *C = c;
        IterRec z{};
        rec[iter] = z;
        rec[iter + 1] = z;
        rec[iter].mode = sparse;
        rec[iter].k = k;
        const unsigned n = sparse ? *count_in : 0u;
        rec[iter].nchunks = n < cap ? n : cap;  // never read past the list's documented capacity
    }
}

__global__ void k_rec_set(IterRec* rec, unsigned t, IterRec v) {
    if (threadIdx.x == 0) rec[t] = v;
}

// Frontier size and fullness of a standalone pull, summed over the blocks' slots.
__global__ void k_standalone_out(const BlockStat* __restrict__ bstat, unsigned nblocks, unsigned long long* fullness,
                                 uint32_t* nfront) {
    __shared__ unsigned long long s_F;
    __shared__ unsigned s_n;
    if (threadIdx.x == 0) {
        s_F = 0;
        s_n = 0;
    }
    __syncthreads();
    unsigned long long F = 0;
    unsigned n = 0;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) {
        F += bstat[b].F;
        n += bstat[b].n;
    }
    atomicAdd(&s_F, F);
    atomicAdd(&s_n, n);
    __syncthreads();
    if (threadIdx.x == 0) {
        *fullness = s_F;
        *nfront = s_n;
    }
}

// ------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------
template <int APP>
static void launch_pull(const wedge_graph* g, const PullParams& P, cudaStream_t s) {
    if (P.dense_tma)
        k_pull<APP, true><<<g->pull_blocks_tma[APP], kPullThreads, pull_launch_smem<APP>(true), s>>>(P);
    else
        k_pull<APP, false><<<g->pull_blocks_app[APP], kCW * 32, pull_launch_smem<APP>(false), s>>>(P);
}

static void launch_pull_app(const wedge_graph* g, int app, const PullParams& P, cudaStream_t s) {
    switch (app) {
        case kBFS: launch_pull<kBFS>(g, P, s); break;
        case kCC: launch_pull<kCC>(g, P, s); break;
        case kSSSP: launch_pull<kSSSP>(g, P, s); break;
        default: launch_pull<kPR>(g, P, s); break;
    }
    count_launch();
}

// Blocks per SM for one pull variant, and a shared-memory carveout just
// large enough for them: the rest of the unified L1 caches the gathered
// vertex values.
template <int APP, bool TMA>
static wedge_status set_pull_variant(wedge_graph* g, int* blocks) {
    const int threads = TMA ? kPullThreads : kCW * 32;
    const int bytes = pull_launch_smem<APP>(TMA);
    WEDGE_TRY_CUDA(cudaFuncSetAttribute(k_pull<APP, TMA>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    WEDGE_TRY_CUDA(cudaFuncSetAttribute(k_pull<APP, TMA>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
    int n = 0;
    WEDGE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pull<APP, TMA>, threads, bytes));
    const int cap = g->tuning.blocks_per_sm;
    if (cap > 0 && n > cap) n = cap;
    if (n < 1) n = 1;
    cudaFuncAttributes fa;
    WEDGE_TRY_CUDA(cudaFuncGetAttributes(&fa, k_pull<APP, TMA>));
    const size_t need = (size_t)n * (bytes + fa.sharedSizeBytes + 1024);
    int pct = (int)((need * 100 + g->smem_per_sm - 1) / g->smem_per_sm);
    if (pct > 100) pct = 100;
    WEDGE_TRY_CUDA(cudaFuncSetAttribute(k_pull<APP, TMA>, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    *blocks = g->num_sms * n;
    return WEDGE_OK;
}

template <int APP>
static wedge_status set_pull_attrs(wedge_graph* g) {
    WEDGE_TRY((set_pull_variant<APP, false>(g, &g->pull_blocks_app[APP])));
    WEDGE_TRY((set_pull_variant<APP, true>(g, &g->pull_blocks_tma[APP])));
    return WEDGE_OK;
}

static wedge_status configure_pulls(wedge_graph* g) {
    WEDGE_TRY(set_pull_attrs<kBFS>(g));
    WEDGE_TRY(set_pull_attrs<kCC>(g));
    WEDGE_TRY(set_pull_attrs<kSSSP>(g));
    WEDGE_TRY(set_pull_attrs<kPR>(g));
    g->pull_blocks = g->pull_blocks_app[kCC];
    return WEDGE_OK;
}

static uint64_t visk_words(const wedge_graph* g) { return ((uint64_t)g->NZ + 31) / 32 + 1; }

wedge_status ensure_run_scratch(wedge_graph* g, cudaStream_t s) {
    if (g->ctl) return WEDGE_OK;
    const uint64_t V = g->V, NC = g->NC;
    const uint64_t words = (V + 31) / 32;
    WEDGE_TRY(dev_alloc(g, (void**)&g->vals, V * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->bm[0], words * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->bm[1], words * 4));
    // the Wedge bitmap, list and pieces are sized for the finest entries
    // (8 edges), so that a finer precision never reallocates them
    const uint64_t NU8 = (g->E + 7) / 8;
    g->wb_words = ((NU8 + 31) / 32 + 1 + 3) / 4 * 4;  // whole 16-byte units (cleared with 16-byte stores)
    g->clist_cap = NU8 + 1;
    g->pieces_cap = std::max(g->npieces_max, g->npieces_outdeg_bound) + 1;
    WEDGE_TRY(dev_alloc(g, (void**)&g->wb, g->wb_words * 4));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->wb, 0, g->wb_words * 4, s));
    WEDGE_TRY(dev_alloc(g, (void**)&g->clist, g->clist_cap * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->pieces, g->pieces_cap * sizeof(uint2)));

    WEDGE_TRY(dev_alloc(g, (void**)&g->longs, (uint64_t)kLongCap * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->xf_task, 16));
    WEDGE_TRY(dev_alloc(g, (void**)&g->flist[0], (V + 1) * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->flist[1], (V + 1) * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->visk, visk_words(g) * 4));
    g->rec_cap = kDefaultMaxIters + 2;
    WEDGE_TRY(dev_alloc(g, (void**)&g->rec, (uint64_t)g->rec_cap * sizeof(IterRec)));
    WEDGE_TRY(dev_alloc(g, (void**)&g->ctl, sizeof(RunCtl)));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->ctl, 0, sizeof(RunCtl), s));
    static_assert(sizeof(RunCtl) <= 256, "control block mirror must fit a pinned block");
    g->h_ctl = static_cast<RunCtl*>(pinned_small_alloc(sizeof(RunCtl)));
    if (!g->h_ctl) return set_error(WEDGE_ERR_OUT_OF_MEMORY, "pinned host memory for the control block");
    memset(g->h_ctl, 0, sizeof(RunCtl));
    WEDGE_TRY(dev_alloc(g, (void**)&g->contrib, V * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->acc, V * 8));
    WEDGE_TRY(dev_alloc(g, (void**)&g->rank, V * 4));
    WEDGE_TRY_CUDA(cudaEventCreate(&g->ev0));
    WEDGE_TRY_CUDA(cudaEventCreate(&g->ev1));
    WEDGE_TRY_CUDA(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    WEDGE_TRY(configure_pulls(g));
    g->xform_blocks = g->num_sms * 4;
    int nb = g->xform_blocks;  // the hybrid's push blocks write slots too
    for (int a = 0; a < 4; ++a) nb = std::max(nb, std::max(g->pull_blocks_app[a], g->pull_blocks_tma[a]));
    if (nb > kMaxPullBlocks) return set_error(WEDGE_ERR_NOT_SUPPORTED, "too many pull blocks for this device");
    WEDGE_TRY(dev_alloc(g, (void**)&g->bstat, (uint64_t)nb * sizeof(BlockStat)));
    return WEDGE_OK;
}

static GraphFeat graph_feat(const wedge_graph* g, int app) {
    GraphFeat f;
    f.log2V = (float)std::log2((double)g->V);
    f.log2E = (float)std::log2((double)(g->E ? g->E : 1));
    f.avg_deg = (float)((double)g->E / (double)g->V);
    const double mean = (double)g->E / (double)g->V;
    f.skew = (float)(std::log2(1.0 + (mean > 0 ? g->max_outdeg / mean : 0.0)) / 16.0);
    f.app = app == kBFS ? 0.f : (app == kCC ? 0.5f : 1.f);
    f.band_lo = g->band_lo;
    f.band_hi = g->band_hi;
    return f;
}

static PullParams pull_params(wedge_graph* g, int trace, int app = kCC) {
    PullParams P{};
    P.gf = graph_feat(g, app);
    P.mlp = g->has_model ? reinterpret_cast<const __nv_bfloat16*>(g->mlp_bf16) : nullptr;
    P.src = g->src;
    P.w = g->w;
    P.cmeta = g->cmeta;
    P.vid = g->vid;
    P.outdeg = g->outdeg;
    P.eidx_off = g->eidx_off;
    P.E = g->E;
    P.NC = g->NC;
    P.vals = g->vals;
    P.vread = g->vals;
    P.bm[0] = g->bm[0];
    P.bm[1] = g->bm[1];
    P.clist = g->clist;
    P.wb = g->wb;
    P.rec = g->rec;
    P.ctl = g->ctl;
    P.contrib = g->contrib;
    P.acc = g->acc;
    P.trace = trace;
    P.dense_tma = g->tuning.dense_loader == 1 ? 1 : 0;
    P.flist[0] = g->flist[0];
    P.flist[1] = g->flist[1];
    P.bstat = g->bstat;
    P.visk = app == kBFS ? g->visk : nullptr;
    P.decide = (app == kBFS || app == kCC || app == kSSSP) ? 1 : 0;
    P.cond = 0;
    return P;
}

static XformParams xform_params(wedge_graph* g, int trace) {
    XformParams X{};
    X.eidx = g->eidx;
    X.eidx_off = g->eidx_off;
    X.pieces = g->pieces;
    X.wb = g->wb;
    X.clist = g->clist;
    X.rec = g->rec;
    X.ctl = g->ctl;
    X.bm[0] = g->bm[0];
    X.bm[1] = g->bm[1];
    X.flist[0] = g->flist[0];
    X.flist[1] = g->flist[1];
    X.bm_in = nullptr;
    X.V = g->V;
    X.bm_words = ((uint64_t)g->V + 31) / 32;
    X.count_out = nullptr;
    X.standalone = 0;
    X.standalone_k = 0;
    X.eidx8 = g->eidx8;
    X.eidx8_off = g->eidx8_off;
    X.trace = trace;
    X.wstat = nullptr;
    X.slice_ctr = nullptr;
    X.longs = g->longs;
    X.task_ctr = g->xf_task;
    const bool z = g->tuning.edge_index == 1 && g->zpieces;
    X.zhdr = z ? g->zhdr : nullptr;
    X.zwords = z ? g->zwords : nullptr;
    X.zbo = z ? g->zbo : nullptr;
    X.zpieces = z ? g->zpieces : nullptr;
    return X;
}

// Grid size of the pull variant that P selects.
static unsigned pull_grid(const wedge_graph* g, int app, const PullParams& P) {
    return (unsigned)(P.dense_tma ? g->pull_blocks_tma[app] : g->pull_blocks_app[app]);
}

static void launch_xform(const wedge_graph* g, const XformParams& X, cudaStream_t s) {
    k_xform_scan<<<g->xform_blocks, kXformThreads, 0, s>>>(X);
    k_xform_expand<<<g->xform_blocks, kXformThreads, 0, s>>>(X);
    count_launch(2);
}

// Captures a loop body under a conditional while node: body(cond, stream)
// launches the body's kernels, whose deciding blocks set the condition.
// The body reads everything from the library-owned buffers, so one instance
// serves every run of an application on g.
template <class Body>
static wedge_status capture_while_graph(wedge_graph* g, Body body, cudaGraphExec_t* out) {
    cudaGraph_t graph = nullptr;
    WEDGE_TRY_CUDA(cudaGraphCreate(&graph, 0));
    struct Destroy {
        cudaGraph_t g;
        ~Destroy() {
            if (g) cudaGraphDestroy(g);
        }
    } guard{graph};
    cudaGraphConditionalHandle handle;
    WEDGE_TRY_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1u, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    WEDGE_TRY_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaStream_t cs = g->cap_stream;
    WEDGE_TRY_CUDA(cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeThreadLocal));
    body(handle, cs);
    cudaError_t le = cudaGetLastError();
    cudaGraph_t captured = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &captured);
    if (le != cudaSuccess) return cuda_error(le, "loop body launch");
    if (ce != cudaSuccess) return cuda_error(ce, "cudaStreamEndCapture");
    WEDGE_TRY_CUDA(cudaGraphInstantiate(out, graph, 0));
    return WEDGE_OK;
}

// Wedge's loop body: pull (with the decision), transformation.
static wedge_status build_loop_graph(wedge_graph* g, int app) {
    return capture_while_graph(g, [&](cudaGraphConditionalHandle cond, cudaStream_t cs) {
        PullParams P = pull_params(g, 0, app);
        P.cond = cond;
        launch_pull_app(g, app, P, cs);
        XformParams X = xform_params(g, 0);
        X.direct = 1;
        launch_xform(g, X, cs);
    }, &g->loop_exec[app]);
}

// A precision k as the ABI passes it (uint32): 0 .. 7, or -1 / -2 for
// entries of 16 / 8 edges.
static bool valid_precision(uint32_t k) { return (int)k >= -2 && (int)k <= (int)kMaxCoarsen; }

// Wedge Frontier entries of the graph at precision k: ceil(E / (32 * 2^k)).
static uint64_t entries_at(const wedge_graph* g, int k) {
    const unsigned sh = (unsigned)(5 + k);
    return (g->E + (1ull << sh) - 1) >> sh;
}

// Wedge bitmap words those entries use (at most the allocated words, which
// cover 8-edge entries and are a whole number of 16-byte units).
static uint64_t wb_words_at(const wedge_graph* g, int k) {
    const uint64_t w = (entries_at(g, k) + 31) / 32;
    return w < g->wb_words ? w : g->wb_words;
}

// Finer precisions than one chunk need the edge index in 8-edge units,
// built on first use (the Wedge bitmap, list and pieces are allocated for
// them already).  Loop graphs captured before it existed hold a null index
// and are dropped then.
static wedge_status ensure_fine(wedge_graph* g, cudaStream_t s) {
    if (g->eidx8) return WEDGE_OK;
    WEDGE_TRY(build_eidx8(g, s));
    if (g->npieces8_max + 1 > g->pieces_cap) return set_error(WEDGE_ERR_CUDA, "8-edge index exceeds its piece bound");
    bool cached = g->ms_exec != nullptr;
    for (auto x : g->loop_exec) cached |= x != nullptr;
    for (auto x : g->loop_exec_push) cached |= x != nullptr;
    if (!cached) return WEDGE_OK;
    WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    if (g->last_stream) WEDGE_TRY_CUDA(cudaStreamSynchronize(g->last_stream));
    for (auto& x : g->loop_exec)
        if (x) {
            cudaGraphExecDestroy(x);
            x = nullptr;
        }
    for (auto& x : g->loop_exec_push)
        if (x) {
            cudaGraphExecDestroy(x);
            x = nullptr;
        }
    if (g->ms_exec) {
        cudaGraphExecDestroy(g->ms_exec);
        g->ms_exec = nullptr;
    }
    g->loop_failed = false;
    return WEDGE_OK;
}

static wedge_status check_opts(const wedge_opts* o) {
    if (!valid_precision(o->log2_coarsen))
        return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be 0..7, or -1 / -2 (16- / 8-edge entries)");
    if (o->switch_mode > WEDGE_SWITCH_ALWAYS_SPARSE) return set_error(WEDGE_ERR_INVALID_ARG, "bad switch_mode");
    if (o->reserved[0]) return set_error(WEDGE_ERR_INVALID_ARG, "reserved option fields must be zero");
    return WEDGE_OK;
}

static wedge_status fill_stats(wedge_graph* g, cudaStream_t s, wedge_stats* stats) {
    if (!stats) return WEDGE_OK;
    WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    const uint32_t iters = g->h_ctl->it;
    g->last_iters = iters;
    std::vector<IterRec> r(iters + 1);
    if (iters) WEDGE_TRY_CUDA(cudaMemcpy(r.data(), g->rec, (size_t)iters * sizeof(IterRec), cudaMemcpyDeviceToHost));
    stats->iters = iters;
    stats->sparse_iters = 0;
    stats->edges_pulled = 0;
    stats->chunks_listed = 0;
    for (uint32_t t = 0; t < iters; ++t) {
        if (r[t].mode && g->last_push) {
            stats->sparse_iters++;
            stats->edges_pulled += r[t].fullness;  // the out-edges pushed
        } else if (r[t].mode) {
            stats->sparse_iters++;
            stats->chunks_listed += r[t].nchunks;
            const uint64_t e = (uint64_t)r[t].nchunks << (5 + (int)r[t].k);
            stats->edges_pulled += e < g->E ? e : g->E;
        } else {
            stats->edges_pulled += g->E;
        }
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    stats->device_ms = ms;
    if (g->h_ctl->status & kStatusTimeout) return set_error(WEDGE_ERR_TIMEOUT, "a bounded device wait timed out");
    if (g->h_ctl->status & kStatusMaxIters)
        return set_error(WEDGE_ERR_MAX_ITERS, "frontier still non-empty at max_iters");
    return WEDGE_OK;
}

// Host-polled loop: traced runs, synchronous runs, and graphs whose device
// loop could not be built.  body(i) launches loop body i; after the run is
// done the bodies' kernels return at once.
template <class Body>
static wedge_status host_loop(wedge_graph* g, Body body, uint32_t max_iters, cudaStream_t s) {
    const int batch = 8;
    uint32_t launched = 0;
    for (;;) {
        for (int b = 0; b < batch; ++b) body(launched++);
        WEDGE_TRY_CUDA(cudaGetLastError());
        WEDGE_TRY_CUDA(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost, s));
        WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
        if (g->h_ctl->done || launched > max_iters + 2) return WEDGE_OK;
    }
}

// Synchronous CC/SSSP (the opts' `synchronous`): pull t reads buffer t & 1
// and writes buffer (t + 1) & 1, which first receives a copy of the values
// (destinations outside a Wedge Frontier keep theirs).  Body i is pull i,
// or returns at once after the run is done.
__global__ void k_sync_copy(const RunCtl* C, const uint32_t* __restrict__ from, uint32_t* __restrict__ to,
                            uint32_t V) {
    if (C->done) return;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x)
        to[v] = from[v];
}

static void launch_sync_body(wedge_graph* g, int app, const PullParams& P, const XformParams& X, uint32_t i,
                             cudaStream_t s) {
    uint32_t* vb[2] = {g->vals, g->vals_sync};
    k_sync_copy<<<g->num_sms * 4, 256, 0, s>>>(g->ctl, vb[i & 1], vb[(i + 1) & 1], g->V);
    count_launch();
    PullParams Q = P;
    Q.vread = vb[i & 1];
    Q.vals = vb[(i + 1) & 1];
    launch_pull_app(g, app, Q, s);
    launch_xform(g, X, s);
}

// The push/pull hybrid's loop body: pieces of the frontier's out-edge rows
// (X reads the CSR offsets), the push, the preparation of a dense iteration
// the push may have chosen, the dense pull.
static void launch_hybrid_body(const wedge_graph* g, int app, const PullParams& P, const XformParams& X,
                               const PushParams& Q, cudaStream_t s) {
    k_xform_scan<<<g->xform_blocks, kXformThreads, 0, s>>>(X);
    switch (app) {
        case kBFS: k_push_expand<kBFS><<<g->xform_blocks, kXformThreads, 0, s>>>(P, Q); break;
        case kCC: k_push_expand<kCC><<<g->xform_blocks, kXformThreads, 0, s>>>(P, Q); break;
        default: k_push_expand<kSSSP><<<g->xform_blocks, kXformThreads, 0, s>>>(P, Q); break;
    }
    k_hybrid_prepare<<<g->xform_blocks, kXformThreads, 0, s>>>(X);
    count_launch(3);
    launch_pull_app(g, app, P, s);
}

static PushParams push_params(const wedge_graph* g) {
    PushParams Q{};
    Q.dst = g->csr_dst;
    Q.src = g->csr_src;
    Q.w = g->csr_w;
    Q.kid_of = g->kid_of;
    Q.pieces = g->push_pieces;
    return Q;
}

static wedge_status build_hybrid_graph(wedge_graph* g, int app) {
    return capture_while_graph(g, [&](cudaGraphConditionalHandle cond, cudaStream_t cs) {
        PullParams P = pull_params(g, 0, app);
        P.cond = cond;
        P.mlp = nullptr;
        P.hybrid = 1;
        XformParams X = xform_params(g, 0);
        X.eidx_off = g->csr_off;
        X.pieces = g->push_pieces;
        X.zhdr = nullptr;  // pieces of out-edge rows: never compressed, never listed as long rows,
        X.longs = nullptr; // and read from the CSR at every precision
        X.eidx8_off = X.eidx_off;
        X.eidx8 = nullptr;
        launch_hybrid_body(g, app, P, X, push_params(g), cs);
    }, &g->loop_exec_push[app]);
}

static wedge_status run_frontier_app(wedge_graph* g, int app, uint32_t root, uint32_t* out,
                                     const wedge_opts* opts_in, wedge_stats* stats, cudaStream_t s) {
    wedge_opts o;
    if (opts_in) o = *opts_in;
    else wedge_default_opts((wedge_app)app, &o);
    WEDGE_TRY(check_opts(&o));
    if (!out) return set_error(WEDGE_ERR_INVALID_ARG, "output is NULL");
    if (app != kCC && root >= g->V) return set_error(WEDGE_ERR_INVALID_ARG, "root out of range");
    if (app == kSSSP && !g->w && g->E) return set_error(WEDGE_ERR_INVALID_ARG, "SSSP needs edge weights");
    DeviceGuard dg(g->device);
    const uint32_t max_iters =
        o.max_iters ? (o.max_iters < kDefaultMaxIters ? o.max_iters : kDefaultMaxIters) : kDefaultMaxIters;
    const int trace = o.trace ? 1 : 0;
    RunCtl init{};
    init.max_iters = max_iters;
    init.switch_mode = o.switch_mode;
    init.tau_bp = o.tau_bp;
    init.k = o.log2_coarsen;
    init.E = g->E;
    const uint64_t wb_words = g->wb_words;
    const bool sync = o.synchronous && app != kBFS;
    const bool push = o.sparse_push != 0;
    if (push && o.synchronous) return set_error(WEDGE_ERR_INVALID_ARG, "sparse_push and synchronous exclude each other");
    if (push && init.switch_mode == WEDGE_SWITCH_LEARNED) init.switch_mode = WEDGE_SWITCH_THRESHOLD;
    if (sync && !g->vals_sync) WEDGE_TRY(dev_alloc(g, (void**)&g->vals_sync, (uint64_t)g->V * 4));
    if (push) WEDGE_TRY(build_csr(g, s));
    if (!push && (int)o.log2_coarsen < 0) WEDGE_TRY(ensure_fine(g, s));
    if (push && !trace && !g->loop_exec_push[app] && !g->loop_failed) {
        if (build_hybrid_graph(g, app) != WEDGE_OK) {
            g->loop_failed = true;
            std::fprintf(stderr, "wedge: device loop graph unavailable (%s); using the host-polled loop\n",
                         wedge_last_error());
            cudaGetLastError();
        }
    }
    if (!push && !trace && !sync && !g->loop_exec[app] && !g->loop_failed) {
        if (build_loop_graph(g, app) != WEDGE_OK) {
            g->loop_failed = true;  // this graph keeps the host-polled loop
            std::fprintf(stderr, "wedge: device loop graph unavailable (%s); using the host-polled loop\n",
                         wedge_last_error());
            cudaGetLastError();
        }
    }
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev0, s));
    k_run_init<<<g->num_sms * 4, 256, 0, s>>>(app, g->V, root, g->vals, g->bm[0], g->bm[1], g->wb, wb_words, g->rec,
                                              g->ctl, init, g->flist[0], g->visk, visk_words(g));
    PullParams P = pull_params(g, trace, app);
    if (push) {
        P.mlp = nullptr;
        P.hybrid = 1;
    }
    k_frontier_stats<<<g->num_sms * 4, 256, 0, s>>>(g->bm[0], g->V, g->outdeg, g->eidx_off, g->rec, g->ctl, P.mlp,
                                                    P.gf);
    count_launch(2);
    XformParams X = xform_params(g, trace);
    X.direct = push ? 0 : 1;  // the hybrid's scan cuts out-edge rows for its push
    const uint32_t* result = g->vals;
    if (push) {
        X.eidx_off = g->csr_off;
        X.pieces = g->push_pieces;
        X.zhdr = nullptr;  // pieces of out-edge rows: never compressed, never listed as long rows,
        X.longs = nullptr; // and read from the CSR at every precision
        X.eidx8_off = X.eidx_off;
        X.eidx8 = nullptr;
        const PushParams Q = push_params(g);
        WEDGE_TRY_CUDA(cudaGetLastError());
        if (!trace && g->loop_exec_push[app])
            WEDGE_TRY_CUDA(cudaGraphLaunch(g->loop_exec_push[app], s));
        else
            WEDGE_TRY(host_loop(g, [&](uint32_t) { launch_hybrid_body(g, app, P, X, Q, s); }, max_iters, s));
    } else {
        launch_xform(g, X, s);
        WEDGE_TRY_CUDA(cudaGetLastError());
        if (sync) {
            WEDGE_TRY(host_loop(g, [&](uint32_t i) { launch_sync_body(g, app, P, X, i, s); }, max_iters, s));
            if (g->h_ctl->it & 1) result = g->vals_sync;  // pull it - 1 wrote buffer it & 1
        } else if (!trace && g->loop_exec[app]) {
            WEDGE_TRY_CUDA(cudaGraphLaunch(g->loop_exec[app], s));
        } else {
            WEDGE_TRY(host_loop(g, [&](uint32_t) {
                launch_pull_app(g, app, P, s);
                launch_xform(g, X, s);
            }, max_iters, s));
        }
    }
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev1, s));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost, s));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(out, result, (uint64_t)g->V * 4, cudaMemcpyDefault, s));
    g->last_trace = trace;
    g->last_stream = s;
    g->last_push = push;
    return fill_stats(g, s, stats);
}

// Batched BFS: everything after the roots' upload, enqueued on s (also the
// body of the captured graph).
static wedge_status msbfs_enqueue(wedge_graph* g, uint32_t nroots, uint32_t Q, void* levels, bool u8,
                                  const RunCtl& init, bool sssp, cudaStream_t s) {
    WEDGE_TRY_CUDA(cudaMemsetAsync(levels, 0xFF, (size_t)g->V * Q * (u8 ? 1 : 4), s));
    k_msbfs_clear<<<g->num_sms * 4, 256, 0, s>>>(g->V, g->ms_fb[0], g->ms_fb[1], g->ms_seen, g->bm[0], g->bm[1], g->wb,
                                                 g->wb_words, g->rec, g->ctl, init, g->ms_bar);
    k_msbfs_roots<<<(nroots + 255) / 256, 256, 0, s>>>(g->ms_roots, g->ms_roots + g->ms_cap, nroots, Q, g->ms_fb[0],
                                                       g->ms_seen, u8 ? nullptr : static_cast<uint32_t*>(levels),
                                                       u8 ? static_cast<uint8_t*>(levels) : nullptr, g->bm[0]);
    PullParams P = pull_params(g, 0, kBFS);
    P.mlp = nullptr;
    P.visk = nullptr;  // per-query visits live in the seen masks
    P.decide = 0;      // the persistent launch takes its own decisions
    P.fb[0] = g->ms_fb[0];
    P.fb[1] = g->ms_fb[1];
    P.seen = g->ms_seen;
    P.levels = u8 ? nullptr : static_cast<uint32_t*>(levels);
    P.levels8 = u8 ? static_cast<uint8_t*>(levels) : nullptr;
    P.Q = Q;
    XformParams X = xform_params(g, 0);
    X.zhdr = nullptr;  // batched runs read the plain edge index, all rows as pieces
    X.longs = nullptr;
    k_frontier_stats<<<g->num_sms * 4, 256, 0, s>>>(g->bm[0], g->V, g->outdeg, g->eidx_off, g->rec, g->ctl, nullptr,
                                                    P.gf);
    launch_xform(g, X, s);
    count_launch(3);
    void* args[] = {(void*)&P, (void*)&X, (void*)&g->ms_bar};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(g->ms_blocks);
    cfg.blockDim = dim3(kCW * 32);
    cfg.dynamicSmemBytes = pull_records_bytes<kMSBFS>() + kListCap * 4;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    WEDGE_TRY_CUDA(cudaLaunchKernelExC(&cfg, sssp ? (const void*)k_msbfs<true> : (const void*)k_msbfs<false>, args));
    count_launch();
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

static wedge_status msbfs_prepare(wedge_graph* g, uint32_t nroots, bool sssp) {
    const uint64_t V = g->V;
    if (!g->ms_seen) {
        WEDGE_TRY(dev_alloc(g, (void**)&g->ms_seen, V * 8));
        WEDGE_TRY(dev_alloc(g, (void**)&g->ms_fb[0], V * 8));
        WEDGE_TRY(dev_alloc(g, (void**)&g->ms_fb[1], V * 8));
        WEDGE_TRY(dev_alloc(g, (void**)&g->ms_bar, kBarWords * 4));
        const int smem = pull_records_bytes<kMSBFS>() + kListCap * 4;
        WEDGE_TRY_CUDA(cudaFuncSetAttribute(k_msbfs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        WEDGE_TRY_CUDA(cudaFuncSetAttribute(k_msbfs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        int n = 0, m = 0;
        WEDGE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_msbfs<false>, kCW * 32, smem));
        WEDGE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_msbfs<true>, kCW * 32, smem));
        if (n < 1 || m < 1) return set_error(WEDGE_ERR_NOT_SUPPORTED, "batched kernel does not fit on an SM");
        g->ms_occ = n;
        g->ms_occ_sssp = m;
    }
    int n = sssp ? g->ms_occ_sssp : g->ms_occ;
    if (g->tuning.blocks_per_sm > 0 && (int)g->tuning.blocks_per_sm < n) n = (int)g->tuning.blocks_per_sm;
    if (g->num_sms * n != g->ms_blocks && g->ms_exec) {
        cudaGraphExecDestroy(g->ms_exec);
        g->ms_exec = nullptr;
    }
    g->ms_blocks = g->num_sms * n;  // every block co-resident (cooperative launch)
    if (nroots > g->ms_cap) {
        if (g->ms_exec) {
            cudaGraphExecDestroy(g->ms_exec);
            g->ms_exec = nullptr;
        }
        dev_free(g->ms_roots);
        g->ms_roots = nullptr;
        uint32_t cap = 64;
        while (cap < nroots) cap *= 2;
        WEDGE_TRY(dev_alloc(g, (void**)&g->ms_roots, (uint64_t)cap * 2 * 4));
        g->ms_cap = cap;
    }
    return WEDGE_OK;
}

// PageRank: iters x (dense pull, vertex step).
static void pr_enqueue(wedge_graph* g, uint32_t iters, float damping, cudaStream_t s) {
    const int vb = g->num_sms * 8;
    PullParams P = pull_params(g, 0, kPR);
    P.src = g->pr_src;  // sources in the contributions' gather order
    const float base = (1.0f - damping) / (float)g->V;
    for (uint32_t t = 0; t < iters; ++t) {
        P.pr_iter = t;
        launch_pull_app(g, kPR, P, s);
        const int last = (t + 1 == iters);
        k_pr_apply<<<vb, 256, 0, s>>>(g->V, g->outdeg, g->split_bm, g->pr_perm, g->acc, g->contrib, g->rank, g->ctl,
                                      t, last, base, damping);
        count_launch();
    }
}

// PageRank's dense pull as a run executes it, on contributions already in
// the gather order (`ordered`), else first copied there from the caller's
// by-vertex array.  A dense pull at iteration 0; the caller's zeros take
// the place of the vertex step that clears split destinations between
// iterations.
static wedge_status pr_pull(wedge_graph* g, const float* d_contrib, uint64_t* d_sums, bool ordered, cudaStream_t s) {
    if (!g || !d_contrib || !d_sums) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(g->device);
    WEDGE_TRY(build_pr_order(g, s));
    k_standalone_prep<<<1, 32, 0, s>>>(g->rec, g->ctl, 0, 0, 0, nullptr, 0);
    count_launch();
    if (!ordered) {
        k_pr_scatter<<<g->num_sms * 8, 256, 0, s>>>(g->V, g->pr_perm, d_contrib, g->contrib);
        count_launch();
    }
    PullParams P = pull_params(g, 0, kPR);
    P.src = g->pr_src;
    P.contrib = ordered ? d_contrib : g->contrib;
    P.acc = reinterpret_cast<unsigned long long*>(d_sums);
    P.pr_iter = 0;
    launch_pull_app(g, kPR, P, s);
    WEDGE_TRY_CUDA(cudaGetLastError());
    g->last_stream = s;
    return WEDGE_OK;
}

}  // namespace wedge

using namespace wedge;

extern "C" {

wedge_status wedge_run_bfs(wedge_graph_t g, uint32_t root, uint32_t* d_level, const wedge_opts* opts,
                           wedge_stats* stats, wedge_stream_t stream) {
    if (!g) return set_error(WEDGE_ERR_INVALID_ARG, "graph is NULL");
    return run_frontier_app(g, kBFS, root, d_level, opts, stats, (cudaStream_t)stream);
}

wedge_status wedge_run_cc(wedge_graph_t g, uint32_t* d_label, const wedge_opts* opts, wedge_stats* stats,
                          wedge_stream_t stream) {
    if (!g) return set_error(WEDGE_ERR_INVALID_ARG, "graph is NULL");
    return run_frontier_app(g, kCC, 0, d_label, opts, stats, (cudaStream_t)stream);
}

wedge_status wedge_run_sssp(wedge_graph_t g, uint32_t root, uint32_t* d_dist, const wedge_opts* opts,
                            wedge_stats* stats, wedge_stream_t stream) {
    if (!g) return set_error(WEDGE_ERR_INVALID_ARG, "graph is NULL");
    return run_frontier_app(g, kSSSP, root, d_dist, opts, stats, (cudaStream_t)stream);
}

wedge_status wedge_run_pr(wedge_graph_t g, float* d_rank, uint32_t iters, float damping, const wedge_opts* opts,
                          wedge_stats* stats, wedge_stream_t stream) {
    if (!g) return set_error(WEDGE_ERR_INVALID_ARG, "graph is NULL");
    if (!d_rank) return set_error(WEDGE_ERR_INVALID_ARG, "rank output is NULL");
    if (!(damping >= 0.0f && damping <= 1.0f)) return set_error(WEDGE_ERR_INVALID_ARG, "damping must be in [0,1]");
    if (opts) WEDGE_TRY(check_opts(opts));
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t V = g->V;
    WEDGE_TRY(build_pr_order(g, s));
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev0, s));
    RunCtl init{};
    init.max_iters = 0xFFFFFFFFu;
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->rec, 0, 2 * sizeof(IterRec), s));
    k_ctl_init<<<1, 32, 0, s>>>(g->ctl, init);
    k_pr_init<<<g->num_sms * 8, 256, 0, s>>>(V, g->outdeg, g->pr_perm, g->contrib, g->acc, g->ctl);
    count_launch(2);
    if (iters == 0) {
        std::vector<float> h(V, 1.0f / (float)V);
        WEDGE_TRY_CUDA(cudaMemcpyAsync(d_rank, h.data(), (uint64_t)V * 4, cudaMemcpyHostToDevice, s));
        WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    } else {
        if (!g->pr_exec || g->pr_exec_iters != iters || g->pr_exec_damping != damping) {
            if (g->pr_exec) {
                cudaGraphExecDestroy(g->pr_exec);
                g->pr_exec = nullptr;
            }
            cudaGraph_t graph = nullptr;
            WEDGE_TRY_CUDA(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
            pr_enqueue(g, iters, damping, g->cap_stream);
            cudaError_t le = cudaGetLastError();
            cudaError_t ce = cudaStreamEndCapture(g->cap_stream, &graph);
            if (le != cudaSuccess || ce != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_error(le != cudaSuccess ? le : ce, "PageRank capture");
            }
            cudaError_t ie = cudaGraphInstantiate(&g->pr_exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) return cuda_error(ie, "cudaGraphInstantiate");
            g->pr_exec_iters = iters;
            g->pr_exec_damping = damping;
        } else {
            count_launch(2ull * iters);
        }
        WEDGE_TRY_CUDA(cudaGraphLaunch(g->pr_exec, s));
    }
    WEDGE_TRY_CUDA(cudaGetLastError());
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev1, s));
    if (iters) WEDGE_TRY_CUDA(cudaMemcpyAsync(d_rank, g->rank, (uint64_t)V * 4, cudaMemcpyDefault, s));
    if (stats) {
        WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
        stats->iters = iters;
        stats->sparse_iters = 0;
        stats->edges_pulled = (uint64_t)iters * g->E;
        stats->chunks_listed = 0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->ev0, g->ev1);
        stats->device_ms = ms;
    }
    g->last_iters = iters;
    g->last_trace = false;
    g->last_stream = s;
    return WEDGE_OK;
}

wedge_status wedge_pr_pull(wedge_graph_t g, const float* d_contrib, uint64_t* d_sums, wedge_stream_t stream) {
    return pr_pull(g, d_contrib, d_sums, false, (cudaStream_t)stream);
}

wedge_status wedge_pr_pull_ordered(wedge_graph_t g, const float* d_contrib, uint64_t* d_sums,
                                   wedge_stream_t stream) {
    return pr_pull(g, d_contrib, d_sums, true, (cudaStream_t)stream);
}

wedge_status wedge_pr_order(wedge_graph_t g, uint32_t* d_order, wedge_stream_t stream) {
    if (!g || !d_order) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (classify(d_order) != PtrKind::Device) return set_error(WEDGE_ERR_INVALID_ARG, "d_order must be device memory");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    WEDGE_TRY(build_pr_order(g, s));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(d_order, g->pr_perm, (uint64_t)g->V * 4, cudaMemcpyDeviceToDevice, s));
    g->last_stream = s;
    return WEDGE_OK;
}

wedge_status wedge_selftest_timeout(int kind) {
    if (kind != 0 && kind != 1) return set_error(WEDGE_ERR_INVALID_ARG, "kind must be 0 or 1");
    unsigned* d = nullptr;  // [status, barrier words ...]
    WEDGE_TRY(dev_alloc(nullptr, (void**)&d, (1 + kBarWords) * sizeof(unsigned)));
    cudaError_t e = cudaMemset(d, 0, (1 + kBarWords) * sizeof(unsigned));
    if (e == cudaSuccess) {
        k_selftest_wait<<<kind == 0 ? 1 : 2, 32>>>(kind, d + 1, d);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned status = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&status, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
    dev_free(d);
    if (e != cudaSuccess) return cuda_error(e, "wait self-test");
    if (status & kStatusTimeout) return set_error(WEDGE_ERR_TIMEOUT, "the self-test wait timed out, as it must");
    return WEDGE_OK;
}

}  // extern "C"

namespace wedge {
// Batched BFS (sssp = false) or SSSP (sssp = true) of up to 64 queries.
static wedge_status run_batch(wedge_graph* g, bool sssp, const uint32_t* roots, const uint32_t* root_query,
                              uint32_t nroots, uint32_t nqueries, void* d_levels, bool u8, const wedge_opts* opts_in,
                              wedge_stats* stats, cudaStream_t s) {
    if (!g || !roots || !d_levels) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (sssp && !g->w && g->E) return set_error(WEDGE_ERR_INVALID_ARG, "SSSP needs edge weights");
    if (nqueries < 1 || nqueries > 64) return set_error(WEDGE_ERR_INVALID_ARG, "nqueries must be 1..64");
    if (nroots < 1 || nroots > (1u << 24)) return set_error(WEDGE_ERR_INVALID_ARG, "nroots must be 1..2^24");
    wedge_opts o;
    if (opts_in) o = *opts_in;
    else wedge_default_opts(sssp ? WEDGE_SSSP : WEDGE_BFS, &o);
    WEDGE_TRY(check_opts(&o));
    if ((int)o.log2_coarsen < 0) o.log2_coarsen = 0;  // batched runs list whole chunks
    if (classify(d_levels) != PtrKind::Device) return set_error(WEDGE_ERR_INVALID_ARG, "levels must be device memory");
    DeviceGuard dg(g->device);
    // roots and their queries, checked on the host
    std::vector<uint32_t> hr((size_t)nroots * 2);
    WEDGE_TRY_CUDA(cudaMemcpy(hr.data(), roots, (size_t)nroots * 4, cudaMemcpyDefault));
    if (root_query) WEDGE_TRY_CUDA(cudaMemcpy(hr.data() + nroots, root_query, (size_t)nroots * 4, cudaMemcpyDefault));
    for (uint32_t i = 0; i < nroots; ++i) {
        if (!root_query) hr[nroots + i] = i;
        if (hr[i] >= g->V) return set_error(WEDGE_ERR_INVALID_ARG, "root out of range");
        if (hr[nroots + i] >= nqueries) return set_error(WEDGE_ERR_INVALID_ARG, "query id out of range");
    }
    WEDGE_TRY(msbfs_prepare(g, nroots, sssp));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(g->ms_roots, hr.data(), (size_t)nroots * 4, cudaMemcpyHostToDevice, s));
    WEDGE_TRY_CUDA(
        cudaMemcpyAsync(g->ms_roots + g->ms_cap, hr.data() + nroots, (size_t)nroots * 4, cudaMemcpyHostToDevice, s));
    RunCtl init{};
    init.max_iters = o.max_iters ? (o.max_iters < kDefaultMaxIters ? o.max_iters : kDefaultMaxIters) : kDefaultMaxIters;
    init.switch_mode = o.switch_mode == WEDGE_SWITCH_LEARNED ? WEDGE_SWITCH_THRESHOLD : o.switch_mode;
    init.tau_bp = o.tau_bp;
    init.k = o.log2_coarsen;
    init.E = g->E;
    const uint32_t key[5] = {init.tau_bp, init.k, init.switch_mode, init.max_iters, (sssp ? 1u : 0u) | (u8 ? 2u : 0u)};
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev0, s));
    const bool reuse = g->ms_exec && g->ms_exec_q == nqueries && g->ms_exec_n == nroots &&
                       g->ms_exec_levels == d_levels && !memcmp(key, g->ms_exec_key, sizeof(key));
    if (!reuse && !g->ms_graph_failed) {
        if (g->ms_exec) {
            cudaGraphExecDestroy(g->ms_exec);
            g->ms_exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
        wedge_status es = WEDGE_OK;
        if (e == cudaSuccess) es = msbfs_enqueue(g, nroots, nqueries, d_levels, u8, init, sssp, g->cap_stream);
        cudaError_t ee = e == cudaSuccess ? cudaStreamEndCapture(g->cap_stream, &graph) : e;
        if (e == cudaSuccess && es == WEDGE_OK && ee == cudaSuccess &&
            cudaGraphInstantiate(&g->ms_exec, graph, 0) == cudaSuccess) {
            g->ms_exec_q = nqueries;
            g->ms_exec_n = nroots;
            g->ms_exec_levels = d_levels;
            memcpy(g->ms_exec_key, key, sizeof(key));
        } else {
            g->ms_exec = nullptr;
            g->ms_graph_failed = true;  // direct launches from now on
            std::fprintf(stderr, "wedge: batched run graph capture unavailable; launching directly\n");
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
    }
    if (g->ms_exec) {
        WEDGE_TRY_CUDA(cudaGraphLaunch(g->ms_exec, s));
        count_launch(4);
    } else {
        WEDGE_TRY(msbfs_enqueue(g, nroots, nqueries, d_levels, u8, init, sssp, s));
    }
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev1, s));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost, s));
    g->last_stream = s;
    g->last_trace = false;
    g->last_push = false;
    if (u8) {  // whether every level fit 8 bits is known only once the run ends
        WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
        if (g->h_ctl->status & kStatusLevelOverflow)
            return set_error(WEDGE_ERR_NOT_SUPPORTED,
                             "a level of 255 or more: 8-bit levels do not fit; use wedge_run_bfs_batch");
    }
    if (!stats) return WEDGE_OK;
    return fill_stats(g, s, stats);
}
}  // namespace wedge

extern "C" {

wedge_status wedge_run_bfs_batch(wedge_graph_t g, const uint32_t* roots, const uint32_t* root_query, uint32_t nroots,
                                 uint32_t nqueries, uint32_t* d_levels, const wedge_opts* opts, wedge_stats* stats,
                                 wedge_stream_t stream) {
    return run_batch(g, false, roots, root_query, nroots, nqueries, d_levels, false, opts, stats,
                     (cudaStream_t)stream);
}

wedge_status wedge_run_bfs_batch_u8(wedge_graph_t g, const uint32_t* roots, const uint32_t* root_query,
                                    uint32_t nroots, uint32_t nqueries, uint8_t* d_levels, const wedge_opts* opts,
                                    wedge_stats* stats, wedge_stream_t stream) {
    return run_batch(g, false, roots, root_query, nroots, nqueries, d_levels, true, opts, stats,
                     (cudaStream_t)stream);
}

wedge_status wedge_run_sssp_batch(wedge_graph_t g, const uint32_t* roots, const uint32_t* root_query,
                                  uint32_t nroots, uint32_t nqueries, uint32_t* d_dist, const wedge_opts* opts,
                                  wedge_stats* stats, wedge_stream_t stream) {
    return run_batch(g, true, roots, root_query, nroots, nqueries, d_dist, false, opts, stats, (cudaStream_t)stream);
}

wedge_status wedge_frontier_transform(wedge_graph_t g, const uint32_t* d_vertex_bitmap, uint32_t log2_coarsen,
                                      uint32_t* d_chunk_list, uint32_t* d_chunk_count, wedge_stream_t stream) {
    if (!g || !d_vertex_bitmap || !d_chunk_list || !d_chunk_count)
        return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (!valid_precision(log2_coarsen))
        return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be 0..7, or -1 / -2 (16- / 8-edge entries)");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((int)log2_coarsen < 0) WEDGE_TRY(ensure_fine(g, s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->rec, 0, sizeof(IterRec), s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(d_chunk_count, 0, 4, s));
    XformParams X = xform_params(g, 0);
    X.bm_in = d_vertex_bitmap;
    X.clist = d_chunk_list;
    X.count_out = d_chunk_count;
    X.standalone = 1;
    X.standalone_k = (int)log2_coarsen;
    launch_xform(g, X, s);
    k_clear_listed<<<g->num_sms * 4, 256, 0, s>>>(d_chunk_list, d_chunk_count, g->wb,
                                                  wb_words_at(g, (int)log2_coarsen));
    count_launch();
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

wedge_status wedge_frontier_transform_profile(wedge_graph_t g, const uint32_t* d_vertex_bitmap,
                                              uint32_t log2_coarsen, uint32_t schedule, uint32_t* d_chunk_list,
                                              uint32_t* d_chunk_count, uint64_t* d_warp_stats, uint32_t cap_warps,
                                              uint32_t* n_warps, wedge_stream_t stream) {
    if (!g || !n_warps) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (schedule > 1) return set_error(WEDGE_ERR_INVALID_ARG, "schedule must be 0 or 1");
    const uint32_t nw = (uint32_t)((uint64_t)g->xform_blocks * kXformThreads / 32);
    *n_warps = nw;
    if (!d_warp_stats) return WEDGE_OK;
    if (!d_vertex_bitmap || !d_chunk_list || !d_chunk_count) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (cap_warps < nw) return set_error(WEDGE_ERR_INVALID_ARG, "d_warp_stats holds fewer warps than the launch");
    if (!valid_precision(log2_coarsen))
        return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be 0..7, or -1 / -2 (16- / 8-edge entries)");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((int)log2_coarsen < 0) WEDGE_TRY(ensure_fine(g, s));
    if (!g->slice_ctr) WEDGE_TRY(dev_alloc(g, (void**)&g->slice_ctr, 16));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->rec, 0, sizeof(IterRec), s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(d_chunk_count, 0, 4, s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->slice_ctr, 0, 4, s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(d_warp_stats, 0, (size_t)nw * 8 * sizeof(uint64_t), s));
    XformParams X = xform_params(g, 0);
    X.bm_in = d_vertex_bitmap;
    X.clist = d_chunk_list;
    X.count_out = d_chunk_count;
    X.standalone = 1;
    X.standalone_k = (int)log2_coarsen;
    X.wstat = reinterpret_cast<unsigned long long*>(d_warp_stats);
    X.slice_ctr = g->slice_ctr;
    if (schedule == 0) {
        launch_xform(g, X, s);
    } else {
        k_xform_static<<<g->xform_blocks, kXformThreads, 0, s>>>(X);
        count_launch();
    }
    k_clear_listed<<<g->num_sms * 4, 256, 0, s>>>(d_chunk_list, d_chunk_count, g->wb,
                                                  wb_words_at(g, (int)log2_coarsen));
    count_launch();
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

wedge_status wedge_pull_iterate(wedge_graph_t g, wedge_app app, uint32_t* d_values, uint32_t iter,
                                const uint32_t* d_cur_bitmap, const uint32_t* d_chunk_list,
                                const uint32_t* d_chunk_count, uint32_t log2_coarsen, uint32_t* d_next_bitmap,
                                uint64_t* d_fullness, uint32_t* d_nfront, wedge_stream_t stream) {
    if (!g || !d_values || !d_next_bitmap || !d_fullness || !d_nfront)
        return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (app != WEDGE_BFS && app != WEDGE_CC && app != WEDGE_SSSP)
        return set_error(WEDGE_ERR_INVALID_ARG, "app must be BFS, CC or SSSP");
    if (app == WEDGE_BFS && !d_cur_bitmap) return set_error(WEDGE_ERR_INVALID_ARG, "BFS needs the current frontier");
    if (app == WEDGE_SSSP && !g->w && g->E) return set_error(WEDGE_ERR_INVALID_ARG, "SSSP needs edge weights");
    if (d_chunk_list && !d_chunk_count) return set_error(WEDGE_ERR_INVALID_ARG, "chunk list without count");
    if (!valid_precision(log2_coarsen))
        return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be 0..7, or -1 / -2 (16- / 8-edge entries)");
    if (iter + 2 >= g->rec_cap) return set_error(WEDGE_ERR_INVALID_ARG, "iter too large");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned sparse = d_chunk_list ? 1u : 0u;
    const unsigned cap = (unsigned)entries_at(g, (int)log2_coarsen);
    k_standalone_prep<<<1, 32, 0, s>>>(g->rec, g->ctl, iter, sparse, log2_coarsen, d_chunk_count, cap);
    PullParams P = pull_params(g, 0);
    P.decide = 0;  // one pull: k_standalone_out reduces the block slots
    P.vals = d_values;
    P.vread = d_values;
    P.bm[iter & 1] = const_cast<uint32_t*>(d_cur_bitmap ? d_cur_bitmap : d_next_bitmap);
    P.bm[(iter + 1) & 1] = d_next_bitmap;
    P.clist = d_chunk_list ? d_chunk_list : g->clist;
    P.wb = nullptr;  // a caller's list has no library bitmap behind it
    launch_pull_app(g, app, P, s);
    k_standalone_out<<<1, 256, 0, s>>>(g->bstat, pull_grid(g, app, P), reinterpret_cast<unsigned long long*>(d_fullness),
                                       d_nfront);
    count_launch(2);
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

wedge_status wedge_graph_set_tuning(wedge_graph_t g, const wedge_tuning* t) {
    if (!g || !t) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (t->dense_loader > 1) return set_error(WEDGE_ERR_INVALID_ARG, "dense_loader must be 0 or 1");
    if (t->edge_index > 1) return set_error(WEDGE_ERR_INVALID_ARG, "edge_index must be 0 or 1");
    for (uint32_t r : t->reserved)
        if (r) return set_error(WEDGE_ERR_INVALID_ARG, "reserved tuning fields must be zero");
    DeviceGuard dg(g->device);
    WEDGE_TRY_CUDA(cudaDeviceSynchronize());
    if (t->edge_index == 1) {
        WEDGE_TRY(build_eidx_z(g, g->cap_stream));
        WEDGE_TRY_CUDA(cudaStreamSynchronize(g->cap_stream));
    }
    g->tuning = *t;
    for (auto& e : g->loop_exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    if (g->pr_exec) {
        cudaGraphExecDestroy(g->pr_exec);
        g->pr_exec = nullptr;
    }
    g->loop_failed = false;
    return configure_pulls(g);
}

wedge_status wedge_graph_get_tuning(wedge_graph_t g, wedge_tuning* out) {
    if (!g || !out) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    *out = g->tuning;
    return WEDGE_OK;
}

// Candidate-timing trace (training data of the learned switch; not in the
// paper).  Runs `app` with the threshold policy; before each pull it times
// every candidate (transformation + pull, CUDA events) from the same
// snapshotted state, then restores the state and advances with the
// threshold's choice.
wedge_status wedge_trace_candidates(wedge_graph_t g, wedge_app app, uint32_t root, const wedge_opts* opts_in,
                                    uint32_t max_iters, float* h_features, float* h_ms, uint32_t* h_chosen,
                                    uint32_t cap, uint32_t* n_iters, wedge_stream_t stream) {
    if (!g || !h_features || !h_ms || !h_chosen || !n_iters) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (app != WEDGE_BFS && app != WEDGE_CC && app != WEDGE_SSSP)
        return set_error(WEDGE_ERR_INVALID_ARG, "app must be BFS, CC or SSSP");
    if (app != WEDGE_CC && root >= g->V) return set_error(WEDGE_ERR_INVALID_ARG, "root out of range");
    if (app == WEDGE_SSSP && !g->w && g->E) return set_error(WEDGE_ERR_INVALID_ARG, "SSSP needs edge weights");
    wedge_opts o;
    if (opts_in) o = *opts_in;
    else wedge_default_opts(app, &o);
    WEDGE_TRY(check_opts(&o));
    if (o.log2_coarsen >= kCandidates - 1) return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be <= 4");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!g->snap_vals) WEDGE_TRY(dev_alloc(g, (void**)&g->snap_vals, (uint64_t)g->V * 4));
    if (!g->snap_visk) WEDGE_TRY(dev_alloc(g, (void**)&g->snap_visk, visk_words(g) * 4));
    const uint64_t kbytes = visk_words(g) * 4;
    const uint32_t limit = max_iters ? (max_iters < kDefaultMaxIters ? max_iters : kDefaultMaxIters)
                                     : kDefaultMaxIters;
    RunCtl init{};
    init.max_iters = limit;
    init.switch_mode = o.switch_mode == WEDGE_SWITCH_LEARNED ? WEDGE_SWITCH_THRESHOLD : o.switch_mode;
    init.tau_bp = o.tau_bp;
    init.k = o.log2_coarsen;
    init.E = g->E;
    PullParams P = pull_params(g, 0, app);
    P.mlp = nullptr;
    XformParams X = xform_params(g, 0);
    k_run_init<<<g->num_sms * 4, 256, 0, s>>>(app, g->V, root, g->vals, g->bm[0], g->bm[1], g->wb,
                                              g->wb_words, g->rec, g->ctl, init, g->flist[0], g->visk,
                                              visk_words(g));
    k_frontier_stats<<<g->num_sms * 4, 256, 0, s>>>(g->bm[0], g->V, g->outdeg, g->eidx_off, g->rec, g->ctl, nullptr,
                                                    P.gf);
    count_launch(2);
    WEDGE_TRY_CUDA(cudaGetLastError());
    const uint64_t vbytes = (uint64_t)g->V * 4;
    uint32_t t = 0;
    for (; t < cap; ++t) {
        RunCtl hc;
        IterRec hr;
        WEDGE_TRY_CUDA(cudaMemcpyAsync(&hc, g->ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost, s));
        WEDGE_TRY_CUDA(cudaMemcpyAsync(&hr, g->rec + t, sizeof(IterRec), cudaMemcpyDeviceToHost, s));
        WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
        if (hc.done || hc.it != t) break;
        for (int c = 0; c < kCandidates; ++c)
            mlp_features(P.gf, (double)g->E, hr.nfront, (double)hr.fullness, hr.rowsum, t, c,
                         h_features + ((size_t)t * kCandidates + c) * kMlpIn);
        h_chosen[t] = hr.mode ? hr.k + 1 : 0;
        WEDGE_TRY_CUDA(cudaMemcpyAsync(g->snap_vals, g->vals, vbytes, cudaMemcpyDeviceToDevice, s));
        if (app == WEDGE_BFS)
            WEDGE_TRY_CUDA(cudaMemcpyAsync(g->snap_visk, g->visk, kbytes, cudaMemcpyDeviceToDevice, s));
        for (int c = 0; c <= kCandidates; ++c) {
            // c < kCandidates: time candidate c; c == kCandidates: advance
            IterRec cr = hr;
            if (c < kCandidates) {
                cr.mode = c > 0;
                cr.k = c > 0 ? (unsigned)(c - 1) : hr.k;
            }
            WEDGE_TRY_CUDA(cudaMemcpyAsync(g->vals, g->snap_vals, vbytes, cudaMemcpyDeviceToDevice, s));
            if (app == WEDGE_BFS)
                WEDGE_TRY_CUDA(cudaMemcpyAsync(g->visk, g->snap_visk, kbytes, cudaMemcpyDeviceToDevice, s));
            // a previous candidate's pull marked its frontier in the next bitmap
            WEDGE_TRY_CUDA(cudaMemsetAsync(g->bm[(t + 1) & 1], 0, ((uint64_t)g->V + 31) / 32 * 4, s));
            k_ctl_init<<<1, 32, 0, s>>>(g->ctl, hc);
            k_rec_set<<<1, 32, 0, s>>>(g->rec, t, cr);
            count_launch(2);
            WEDGE_TRY_CUDA(cudaEventRecord(g->ev0, s));
            launch_xform(g, X, s);
            launch_pull_app(g, app, P, s);
            WEDGE_TRY_CUDA(cudaEventRecord(g->ev1, s));
            WEDGE_TRY_CUDA(cudaGetLastError());
            if (c < kCandidates) {
                WEDGE_TRY_CUDA(cudaEventSynchronize(g->ev1));
                float ms = 0.f;
                WEDGE_TRY_CUDA(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
                h_ms[(size_t)t * kCandidates + c] = ms;
            }
        }
    }
    WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    *n_iters = t;
    g->last_stream = s;
    WEDGE_TRY_CUDA(cudaMemcpy(g->h_ctl, g->ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost));
    return WEDGE_OK;
}

wedge_status wedge_get_trace(wedge_graph_t g, wedge_iter_record* out, uint32_t cap, uint32_t* n) {
    if (!g || !n || (!out && cap)) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(g->device);
    WEDGE_TRY_CUDA(cudaStreamSynchronize(g->last_stream));
    const uint32_t iters = g->h_ctl->it;
    *n = iters;
    const uint32_t m = iters < cap ? iters : cap;
    if (!m) return WEDGE_OK;
    std::vector<IterRec> r(m);
    WEDGE_TRY_CUDA(cudaMemcpy(r.data(), g->rec, (size_t)m * sizeof(IterRec), cudaMemcpyDeviceToHost));
    for (uint32_t t = 0; t < m; ++t) {
        out[t].fullness = r[t].fullness;
        out[t].nfront = r[t].nfront;
        out[t].mode = r[t].mode;
        out[t].log2_coarsen = r[t].k;
        out[t].nchunks = r[t].nchunks;
        out[t].rowsum = r[t].rowsum;
        out[t].npieces = r[t].npieces;
        out[t].t_pull_ns = (r[t].t_pull1 > r[t].t_pull0 && r[t].t_pull0) ? r[t].t_pull1 - r[t].t_pull0 : 0;
        out[t].t_xform_ns = (r[t].t_xf1 > r[t].t_xf0 && r[t].t_xf0) ? r[t].t_xf1 - r[t].t_xf0 : 0;
    }
    return WEDGE_OK;
}

}  // extern "C"

// The pull (Sections 2.1, 3.2; K1/K4 with the frontier epilogue K5) and the
// fullness decision its last block takes (Section 3.4, Fig. 5): the
// kernel parameters, the applications' per-edge operators, the dense and
// sparse pulls over the CSC chunks, and the decision step.  Included by
// engine.cu only.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "mlp.cuh"
#include "tma.cuh"

namespace wedge {


// Sparse BFS pulls over fewer listed chunks than this do not check visited
// destinations (measured on the rewired 4096^2 grid: the extra dependent
// load cost 4% there, while R-MAT's large sparse pulls gain from the check).
constexpr unsigned long long kSkipVisitedMinChunks = 1ull << 14;
enum AppId { kBFS = 0, kCC = 1, kSSSP = 2, kPR = 3, kMSBFS = 4 };
// Resident 256-thread blocks per SM that the register allocation of a
// direct-load pull must allow.  Measured on R-MAT s22: 4 blocks (64
// registers) beat 5 (48 registers) for every application -- BFS by 25%, as
// the fifth block's shared memory comes out of the L1 that caches the
// frontier bitmap, and PageRank by 15%, as 48 registers spill.
#ifndef WEDGE_MIN_BLOCKS_BFS
#define WEDGE_MIN_BLOCKS_BFS 4
#endif
#ifndef WEDGE_MIN_BLOCKS_CC
#define WEDGE_MIN_BLOCKS_CC 4
#endif
#ifndef WEDGE_MIN_BLOCKS_SSSP
#define WEDGE_MIN_BLOCKS_SSSP 4
#endif
#ifndef WEDGE_MIN_BLOCKS_PR
#define WEDGE_MIN_BLOCKS_PR 4
#endif
constexpr int direct_min_blocks(int app) {
    return app == kBFS ? WEDGE_MIN_BLOCKS_BFS
                       : app == kCC ? WEDGE_MIN_BLOCKS_CC : app == kSSSP ? WEDGE_MIN_BLOCKS_SSSP : WEDGE_MIN_BLOCKS_PR;
}

// ------------------------------------------------------------------------
// Kernel parameter blocks
// ------------------------------------------------------------------------
struct PullParams {
    const uint32_t* src;
    const uint32_t* w;
    const uint2* cmeta;          // padded: entries up to a full tile past NC
    const uint32_t* vid;
    const uint32_t* outdeg;
    const uint32_t* eidx_off;
    unsigned long long E;
    unsigned long long NC;
    uint32_t* vals;              // BFS levels / CC labels / SSSP distances (written by the pull)
    const uint32_t* vread;       // CC/SSSP values the pull gathers: vals, or the previous
                                 // iteration's buffer in synchronous runs
    uint32_t* bm[2];             // vertex frontier bitmaps indexed by iteration parity
    const uint32_t* clist;       // Wedge Frontier list (sparse pulls)
    uint32_t* wb;                // Wedge Frontier bitmap: consumed words are zeroed
    IterRec* rec;
    RunCtl* ctl;
    const float* contrib;        // PageRank: pr(u)/outdeg(u)
    unsigned long long* acc;     // PageRank: fixed-point in-edge sums
    unsigned int pr_iter;
    int trace;
    int dense_tma;               // dense pulls stage tiles with bulk copies
    const __nv_bfloat16* mlp;    // learned switch weights (nullptr: threshold)
    GraphFeat gf;                // graph statistics of the learned switch's features
    // batched BFS: per-vertex 64-bit query masks and the vertex-major levels
    unsigned long long* fb[2];   // frontier masks by iteration parity
    unsigned long long* seen;    // queries that have reached each vertex
    uint32_t* levels;            // levels[v * Q + q]
    uint8_t* levels8;            // non-null: 8-bit batched BFS levels instead (0xFF: unreached)
    uint32_t Q;
    uint32_t* flist[2];          // frontier vertex lists by iteration parity
    BlockStat* bstat;            // per-block results
    uint32_t* visk;              // BFS runs: visited bit per destination index (nullptr: no skipping)
    int decide;                  // runs: the pull's last block takes the decision for the next pull
    int hybrid;                  // push/pull hybrid runs: the pull only serves dense iterations
    cudaGraphConditionalHandle cond;  // device loop: the while node's condition (0 outside a graph)
};

// The push/pull hybrid's out-edges and work pieces (rows of the frontier's
// out-edges cut into pieces of at most 32 edges by k_xform_scan).
struct PushParams {
    const uint32_t* dst;         // CSR: edge j ends at dst[j]
    const uint32_t* src;         //      and leaves src[j]
    const uint32_t* w;           //      with weight w[j] (SSSP)
    const uint32_t* kid_of;      // index of a vertex in vid (BFS visited bits)
    const uint2* pieces;
};

// ------------------------------------------------------------------------
// Application traits: per-edge candidate and combine operator
// ------------------------------------------------------------------------
template <int APP>
struct Traits;
template <>
struct Traits<kBFS> {  // found-a-parent flag, OR
    using T = uint32_t;
    static __device__ __forceinline__ T neutral() { return 0u; }
    static __device__ __forceinline__ T op(T a, T b) { return a | b; }
    static __device__ __forceinline__ bool keep(T a) { return a != 0u; }
};
template <>
struct Traits<kCC> {  // label, min
    using T = uint32_t;
    static __device__ __forceinline__ T neutral() { return kInf; }
    static __device__ __forceinline__ T op(T a, T b) { return a < b ? a : b; }
    static __device__ __forceinline__ bool keep(T a) { return a != kInf; }
};
template <>
struct Traits<kSSSP> {  // distance, min
    using T = uint32_t;
    static __device__ __forceinline__ T neutral() { return kInf; }
    static __device__ __forceinline__ T op(T a, T b) { return a < b ? a : b; }
    static __device__ __forceinline__ bool keep(T a) { return a != kInf; }
};
template <>
struct Traits<kMSBFS> {  // union of the sources' frontier query masks, OR
    using T = unsigned long long;
    static __device__ __forceinline__ T neutral() { return 0ull; }
    static __device__ __forceinline__ T op(T a, T b) { return a | b; }
    static __device__ __forceinline__ bool keep(T a) { return a != 0ull; }
};
template <>
struct Traits<kPR> {  // fixed-point contribution, sum (every segment is stored)
    using T = unsigned long long;
    static __device__ __forceinline__ T neutral() { return 0ull; }
    static __device__ __forceinline__ T op(T a, T b) { return a + b; }
    static __device__ __forceinline__ bool keep(T) { return true; }
};

template <int APP>
__device__ __forceinline__ typename Traits<APP>::T candidate(const PullParams& P, const uint32_t* cur, uint32_t u,
                                                             uint32_t w, unsigned it) {
    if constexpr (APP == kBFS) {
        return (__ldg(cur + (u >> 5)) >> (u & 31)) & 1u;
    } else if constexpr (APP == kCC) {
        return P.vread[u];
    } else if constexpr (APP == kMSBFS) {
        // written earlier in the same persistent launch: read through L2
        return __ldcg(((it & 1) ? P.fb[1] : P.fb[0]) + u);
    } else if constexpr (APP == kSSSP) {
        const uint32_t d = P.vread[u];
        if (d == kInf) return kInf;
        const unsigned long long s = (unsigned long long)d + w;
        return s > kSat ? kSat : (uint32_t)s;
    } else {
        // exact 64-bit fixed point of the FP32 contribution (2^-62 units)
        return __float2ull_rn(__ldg(P.contrib + u) * 0x1p62f);
    }
}

__device__ __forceinline__ bool set_bit(uint32_t* bm, uint32_t v) {
    const uint32_t bit = 1u << (v & 31);
    return (atomicOr(bm + (v >> 5), bit) & bit) == 0;
}

// The fullness decision (Section 3.4, "Frontier Fullness Threshold"; Fig. 5)
// for pull it_next, taken by one block once every block has published its
// frontier sums.  With the learned switch, the block first evaluates the
// cost model on the six candidates (dense; Wedge Frontier with k = 0..4):
// BF16 weights and activations, FP32 accumulation; the lowest predicted
// time wins.  Without a model, or if no prediction is finite, the threshold
// decides.  `sm` needs kDecideSmemBytes of shared memory: the activations
// and features, then a copy of the weights (read straight from global memory
// inside the dot products, each decision took ~20 us).  The device copy
// stores W2 k-major, so that the threads of a layer read consecutive
// weights; stage_model() copies it with 16-byte loads (`staged`: done
// already, overlapped with other loads by the caller).
constexpr int kDecideFloats = 2 * kCandidates * kMlpHidden + 8 + kCandidates * kMlpIn;
constexpr int kModelBytes16 = ((kMlpParams * 2 + 15) / 16) * 16;
constexpr int kDecideSmemBytes = kDecideFloats * 4 + kModelBytes16;
static_assert((kDecideFloats * 4) % 16 == 0, "weights must start 16-byte aligned");

__device__ __forceinline__ void stage_model(const __nv_bfloat16* mlp_global, float* sm) {
    uint4* dst = reinterpret_cast<uint4*>(sm + kDecideFloats);
    const uint4* src = reinterpret_cast<const uint4*>(mlp_global);
    for (int i = threadIdx.x; i < kModelBytes16 / 16; i += blockDim.x) dst[i] = __ldg(src + i);
}

__device__ void decide_block(IterRec* rec, RunCtl* C, unsigned it_next, const __nv_bfloat16* mlp_global,
                             const GraphFeat& gf, float* sm, bool staged = false) {
    IterRec* r = rec + it_next;
    const unsigned long long F = __ldcg(&r->fullness);
    const unsigned nf = __ldcg(&r->nfront);
    const unsigned rows = __ldcg(&r->rowsum);
    const bool model = C->switch_mode == WEDGE_SWITCH_LEARNED && mlp_global != nullptr && nf > 0;
    const float frac = C->E ? (float)((double)F / (double)C->E) : 0.f;
    const bool learned = model && frac >= gf.band_lo && frac <= gf.band_hi;
    float* h1 = sm;
    float* h2 = sm + kCandidates * kMlpHidden;
    float* out = sm + 2 * kCandidates * kMlpHidden;
    float* xs = out + 8;  // the candidates' features, BF16-rounded
    __nv_bfloat16* mlp = reinterpret_cast<__nv_bfloat16*>(sm + kDecideFloats);
    __nv_bfloat16* w2t = mlp + kMlpW2;  // W2 transposed: w2t[k * 64 + j] = W2[j][k]
    if (learned) {
        if (!staged) stage_model(mlp_global, sm);
        if (threadIdx.x < kCandidates) {
            float x[kMlpIn];
            mlp_features(gf, (double)C->E, nf, (double)F, rows, it_next, threadIdx.x, x);
            for (int f = 0; f < kMlpIn; ++f) xs[threadIdx.x * kMlpIn + f] = __bfloat162float(__float2bfloat16_rn(x[f]));
        }
        __syncthreads();
        for (int o = threadIdx.x; o < kCandidates * kMlpHidden; o += blockDim.x) {
            const int c = o / kMlpHidden, j = o % kMlpHidden;
            float a = __bfloat162float(mlp[kMlpB1 + j]);
            for (int f = 0; f < kMlpIn; ++f)
                a = fmaf(__bfloat162float(mlp[kMlpW1 + j * kMlpIn + f]), xs[c * kMlpIn + f], a);
            h1[o] = __bfloat162float(__float2bfloat16_rn(fmaxf(a, 0.f)));
        }
        __syncthreads();
        for (int o = threadIdx.x; o < kCandidates * kMlpHidden; o += blockDim.x) {
            const int c = o / kMlpHidden, j = o % kMlpHidden;
            float a = __bfloat162float(mlp[kMlpB2 + j]);
            for (int k = 0; k < kMlpHidden; ++k)
                a = fmaf(__bfloat162float(w2t[k * kMlpHidden + j]), h1[c * kMlpHidden + k], a);
            h2[o] = __bfloat162float(__float2bfloat16_rn(fmaxf(a, 0.f)));
        }
        __syncthreads();
        if (threadIdx.x < kCandidates) {
            float y = __bfloat162float(mlp[kMlpB3]);
            for (int j = 0; j < kMlpHidden; ++j)
                y = fmaf(__bfloat162float(mlp[kMlpW3 + j]), h2[threadIdx.x * kMlpHidden + j], y);
            out[threadIdx.x] = y;
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    int choice = -1;
    if (learned) {
        float best = 0.f;
        for (int c = 0; c < kCandidates; ++c)
            if (isfinite(out[c]) && (choice < 0 || out[c] < best)) {
                best = out[c];
                choice = c;
            }
    } else if (model) {
        choice = frac < gf.band_lo ? 1 : 0;  // outside the band: no inference
    }
    unsigned sparse, k = C->k;
    if (choice >= 0) {
        sparse = choice > 0;
        if (sparse) k = (unsigned)(choice - 1);
    } else if (C->switch_mode == WEDGE_SWITCH_ALWAYS_DENSE) {
        sparse = 0;
    } else if (C->switch_mode == WEDGE_SWITCH_ALWAYS_SPARSE) {
        sparse = 1;
    } else {
        sparse = (F * 10000ull < (unsigned long long)C->tau_bp * C->E) ? 1u : 0u;
    }
    r->mode = sparse;
    r->k = k;
    if (nf == 0) {
        C->done = 1;
    } else if (it_next >= C->max_iters) {
        C->done = 1;
        C->status |= kStatusMaxIters;
    }
    C->it = it_next;
}

struct Stats {
    unsigned long long F;
    unsigned int n;
    unsigned int row;
    unsigned int rowmax;
};

// A vertex activated for the next frontier: its out-degree (fullness), its
// edge-index row length (a feature of the learned switch; the longest row
// decides whether the transformation may expand rows directly) and the
// count.
__device__ __forceinline__ void count_active(const PullParams& P, uint32_t v, Stats& st) {
    st.F += __ldg(P.outdeg + v);
    st.n += 1;
    const uint32_t len = __ldg(P.eidx_off + v + 1) - __ldg(P.eidx_off + v);
    st.row += len;
    st.rowmax = max(st.rowmax, len);
}

// The block's frontier list (whole warp): one shared-memory reservation per
// warp and call, none once the block's stage has overflowed.
__device__ __forceinline__ void stage_list(bool act, uint32_t v, unsigned* s_lcnt, uint32_t* s_list) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned am = __ballot_sync(kFull, act);
    if (am && *reinterpret_cast<volatile unsigned*>(s_lcnt) <= (unsigned)kListCap) {
        const unsigned leader = __ffs(am) - 1;
        unsigned base = 0;
        if (lane == leader) base = atomicAdd(s_lcnt, (unsigned)__popc(am));
        base = __shfl_sync(kFull, base, leader);
        const unsigned slot = base + __popc(am & ((1u << lane) - 1u));
        if (act && slot < (unsigned)kListCap) s_list[slot] = v;
    }
}

// ------------------------------------------------------------------------
// One warp slice of the pull (K1/K4 + K5): kEPL = 8 consecutive edges per
// lane, edges o .. o+7 of the lane's chunk c (dense pulls: lane L holds
// edges 8*(L&3) .. +7 of slice chunk L>>2; sparse pulls: the lanes' 8-edge
// units as listed).  lane_break: the previous lane does not hold the 8
// edges just before this lane's (a run of lanes starts here).
//
// Destinations come from the chunk's head mask (bit i: position 32c+i is
// the first in-edge of its destination) and the index of the destination of
// position 32c.  Each lane combines its edges per destination; a segmented
// scan across lanes carries partial segments.  Every segment end becomes a
// record (destination index, combined value) in the warp's shared buffer;
// the warp then applies the records with all 32 lanes.  A segment that starts
// at its destination's first edge and ends just before the next
// destination's first edge holds all in-edges of that destination: its
// record is applied with a plain read-modify-write, others with atomics.
// ------------------------------------------------------------------------
template <int APP>
__device__ __forceinline__ void apply_records(const PullParams& P, unsigned it, uint32_t* next, const uint32_t* s_kid,
                                              const typename Traits<APP>::T* s_val, unsigned base, unsigned end,
                                              Stats& st, unsigned* s_lcnt, uint32_t* s_list);

template <int APP>
__device__ __forceinline__ void process_slice(const PullParams& P, unsigned it, const uint32_t* cur, uint32_t* next,
                                              const uint32_t (&sv)[kEPL], const uint32_t (&wv)[kEPL], int nvalid,
                                              uint32_t live, unsigned long long c, uint2 meta, unsigned next_head,
                                              unsigned o, bool lane_break,
                                              uint32_t* s_kid, typename Traits<APP>::T* s_val, Stats& st,
                                              unsigned* s_lcnt, uint32_t* s_list) {
    using Tr = Traits<APP>;
    using T = typename Tr::T;
    const unsigned lane = threadIdx.x & 31;
    const uint32_t heads = meta.x;
    const uint32_t vmask = (nvalid >= 8) ? 0xFFu : ((1u << nvalid) - 1u);
    const uint32_t hb = (heads >> o) & vmask;
    const uint32_t brk = (hb | (lane_break ? 1u : 0u)) & vmask;
    live &= vmask;

    T inc[kEPL];
    T run = Tr::neutral();
#pragma unroll
    for (int i = 0; i < kEPL; ++i) {
        const T cv = ((live >> i) & 1u) ? candidate<APP>(P, cur, sv[i], wv[i], it) : Tr::neutral();
        run = ((brk >> i) & 1u) ? cv : Tr::op(run, cv);
        inc[i] = run;
    }
    // Segmented scan of the lanes' tail values.  A lane with a break (or no
    // edges) starts a run of lanes; lane L's run starts at the highest such
    // lane <= L, found by ballot, so only the values move through shuffles.
    const unsigned below_me = (1u << lane) - 1u;
    const int last_brk = brk ? 31 - __clz(brk) : -1;
    const unsigned Fm = __ballot_sync(kFull, brk != 0 || nvalid == 0);
    // does the tail segment of a breaking lane start at a destination's first edge?
    const unsigned Sm = __ballot_sync(kFull, brk ? ((hb >> last_brk) & 1u) : 0u);
    const unsigned fle = Fm & (below_me | (1u << lane));
    const unsigned start = fle ? 31 - __clz(fle) : 0u;
    T v = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T v2 = __shfl_up_sync(kFull, v, d);
        if (lane >= start + d) v = Tr::op(v2, v);
    }
    T carry = __shfl_up_sync(kFull, v, 1);
    if (lane == 0) carry = Tr::neutral();
    const unsigned flt = Fm & below_me;
    const unsigned carry_sr = flt ? (Sm >> (31 - __clz(flt))) & 1u : 0u;
    // does this lane's last segment end at its last edge?
    const unsigned nb0 = __ballot_sync(kFull, brk & 1u);
    const unsigned nbv = __ballot_sync(kFull, nvalid > 0);
    const unsigned up = lane < 31 ? 2u << lane : 0u;
    const bool nx_valid = (nbv & up) != 0;
    const bool tail_close = nvalid > 0 && (nvalid < kEPL || !nx_valid || (nb0 & up) != 0);
    const bool next_past_end = c * 32 + o + kEPL >= P.E;
    const bool tail_real = nvalid < kEPL || next_past_end ||
                           ((o == 32 - kEPL) ? (next_head != 0) : (((heads >> (o + kEPL)) & 1u) != 0));
    // record positions: every break b >= 1 closes a segment at b-1; plus the tail
    uint32_t R = brk >> 1;
    if (tail_close) R |= 1u << (nvalid - 1);
    const int first = brk ? __ffs(brk) - 1 : kEPL;
    T rv[kEPL];
    uint32_t K = 0, X = 0;
#pragma unroll
    for (int e = 0; e < kEPL; ++e) {
        rv[e] = Tr::neutral();
        if ((R >> e) & 1u) {
            const T val = (e < first) ? Tr::op(carry, inc[e]) : inc[e];
            rv[e] = val;
            if (Tr::keep(val)) {
                K |= 1u << e;
                const uint32_t below = brk & ((2u << e) - 1u);
                const int lb = below ? 31 - __clz(below) : 0;
                const unsigned sreal = (e < first) ? carry_sr : ((hb >> lb) & 1u);
                const unsigned ereal = (e == nvalid - 1 && tail_close) ? (unsigned)tail_real : 1u;
                X |= (sreal & ereal) << e;
            }
        }
    }
    // compact the records of the warp into its shared buffer: the exclusive
    // prefix of the lanes' record counts (at most 8, four bits) by ballots
    const unsigned cnt = __popc(K);
    unsigned slot = 0, total = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const unsigned Bb = __ballot_sync(kFull, (cnt >> b) & 1u);
        slot += (unsigned)__popc(Bb & below_me) << b;
        total += (unsigned)__popc(Bb) << b;
    }
    // the buffer holds kRecCap records: more take further passes (a slice
    // of many short segments), so that little shared memory is taken from L1
    for (unsigned base = 0; base < total; base += kRecCap) {
        if (base) __syncwarp();  // the previous pass's records are applied
        unsigned sl = slot;
#pragma unroll
        for (int e = 0; e < kEPL; ++e) {
            if ((K >> e) & 1u) {
                if (sl - base < (unsigned)kRecCap) {
                    const uint32_t kid = meta.y + __popc(heads & ((2u << (o + e)) - 1u) & ~1u);
                    s_kid[sl - base] = kid | (((X >> e) & 1u) << 31);
                    s_val[sl - base] = rv[e];
                }
                ++sl;
            }
        }
        __syncwarp();
        const unsigned end = total - base < (unsigned)kRecCap ? total : base + kRecCap;
        apply_records<APP>(P, it, next, s_kid, s_val, base, end, st, s_lcnt, s_list);
    }
    __syncwarp();
}

// Applies records base .. end-1 of the warp's buffer (entry r - base) with
// the warp's lanes: exclusive records by plain read-modify-write, others by
// atomics; activated vertices are added to the frontier sums and staged for
// the block's frontier list.
template <int APP>
__device__ __forceinline__ void apply_records(const PullParams& P, unsigned it, uint32_t* next, const uint32_t* s_kid,
                                              const typename Traits<APP>::T* s_val, unsigned base, unsigned end,
                                              Stats& st, unsigned* s_lcnt, uint32_t* s_list) {
    using T = typename Traits<APP>::T;
    const unsigned lane = threadIdx.x & 31;
    for (unsigned r0 = base; r0 < end; r0 += 32) {
        const unsigned r = r0 + lane;
        bool act = false;
        uint32_t dv = 0;
        if (r < end) {
            const uint32_t kx = s_kid[r - base];
            const T m = s_val[r - base];
            const bool excl = kx >> 31;
            dv = __ldg(P.vid + (kx & 0x7FFFFFFFu));
            if constexpr (APP == kBFS) {
                if (P.vals[dv] == kInf) {
                    P.vals[dv] = it + 1;
                    act = set_bit(next, dv);
                    if (P.visk) {
                        const uint32_t kid = kx & 0x7FFFFFFFu;
                        atomicOr(P.visk + (kid >> 5), 1u << (kid & 31));
                    }
                }
            } else if constexpr (APP == kMSBFS) {
                // queries reaching dv for the first time take level it+1
                unsigned long long* nxt = (it & 1) ? P.fb[0] : P.fb[1];
                unsigned long long fresh, prev;
                if (excl) {
                    const unsigned long long old = __ldcg(P.seen + dv);
                    fresh = m & ~old;
                    if (fresh) P.seen[dv] = old | fresh;
                } else {
                    fresh = m & ~atomicOr(P.seen + dv, m);
                }
                if (fresh) {
                    if (P.levels8 && it + 1 >= 255u) {
                        atomicOr(&P.ctl->status, kStatusLevelOverflow);  // not representable: the run stops
                    } else {
                        for (unsigned long long b = fresh; b; b &= b - 1) {
                            const size_t at = (size_t)dv * P.Q + (__ffsll((long long)b) - 1);
                            if (P.levels8) P.levels8[at] = (uint8_t)(it + 1);
                            else P.levels[at] = it + 1;
                        }
                    }
                    if (excl) {
                        prev = __ldcg(nxt + dv);
                        nxt[dv] = prev | fresh;
                    } else {
                        prev = atomicOr(nxt + dv, fresh);
                    }
                    act = prev == 0ull && set_bit(next, dv);
                }
            } else if constexpr (APP == kPR) {
                if (excl) P.acc[dv] = m;
                else if (m) atomicAdd(P.acc + dv, m);
            } else {
                bool changed;
                if (excl) {
                    const uint32_t old = P.vals[dv];
                    changed = m < old;
                    if (changed) P.vals[dv] = m;
                } else {
                    changed = m < atomicMin(P.vals + dv, m);
                }
                act = changed && set_bit(next, dv);
            }
            if (act) count_active(P, dv, st);
        }
        if constexpr (APP != kPR) stage_list(act, dv, s_lcnt, s_list);
    }
}

template <int APP>
constexpr int pull_records_bytes() {
    using T = typename Traits<APP>::T;
    return kCW * kRecCap * (4 + (int)sizeof(T));
}

template <int APP>
constexpr int pull_stage_bytes() {
    return 2 * kStages * 8                                        // mbarriers
           + kStages * kTileE * 4 * (APP == kSSSP ? 2 : 1)        // src (+ w)
           + kStages * (kTileC + kMetaPad) * 8;                   // chunk metadata
}

// Shared memory of a pull: the record buffers and the block's frontier
// list, plus the stages when dense pulls use bulk copies.
// (PageRank keeps no frontier list)
template <int APP>
constexpr int pull_list_bytes() {
    return APP == kPR ? 0 : kListCap * 4;
}

template <int APP>
constexpr int pull_smem_bytes(bool tma) {
    return pull_records_bytes<APP>() + pull_list_bytes<APP>() + (tma ? pull_stage_bytes<APP>() : 0);
}

// ... at least the decision's activations and weights for the applications
// whose last pull block decides (it reuses the block's buffers)
template <int APP>
constexpr int pull_launch_smem(bool tma) {
    return (APP != kPR && pull_smem_bytes<APP>(tma) < kDecideSmemBytes) ? kDecideSmemBytes : pull_smem_bytes<APP>(tma);
}

// Which of a lane's edges still have to be pulled: bit i is set if edge
// o + i of the chunk is valid and, for BFS runs, its destination is not yet
// visited (Section 5: the BFS pull skips visited vertices whatever the
// frontier).  The destinations of the lane's 8 edges are the consecutive
// indices kid0 .. kid0 + 7 at most, so one or two bitmap words cover them.
// The bitmap only gains bits during a run, so a stale word only costs work.
template <int APP>
__device__ __forceinline__ uint32_t lane_live(const PullParams& P, uint2 meta, unsigned o, int nvalid,
                                              bool skip_visited = true) {
    const uint32_t vmask = (nvalid >= kEPL) ? 0xFFu : ((1u << nvalid) - 1u);
    if constexpr (APP != kBFS) {
        return vmask;
    } else {
        if (!P.visk || !skip_visited || nvalid == 0) return vmask;
        const uint32_t heads = meta.x;
        const uint32_t kid0 = meta.y + __popc(heads & ~1u & ((2u << o) - 1u));
        const uint32_t* wp = P.visk + (kid0 >> 5);
        unsigned long long win = wp[0];
        if ((kid0 & 31) > 32 - kEPL) win |= (unsigned long long)wp[1] << 32;
        win >>= (kid0 & 31);
        const uint32_t hn = heads >> (o + 1);
        uint32_t live = 0;
#pragma unroll
        for (int i = 0; i < kEPL; ++i) {
            const unsigned r = __popc(hn & ((1u << i) - 1u));
            live |= (((unsigned)(win >> r) & 1u) ^ 1u) << i;
        }
        return live & vmask;
    }
}

// A lane's 8 consecutive edges (and weights) straight from global memory;
// a half whose edges are all skipped (live) is not loaded.
template <int APP>
__device__ __forceinline__ void load_lane_edges(const PullParams& P, unsigned long long e_lane, int nvalid,
                                                uint32_t live, uint32_t (&sv)[kEPL], uint32_t (&wv)[kEPL]) {
    if (nvalid == kEPL) {
        uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a;
        if (live & 0x0Fu) a = ld_stream(P.src + e_lane);
        if (live & 0xF0u) b = ld_stream(P.src + e_lane + 4);
        sv[0] = a.x; sv[1] = a.y; sv[2] = a.z; sv[3] = a.w;
        sv[4] = b.x; sv[5] = b.y; sv[6] = b.z; sv[7] = b.w;
        if constexpr (APP == kSSSP) {
            const uint4 x = ld_stream(P.w + e_lane);
            const uint4 y = ld_stream(P.w + e_lane + 4);
            wv[0] = x.x; wv[1] = x.y; wv[2] = x.z; wv[3] = x.w;
            wv[4] = y.x; wv[5] = y.y; wv[6] = y.z; wv[7] = y.w;
        } else {
#pragma unroll
            for (int i = 0; i < kEPL; ++i) wv[i] = 0;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kEPL; ++i) {
            sv[i] = ((live >> i) & 1u) ? P.src[e_lane + i] : 0u;
            wv[i] = 0;
            if constexpr (APP == kSSSP) wv[i] = i < nvalid ? P.w[e_lane + i] : 0u;
        }
    }
}

// Copies a block's staged frontier list to its reserved range (base == ~0:
// the block overflowed its stage; the iteration falls back to the bitmap).
__device__ __forceinline__ void publish_list(uint32_t* list, const uint32_t* s_list, unsigned n, unsigned base) {
    if (base == ~0u) return;
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) list[base + i] = s_list[i];
}

// Dense pull over all chunks with direct loads: warp gw of nw takes slices
// gw, gw + nw, ...  The next slice's edges and chunk metadata are loaded
// before the current slice is processed, so the stream overlaps the gathers.
template <int APP>
__device__ __forceinline__ void pull_dense_direct(const PullParams& P, unsigned it, const uint32_t* cur,
                                                  uint32_t* next, uint32_t* my_kid, typename Traits<APP>::T* my_val,
                                                  Stats& st, unsigned long long gw, unsigned long long nw,
                                                  unsigned* s_lcnt, uint32_t* s_list) {
    const unsigned lane = threadIdx.x & 31, q = lane >> 2, sub = lane & 3;
    const unsigned long long nslices = (P.NC + kSliceC - 1) / kSliceC;
    uint32_t sv[kEPL], wv[kEPL];
    uint2 meta = make_uint2(0u, 0u);
    unsigned next_head = 1u;
    int nvalid = 0;
    uint32_t live = 0;
    unsigned long long c = 0;
    auto fetch = [&](unsigned long long sl) {
        c = sl * kSliceC + q;
        const unsigned long long e_lane = c * 32 + 8 * sub;
        nvalid = 0;
        meta = make_uint2(0u, 0u);
        next_head = 1u;
        if (sl < nslices && c < P.NC) {
            const long long left = (long long)P.E - (long long)e_lane;
            nvalid = left >= kEPL ? kEPL : (left > 0 ? (int)left : 0);
            meta = __ldg(P.cmeta + c);
            next_head = __ldg(&P.cmeta[c + 1].x) & 1u;
        }
        live = lane_live<APP>(P, meta, 8 * sub, nvalid);
        load_lane_edges<APP>(P, e_lane, nvalid, live, sv, wv);
    };
    if (gw < nslices) fetch(gw);
    for (unsigned long long sl = gw; sl < nslices; sl += nw) {
        uint32_t cs[kEPL], cw[kEPL];
#pragma unroll
        for (int i = 0; i < kEPL; ++i) {
            cs[i] = sv[i];
            cw[i] = wv[i];
        }
        const uint2 cmeta = meta;
        const unsigned cnh = next_head;
        const int cnv = nvalid;
        const uint32_t clive = live;
        const unsigned long long cc = c;
        fetch(sl + nw);
        process_slice<APP>(P, it, cur, next, cs, cw, cnv, clive, cc, cmeta, cnh, 8 * sub, lane == 0, my_kid, my_val,
                           st, s_lcnt, s_list);
    }
}

// Pull over the Wedge Frontier list.  A list entry b at precision k covers
// 32 * 2^k edges: the 8-edge units b * 2^(k+2) .. (b+1) * 2^(k+2) - 1
// (k >= -2: k = -2, -1 are entries of 8 and 16 edges, the paper's finer
// precisions, Section 3.4 "Frontier Precision").  Slices of 32 listed units,
// one per lane, loaded directly; contiguous units continue each other's
// segments.  The Wedge bitmap words of the entries are zeroed as consumed.
template <int APP>
__device__ __forceinline__ void pull_sparse(const PullParams& P, unsigned it, int k, unsigned nentries,
                                            const uint32_t* cur, uint32_t* next, uint32_t* my_kid,
                                            typename Traits<APP>::T* my_val, Stats& st, unsigned long long gw,
                                            unsigned long long nw, unsigned* s_lcnt, uint32_t* s_list) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned ls = (unsigned)(k + 2);  // log2 of 8-edge units per entry
    const unsigned long long nunits = (unsigned long long)nentries << ls;
    const unsigned long long nslices = (nunits + 31) / 32;
    const unsigned long long umask = (1ull << ls) - 1;
    const unsigned long long NU = (P.E + kEPL - 1) / kEPL;
    // a small pull is bound by its chain of dependent loads: the visited
    // check would add one more link than the gathers it saves
    const bool skip_visited = (nunits >> 2) >= kSkipVisitedMinChunks;
    for (unsigned long long sl = gw; sl < nslices; sl += nw) {
        const unsigned long long j = sl * 32 + lane;
        bool uvalid = j < nunits;
        unsigned long long id = 0;  // the lane's 8-edge unit
        if (uvalid) {
            const uint32_t b = __ldcg(P.clist + (j >> ls));
            id = ((unsigned long long)b << ls) | (j & umask);
            uvalid = id < NU;
            if (uvalid && P.wb && (j & umask) == 0) P.wb[b >> 5] = 0u;
        }
        const unsigned long long idprev = __shfl_up_sync(kFull, id, 1);
        const unsigned pvalid = __shfl_up_sync(kFull, (unsigned)uvalid, 1);
        const bool contig = lane > 0 && pvalid && uvalid && id == idprev + 1;
        const unsigned long long c = id >> 2;
        const unsigned o = kEPL * (unsigned)(id & 3);
        const unsigned long long e_lane = c * 32 + o;
        int nvalid = 0;
        uint2 meta = make_uint2(0u, 0u);
        unsigned next_head = 1u;
        if (uvalid) {
            const long long left = (long long)P.E - (long long)e_lane;
            nvalid = left >= kEPL ? kEPL : (left > 0 ? (int)left : 0);
            meta = __ldg(P.cmeta + c);
            if (o == 32 - kEPL) next_head = __ldg(&P.cmeta[c + 1].x) & 1u;
        }
        const uint32_t live = lane_live<APP>(P, meta, o, nvalid, skip_visited);
        uint32_t sv[kEPL], wv[kEPL];
        load_lane_edges<APP>(P, e_lane, nvalid, live, sv, wv);
        process_slice<APP>(P, it, cur, next, sv, wv, nvalid, live, c, meta, next_head, o, !contig, my_kid, my_val,
                           st, s_lcnt, s_list);
    }
}

__device__ void decide_after_pull(const PullParams& P, unsigned it, unsigned nblocks, float* dsm);

// End of a pull (or push) block: the warps' frontier sums are added up, the
// block's sums go to its own slot and its staged frontier list to a range
// of the next list reserved with one atomic (none if the stage overflowed:
// the list then stays short of the frontier and the transformation scans
// the bitmap instead).  With DECIDE, the last block to finish (ticket) sums
// the slots and takes the decision for the next iteration.
template <bool DECIDE>
__device__ __forceinline__ void finish_block(const PullParams& P, unsigned it, Stats st, unsigned long long* s_F,
                                             unsigned* s_n, unsigned* s_row, unsigned* s_rmax, unsigned* s_lcnt,
                                             const uint32_t* s_list, float* dsm) {
    __shared__ unsigned s_lbase;
    if constexpr (DECIDE) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            st.F += __shfl_down_sync(kFull, st.F, d);
            st.n += __shfl_down_sync(kFull, st.n, d);
            st.row += __shfl_down_sync(kFull, st.row, d);
            st.rowmax = max(st.rowmax, __shfl_down_sync(kFull, st.rowmax, d));
        }
        if ((threadIdx.x & 31) == 0 && st.n) {
            atomicAdd(s_F, st.F);
            atomicAdd(s_n, st.n);
            atomicAdd(s_row, st.row);
            atomicMax(s_rmax, st.rowmax);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        BlockStat b;
        b.F = *s_F;
        b.n = *s_n;
        b.row = *s_row;
        b.lcnt = *s_lcnt;
        b.rowmax = *s_rmax;
        P.bstat[blockIdx.x] = b;
        s_lbase = (*s_lcnt && *s_lcnt <= (unsigned)kListCap) ? atomicAdd(&P.rec[it + 1].nlist, *s_lcnt) : ~0u;
    }
    __syncthreads();
    publish_list(P.flist[(it + 1) & 1], s_list, *s_lcnt, s_lbase);
    if constexpr (DECIDE) {
        if (P.decide) {
            __shared__ unsigned s_last;
            RunCtl* C = P.ctl;
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) s_last = atomicAdd(&C->ticket, 1u) == gridDim.x - 1;
            __syncthreads();
            if (s_last) {
                __threadfence();
                decide_after_pull(P, it, gridDim.x, dsm);
                if (threadIdx.x == 0) C->ticket = 0;
            }
        }
    }
}

template <int APP, bool TMA>
__global__ void __launch_bounds__(TMA ? kPullThreads : kCW * 32, TMA ? 1 : direct_min_blocks(APP))
    k_pull(const PullParams P) {
    using T = typename Traits<APP>::T;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned long long s_F;
    __shared__ unsigned s_n, s_row, s_rmax, s_lcnt;
    RunCtl* C = P.ctl;
    if (C->done) {
        // nothing left to pull: end the device loop (PageRank's pulls never
        // decide, and carry no conditional-node code, so that profilers see
        // them inside graphs)
        if constexpr (APP != kPR) {
            if (P.cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(P.cond, 0u);
        }
        return;
    }
    const unsigned it = C->it;
    const unsigned mode = P.rec[it].mode;
    if (P.hybrid && mode != 0) return;  // the push serves this iteration
    const int k = (int)P.rec[it].k;  // precision: -2 .. 7
    const unsigned nchunks = P.rec[it].nchunks;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // layout: [records: values, ids][stages: barriers, src, w, metadata]
    T* s_val = reinterpret_cast<T*>(smem);
    uint32_t* s_kid = reinterpret_cast<uint32_t*>(s_val + kCW * kRecCap);
    uint32_t* s_list = reinterpret_cast<uint32_t*>(smem + pull_records_bytes<APP>());
    unsigned char* stage = smem + pull_records_bytes<APP>() + pull_list_bytes<APP>();
    uint64_t* full = reinterpret_cast<uint64_t*>(stage);
    uint64_t* empty = full + kStages;
    uint32_t* s_src = reinterpret_cast<uint32_t*>(stage + 2 * kStages * 8);
    uint32_t* s_w = s_src + kStages * kTileE;
    uint2* s_meta = reinterpret_cast<uint2*>(s_w + (APP == kSSSP ? kStages * kTileE : 0));
    const unsigned wsel = warp < kCW ? warp : 0;
    uint32_t* my_kid = s_kid + wsel * kRecCap;
    T* my_val = s_val + wsel * kRecCap;
    constexpr bool tma = TMA;
    if (threadIdx.x == 0) {
        s_F = 0;
        s_n = 0;
        s_row = 0;
        s_rmax = 0;
        s_lcnt = 0;
        if (P.trace && blockIdx.x == 0) P.rec[it].t_pull0 = global_timer();
        if constexpr (APP == kPR) {
            if (blockIdx.x == 0) C->dangling[(P.pr_iter + 1) & 1] = 0ull;
        }
        if (mode == 0 && tma) {
            for (int s = 0; s < kStages; ++s) {
                mbar_init(full + s, 1);
                mbar_init(empty + s, kCW);
            }
            fence_mbar_init();
        }
    }
    __syncthreads();
    const uint32_t* cur = P.bm[it & 1];
    uint32_t* next = P.bm[(it + 1) & 1];
    Stats st{0ull, 0u, 0u, 0u};
    const unsigned q = lane >> 2;

    if constexpr (!TMA) {
        if (mode == 0)
            pull_dense_direct<APP>(P, it, cur, next, my_kid, my_val, st, (unsigned long long)blockIdx.x * kCW + warp,
                                   (unsigned long long)gridDim.x * kCW, &s_lcnt, s_list);
    }
    if (TMA && mode == 0) {
        // ---- dense, staged: tiles of kTileC chunks streamed by bulk copies ----
        const unsigned long long ntile = (P.NC + kTileC - 1) / kTileC;
        if (warp == kCW) {
            if (lane == 0) {
                unsigned kk = 0;
                for (unsigned long long t = blockIdx.x; t < ntile; t += gridDim.x, ++kk) {
                    const unsigned s = kk % kStages;
                    if (kk >= kStages && !mbar_wait(empty + s, ((kk / kStages) - 1) & 1u, &C->status)) break;
                    fence_proxy_async();
                    const unsigned long long c0 = t * kTileC, e0 = c0 * 32;
                    const unsigned long long rem = P.E - e0;
                    const uint32_t ne = rem < (unsigned long long)kTileE ? (uint32_t)rem : (uint32_t)kTileE;
                    const uint32_t nb = (ne * 4u) & ~15u;
                    const uint32_t mb = (kTileC + kMetaPad) * 8;
                    const uint32_t bytes = mb + nb * (APP == kSSSP ? 2u : 1u);
                    mbar_arrive_expect_tx(full + s, bytes);
                    bulk_load(s_meta + s * (kTileC + kMetaPad), P.cmeta + c0, mb, full + s);
                    if (nb) {
                        bulk_load(s_src + s * kTileE, P.src + e0, nb, full + s);
                        if constexpr (APP == kSSSP) bulk_load(s_w + s * kTileE, P.w + e0, nb, full + s);
                    }
                }
            }
            __syncwarp();
        } else {
            unsigned kk = 0;
            for (unsigned long long t = blockIdx.x; t < ntile; t += gridDim.x, ++kk) {
                const unsigned s = kk % kStages;
                if (!mbar_wait(full + s, (kk / kStages) & 1u, &C->status)) break;
                const unsigned long long c0 = t * kTileC, e0 = c0 * 32;
                const unsigned long long rem = P.E - e0;
                const uint32_t ne = rem < (unsigned long long)kTileE ? (uint32_t)rem : (uint32_t)kTileE;
                const uint32_t staged = ne & ~3u;  // edges delivered by the bulk copy
                const unsigned long long c = c0 + warp * kSliceC + q;
                const uint32_t local = warp * kSliceE + lane * kEPL;
                const long long left = (long long)ne - (long long)local;
                const int nvalid = left >= kEPL ? kEPL : (left > 0 ? (int)left : 0);
                uint32_t sv[kEPL], wv[kEPL];
                const uint32_t* ss = s_src + s * kTileE + local;
                const uint32_t* sw = s_w + s * kTileE + local;
                if (local + kEPL <= staged) {
                    const uint4 a = *reinterpret_cast<const uint4*>(ss);
                    const uint4 b = *reinterpret_cast<const uint4*>(ss + 4);
                    sv[0] = a.x; sv[1] = a.y; sv[2] = a.z; sv[3] = a.w;
                    sv[4] = b.x; sv[5] = b.y; sv[6] = b.z; sv[7] = b.w;
                    if constexpr (APP == kSSSP) {
                        const uint4 x = *reinterpret_cast<const uint4*>(sw);
                        const uint4 y = *reinterpret_cast<const uint4*>(sw + 4);
                        wv[0] = x.x; wv[1] = x.y; wv[2] = x.z; wv[3] = x.w;
                        wv[4] = y.x; wv[5] = y.y; wv[6] = y.z; wv[7] = y.w;
                    } else {
#pragma unroll
                        for (int i = 0; i < kEPL; ++i) wv[i] = 0;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < kEPL; ++i) {
                        sv[i] = 0;
                        wv[i] = 0;
                        if (i < nvalid) {
                            const uint32_t li = local + i;
                            sv[i] = li < staged ? ss[i] : P.src[e0 + li];
                            if constexpr (APP == kSSSP) wv[i] = li < staged ? sw[i] : P.w[e0 + li];
                        }
                    }
                }
                const uint2* sm = s_meta + s * (kTileC + kMetaPad) + warp * kSliceC + q;
                const uint2 meta = sm[0];
                const unsigned next_head = sm[1].x & 1u;
                // the stage is no longer read past this point
                __syncwarp();
                if (lane == 0) mbar_arrive(empty + s);
                const uint32_t live = lane_live<APP>(P, meta, 8 * (lane & 3), nvalid);
                process_slice<APP>(P, it, cur, next, sv, wv, nvalid, live, c, meta, next_head, 8 * (lane & 3), lane == 0,
                                   my_kid,
                                   my_val, st, &s_lcnt, s_list);
            }
        }
    }
    if (mode != 0 && warp < kCW)
        pull_sparse<APP>(P, it, k, nchunks, cur, next, my_kid, my_val, st, (unsigned long long)blockIdx.x * kCW + warp,
                         (unsigned long long)gridDim.x * kCW, &s_lcnt, s_list);

    finish_block<APP != kPR>(P, it, st, &s_F, &s_n, &s_row, &s_rmax, &s_lcnt, s_list,
                             reinterpret_cast<float*>(smem));
}

// Decision step (Section 3.4, Fig. 5), taken by the last pull block to
// finish (a block ticket): sums the pull blocks' slots into the record of
// the next iteration and takes the fullness decision (or the learned
// switch's).  Then the device loop's control: count this body execution and
// keep looping while the frontier is non-empty, never more than
// max_iters + 2 times.  `dsm` (the cost model's activations) lives in the
// block's record buffer, free once the block's own slices are done.
__device__ void decide_after_pull(const PullParams& P, unsigned it, unsigned nblocks, float* dsm) {
    __shared__ unsigned long long d_F;
    __shared__ unsigned d_n, d_row, d_rmax;
    IterRec* rec = P.rec;
    RunCtl* C = P.ctl;
    // the cost model's weights load while the slots are summed
    const bool stage = C->switch_mode == WEDGE_SWITCH_LEARNED && P.mlp != nullptr;
    if (stage) stage_model(P.mlp, dsm);
    if (threadIdx.x == 0) {
        d_F = 0;
        d_n = 0;
        d_row = 0;
        d_rmax = 0;
    }
    __syncthreads();
    // the slots were written by other blocks of this launch: read through L2
    unsigned long long F = 0;
    unsigned n = 0, row = 0, rmax = 0;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) {
        F += __ldcg(&P.bstat[b].F);
        n += __ldcg(&P.bstat[b].n);
        row += __ldcg(&P.bstat[b].row);
        rmax = max(rmax, __ldcg(&P.bstat[b].rowmax));
    }
    for (int d = 16; d > 0; d >>= 1) {
        F += __shfl_down_sync(kFull, F, d);
        n += __shfl_down_sync(kFull, n, d);
        row += __shfl_down_sync(kFull, row, d);
        rmax = max(rmax, __shfl_down_sync(kFull, rmax, d));
    }
    if ((threadIdx.x & 31) == 0 && n) {
        atomicAdd(&d_F, F);
        atomicAdd(&d_n, n);
        atomicAdd(&d_row, row);
        atomicMax(&d_rmax, rmax);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        IterRec* r = rec + it + 1;
        r->fullness = d_F;
        r->nfront = d_n;
        r->rowsum = d_row;
        r->rowmax = d_rmax;
        if (P.trace) rec[it].t_pull1 = global_timer();
    }
    __syncthreads();
    decide_block(rec, C, it + 1, P.mlp, P.gf, dsm, stage);
    if (threadIdx.x == 0) {
        const unsigned loops = ++C->loops;
        const bool more = !C->done && loops < C->max_iters + 2;
        if (P.cond) cudaGraphSetConditional(P.cond, more ? 1u : 0u);
    }
}

}  // namespace wedge

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
#include "tma.cuh"

namespace wedge {

constexpr unsigned kFull = 0xFFFFFFFFu;
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

struct XformParams {
    const uint32_t* eidx;
    const uint32_t* eidx_off;
    uint2* pieces;
    uint32_t* wb;
    uint32_t* clist;
    IterRec* rec;
    RunCtl* ctl;
    uint32_t* bm[2];             // run mode: frontier bitmaps by parity
    uint32_t* flist[2];          // run mode: frontier lists by parity
    const uint32_t* bm_in;       // standalone mode: the caller's frontier bitmap
    uint32_t V;
    unsigned long long bm_words;
    unsigned int* count_out;     // standalone mode: list count (else rec[it].nchunks)
    int standalone_k;            // >= 0: standalone transformation at this coarsening
    int trace;
    // load-balance accounting of a standalone transformation (nullptr: off):
    // per warp and kernel {start ns, end ns, busy SM cycles, SM id}
    unsigned long long* wstat;
    unsigned* slice_ctr;         // the paper's schedule: next frontier slice
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
    const bool learned = C->switch_mode == WEDGE_SWITCH_LEARNED && mlp_global != nullptr && nf > 0;
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
};

// A vertex activated for the next frontier: its out-degree (fullness), its
// edge-index row length (a feature of the learned switch) and the count.
__device__ __forceinline__ void count_active(const PullParams& P, uint32_t v, Stats& st) {
    st.F += __ldg(P.outdeg + v);
    st.n += 1;
    st.row += __ldg(P.eidx_off + v + 1) - __ldg(P.eidx_off + v);
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
// One warp slice of the pull (K1/K4 + K5): kSliceC chunks, kEPL = 8 edges
// per lane (lane L holds edges 8*(L&3) .. +7 of slice chunk L>>2).
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
                                              bool contig,
                                              uint32_t* s_kid, typename Traits<APP>::T* s_val, Stats& st,
                                              unsigned* s_lcnt, uint32_t* s_list) {
    using Tr = Traits<APP>;
    using T = typename Tr::T;
    const unsigned lane = threadIdx.x & 31, sub = lane & 3, o = 8 * sub;
    const uint32_t heads = meta.x;
    const uint32_t vmask = (nvalid >= 8) ? 0xFFu : ((1u << nvalid) - 1u);
    const uint32_t hb = (heads >> o) & vmask;
    const uint32_t brk = (hb | ((sub == 0 && !contig) ? 1u : 0u)) & vmask;
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
                           ((sub == 3) ? (next_head != 0) : (((heads >> (o + kEPL)) & 1u) != 0));
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
                    for (unsigned long long b = fresh; b; b &= b - 1)
                        P.levels[(size_t)dv * P.Q + (__ffsll((long long)b) - 1)] = it + 1;
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
        process_slice<APP>(P, it, cur, next, cs, cw, cnv, clive, cc, cmeta, cnh, q > 0, my_kid, my_val, st, s_lcnt,
                           s_list);
    }
}

// Pull over the Wedge Frontier list: slices of 8 listed chunks (list entry
// b at coarsening k stands for chunks b*2^k .. b*2^k + 2^k - 1), loaded
// directly; the Wedge bitmap words of the entries are zeroed as consumed.
template <int APP>
__device__ __forceinline__ void pull_sparse(const PullParams& P, unsigned it, unsigned k, unsigned nchunks,
                                            const uint32_t* cur, uint32_t* next, uint32_t* my_kid,
                                            typename Traits<APP>::T* my_val, Stats& st, unsigned long long gw,
                                            unsigned long long nw, unsigned* s_lcnt, uint32_t* s_list) {
    const unsigned lane = threadIdx.x & 31, q = lane >> 2, sub = lane & 3;
    const unsigned long long nunits = (unsigned long long)nchunks << k;
    const unsigned long long nslices = (nunits + kSliceC - 1) / kSliceC;
    const unsigned long long kmask = (1ull << k) - 1;
    // a small pull is bound by its chain of dependent loads: the visited
    // check would add one more link than the gathers it saves
    const bool skip_visited = nunits >= kSkipVisitedMinChunks;
    for (unsigned long long sl = gw; sl < nslices; sl += nw) {
        const unsigned long long j = sl * kSliceC + q;
        bool uvalid = j < nunits;
        unsigned long long c = 0;
        if (uvalid) {
            const uint32_t b = __ldcg(P.clist + (j >> k));
            c = ((unsigned long long)b << k) | (j & kmask);
            uvalid = c < P.NC;
            if (uvalid && P.wb && sub == 0 && (j & kmask) == 0) P.wb[b >> 5] = 0u;
        }
        const unsigned long long cprev = __shfl_up_sync(kFull, c, 4);
        const unsigned pvalid = __shfl_up_sync(kFull, (unsigned)uvalid, 4);
        const bool contig = q > 0 && pvalid && uvalid && c == cprev + 1;
        const unsigned long long e_lane = c * 32 + 8 * sub;
        int nvalid = 0;
        uint2 meta = make_uint2(0u, 0u);
        unsigned next_head = 1u;
        if (uvalid) {
            const long long left = (long long)P.E - (long long)e_lane;
            nvalid = left >= kEPL ? kEPL : (left > 0 ? (int)left : 0);
            meta = __ldg(P.cmeta + c);
            next_head = __ldg(&P.cmeta[c + 1].x) & 1u;
        }
        const uint32_t live = lane_live<APP>(P, meta, 8 * sub, nvalid, skip_visited);
        uint32_t sv[kEPL], wv[kEPL];
        load_lane_edges<APP>(P, e_lane, nvalid, live, sv, wv);
        process_slice<APP>(P, it, cur, next, sv, wv, nvalid, live, c, meta, next_head, contig, my_kid, my_val, st,
                           s_lcnt, s_list);
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
                                             unsigned* s_n, unsigned* s_row, unsigned* s_lcnt,
                                             const uint32_t* s_list, float* dsm) {
    __shared__ unsigned s_lbase;
    if constexpr (DECIDE) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            st.F += __shfl_down_sync(kFull, st.F, d);
            st.n += __shfl_down_sync(kFull, st.n, d);
            st.row += __shfl_down_sync(kFull, st.row, d);
        }
        if ((threadIdx.x & 31) == 0 && st.n) {
            atomicAdd(s_F, st.F);
            atomicAdd(s_n, st.n);
            atomicAdd(s_row, st.row);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        BlockStat b;
        b.F = *s_F;
        b.n = *s_n;
        b.row = *s_row;
        b.lcnt = *s_lcnt;
        b.pad_ = 0;
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
    __shared__ unsigned s_n, s_row, s_lcnt;
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
    const unsigned k = P.rec[it].k;
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
    Stats st{0ull, 0u, 0u};
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
                process_slice<APP>(P, it, cur, next, sv, wv, nvalid, live, c, meta, next_head, q > 0, my_kid,
                                   my_val, st, &s_lcnt, s_list);
            }
        }
    }
    if (mode != 0 && warp < kCW)
        pull_sparse<APP>(P, it, k, nchunks, cur, next, my_kid, my_val, st, (unsigned long long)blockIdx.x * kCW + warp,
                         (unsigned long long)gridDim.x * kCW, &s_lcnt, s_list);

    finish_block<APP != kPR>(P, it, st, &s_F, &s_n, &s_row, &s_lcnt, s_list, reinterpret_cast<float*>(smem));
}

// ------------------------------------------------------------------------
// Transformation (K2), two kernels.
//   A (k_xform_scan): walk the vertex frontier bitmap; every active vertex's
//     edge-index row is cut into pieces of at most 32 entries; one
//     reservation per warp.  In run mode it also clears the bitmap the next
//     pull fills and the record that pull accumulates into.
//   B (k_xform_expand): expand the pieces with the warp's lanes balanced over
//     up to 32 pieces at a time, set the Wedge Frontier bits (bit b = list
//     entry b at coarsening k) and append every newly set bit to the list:
//     the bitmap removes duplicates (Section 4).
// ------------------------------------------------------------------------
// The warp's rows (lane L: row start rb, length rl, np pieces, exclusive
// piece offset excl among the warp's pieces) written as pieces of at most 32
// entries to pieces[slot0 ...] by all 32 lanes: piece i goes to the lane
// whose range holds it (binary search over the lanes' offsets), so one long
// row (a hub's) is written by the whole warp.
__device__ __forceinline__ void write_pieces(uint2* pieces, unsigned slot0, unsigned total, uint32_t rb, uint32_t rl,
                                             unsigned excl) {
    const unsigned lane = threadIdx.x & 31;
    for (unsigned i0 = 0; i0 < total; i0 += 32) {
        const unsigned i = i0 + lane;
        unsigned jx = 0;
#pragma unroll
        for (unsigned stp = 16; stp >= 1; stp >>= 1) {
            const unsigned ex = __shfl_sync(kFull, excl, jx + stp);
            if (ex <= i) jx += stp;
        }
        const uint32_t b = __shfl_sync(kFull, rb, jx);
        const uint32_t l = __shfl_sync(kFull, rl, jx);
        const unsigned q = (i - __shfl_sync(kFull, excl, jx)) * 32u;
        if (i < total) pieces[slot0 + i] = make_uint2(b + q, min(32u, l - q));
    }
}

// Warp-level scan of bitmap words [gw*32, ...) step nw*32: pieces of the
// active vertices' edge-index rows, one reservation per warp on *npieces.
__device__ __forceinline__ void xform_scan_words(const uint32_t* bm, uint32_t V, unsigned long long words,
                                                 const uint32_t* __restrict__ eidx_off, uint2* pieces,
                                                 unsigned* npieces, unsigned long long gw, unsigned long long nw) {
    const unsigned lane = threadIdx.x & 31;
    for (unsigned long long base = gw * 32; base < words; base += nw * 32) {
        const unsigned long long wi = base + lane;
        uint32_t word = wi < words ? __ldcg(bm + wi) : 0u;
        if (wi == words - 1 && (V & 31)) word &= (1u << (V & 31)) - 1u;
        unsigned np = 0;
        for (uint32_t w = word; w; w &= w - 1) {
            const uint32_t u = (uint32_t)(wi * 32 + __ffs(w) - 1);
            np += (__ldg(eidx_off + u + 1) - __ldg(eidx_off + u) + 31u) >> 5;
        }
        unsigned incl = np;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, d);
            if (lane >= (unsigned)d) incl += y;
        }
        const unsigned total = __shfl_sync(kFull, incl, 31);
        if (!total) continue;
        unsigned slot = 0;
        if (lane == 31) slot = atomicAdd(npieces, total);
        slot = __shfl_sync(kFull, slot, 31);
        // one vertex per lane and round: every round's rows go out together
        unsigned rem = word, done = 0;
        while (__any_sync(kFull, rem != 0)) {
            uint32_t rb = 0, rl = 0;
            if (rem) {
                const uint32_t u = (uint32_t)(wi * 32 + __ffs(rem) - 1);
                rem &= rem - 1;
                rb = __ldg(eidx_off + u);
                rl = __ldg(eidx_off + u + 1) - rb;
            }
            const unsigned p = (rl + 31u) >> 5;
            unsigned pi = p;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned y = __shfl_up_sync(kFull, pi, d);
                if (lane >= (unsigned)d) pi += y;
            }
            const unsigned rt = __shfl_sync(kFull, pi, 31);
            write_pieces(pieces, slot + done, rt, rb, rl, pi - p);
            done += rt;
        }
    }
}

// Same as xform_scan_words over an explicit list of n frontier vertices.
__device__ __forceinline__ void xform_scan_list(const uint32_t* list, unsigned n,
                                                const uint32_t* __restrict__ eidx_off, uint2* pieces,
                                                unsigned* npieces, unsigned long long gw, unsigned long long nw) {
    const unsigned lane = threadIdx.x & 31;
    for (unsigned long long base = gw * 32; base < n; base += nw * 32) {
        const unsigned long long i = base + lane;
        uint32_t rb = 0, rl = 0;
        if (i < n) {
            const uint32_t u = __ldcg(list + i);
            rb = __ldg(eidx_off + u);
            rl = __ldg(eidx_off + u + 1) - rb;
        }
        const unsigned np = (rl + 31u) >> 5;
        unsigned incl = np;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, d);
            if (lane >= (unsigned)d) incl += y;
        }
        const unsigned total = __shfl_sync(kFull, incl, 31);
        if (!total) continue;
        unsigned slot = 0;
        if (lane == 31) slot = atomicAdd(npieces, total);
        slot = __shfl_sync(kFull, slot, 31);
        write_pieces(pieces, slot, total, rb, rl, incl - np);
    }
}

// Zeroes the bitmap words of a frontier: by its list when complete,
// otherwise every word.  Optionally zeroes the vertices' query masks too.
__device__ __forceinline__ void clear_frontier(uint32_t* bm, unsigned long long words, const uint32_t* list,
                                               bool complete, unsigned n, unsigned long long* masks,
                                               unsigned long long tid, unsigned long long nth) {
    if (complete) {
        for (unsigned long long i = tid; i < n; i += nth) {
            const uint32_t v = __ldcg(list + i);
            bm[v >> 5] = 0u;
            if (masks) masks[v] = 0ull;
        }
    } else if (masks) {
        for (unsigned long long wi = tid; wi < words; wi += nth) {
            uint32_t w = __ldcg(bm + wi);
            if (!w) continue;
            bm[wi] = 0u;
            for (; w; w &= w - 1) masks[wi * 32 + __ffs(w) - 1] = 0ull;
        }
    } else {
        for (unsigned long long wi = tid; wi < words; wi += nth) bm[wi] = 0u;
    }
}

// Warp-level expansion of n pieces: Wedge bitmap bits (entry = chunk >> k),
// fresh bits appended to list with a warp-aggregated reservation on *count.
// A warp task is up to 32 pieces, fewer when there are too few pieces to
// give every warp a task (one hub's row): a task's entries are walked 32 at
// a time, so its length is the latency that matters.
// Fresh list entries staged by a warp are appended with one reservation on
// the list's counter per kAppendStage entries (appending every round put up
// to one atomic per 32 entries on that single address).
constexpr unsigned kAppendStage = 256;

__device__ __forceinline__ void flush_staged(uint32_t* list, unsigned* count, const uint32_t* stage, unsigned n) {
    const unsigned lane = threadIdx.x & 31;
    __syncwarp();
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(count, n);
    base = __shfl_sync(kFull, base, 0);
    for (unsigned i = lane; i < n; i += 32) list[base + i] = stage[i];
    __syncwarp();
}

__device__ __forceinline__ void xform_expand_pieces(const uint2* pieces, unsigned n, unsigned k,
                                                    const uint32_t* __restrict__ eidx, uint32_t* wb, uint32_t* list,
                                                    unsigned* count, unsigned long long gw, unsigned long long nw,
                                                    uint32_t* stage = nullptr) {
    unsigned staged = 0;  // warp-uniform
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const unsigned long long per = (unsigned long long)n / nw;
    const unsigned ppt = per >= 32 ? 32u : (per < 1 ? 1u : (unsigned)per);
    for (unsigned long long base = gw * ppt; base < n; base += nw * ppt) {
        const unsigned long long idx = base + lane;
        const uint2 pc = (lane < ppt && idx < n) ? __ldcg(pieces + idx) : make_uint2(0u, 0u);
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
            const bool act = e < total;
            unsigned jx = 0;
#pragma unroll
            for (unsigned stp = 16; stp >= 1; stp >>= 1) {
                const unsigned cj = jx + stp;
                const unsigned ex = __shfl_sync(kFull, excl, cj);
                if (ex <= e) jx = cj;
            }
            const unsigned st = __shfl_sync(kFull, pc.x, jx);
            const unsigned ex = __shfl_sync(kFull, excl, jx);
            // Lanes are runs of consecutive rows' entries, so neighbouring
            // lanes often hit the same bitmap word (always for a hub's row
            // at coarse precision).  Each run of lanes on one word sets its
            // bits with one atomicOr by the run's last lane; within the
            // run, the first lane holding an entry owns it, and it is fresh
            // if the word did not have its bit before.
            const uint32_t b = act ? __ldg(eidx + st + (e - ex)) >> k : 0xFFFFFFFFu;
            const uint32_t word = b >> 5;
            const uint32_t bit = act ? 1u << (b & 31) : 0u;
            const uint32_t wprev = __shfl_up_sync(kFull, word, 1);
            const unsigned starts = __ballot_sync(kFull, lane == 0 || word != wprev);
            const unsigned rs = 31 - __clz(starts & (lt_mask | (1u << lane)));      // run start
            const unsigned above = starts & ~(lt_mask | (1u << lane));
            const unsigned re = above ? (unsigned)__ffs(above) - 2 : 31u;           // run end
            uint32_t bits = bit;
#pragma unroll
            for (unsigned d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, bits, d);
                if (lane >= rs + d) bits |= y;
            }
            uint32_t old = 0;
            if (lane == re && act) old = atomicOr(wb + word, bits);
            old = __shfl_sync(kFull, old, re);
            const unsigned run = (re == 31 ? kFull : ((2u << re) - 1u)) & ~((1u << rs) - 1u);
            const unsigned same = __match_any_sync(kFull, b) & run;
            const bool fresh = act && (unsigned)(__ffs(same) - 1) == lane && !(old & bit);
            const unsigned m = __ballot_sync(kFull, fresh);
            if (m && stage) {
                const unsigned nm = __popc(m);
                if (staged + nm > kAppendStage) {
                    flush_staged(list, count, stage, staged);
                    staged = 0;
                }
                if (fresh) stage[staged + __popc(m & lt_mask)] = b;
                staged += nm;
            } else if (m) {
                const unsigned leader = __ffs(m) - 1;
                unsigned slot = 0;
                if (lane == leader) slot = atomicAdd(count, (unsigned)__popc(m));
                slot = __shfl_sync(kFull, slot, leader);
                if (fresh) list[slot + __popc(m & lt_mask)] = b;
            }
        }
    }
    if (stage && staged) flush_staged(list, count, stage, staged);
}

// Before iteration `it` fills the next frontier: the bitmap it fills held
// F_{it-1}, so clear it (by its list when that list is complete), and zero
// the record the iteration accumulates into.  Idempotent until then.
__device__ __forceinline__ void prepare_iteration(const XformParams& X, unsigned it, unsigned long long tid,
                                                  unsigned long long nth) {
    if (it > 0) {
        const IterRec& pr = X.rec[it - 1];
        uint32_t* clr = ((it + 1) & 1) ? X.bm[1] : X.bm[0];
        clear_frontier(clr, X.bm_words, ((it + 1) & 1) ? X.flist[1] : X.flist[0], pr.nlist == pr.nfront, pr.nfront,
                       nullptr, tid, nth);
    }
    if (blockIdx.x == 0 && threadIdx.x < sizeof(IterRec) / 4)
        reinterpret_cast<unsigned*>(X.rec + it + 1)[threadIdx.x] = 0u;
}

// Load-balance accounting (standalone transformations only): warp `gw`'s
// record {start ns, end ns, busy cycles, SM} in slot `kernel` (0: scan or
// the paper's schedule, 1: expansion).
struct WarpStamp {
    unsigned long long t0 = 0, c0 = 0;
    __device__ __forceinline__ void start(const XformParams& X) {
        if (X.wstat) {
            t0 = global_timer();
            c0 = clock64();
        }
    }
    __device__ __forceinline__ void stop(const XformParams& X, unsigned long long gw, int kernel) {
        if (!X.wstat) return;
        __syncwarp();
        if ((threadIdx.x & 31) == 0) {
            unsigned smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            unsigned long long* w = X.wstat + gw * 8 + kernel * 4;
            w[0] = t0;
            w[1] = global_timer();
            w[2] = clock64() - c0;
            w[3] = smid;
        }
    }
};

__global__ void __launch_bounds__(kXformThreads) k_xform_scan(const XformParams X) {
    RunCtl* C = X.ctl;
    const uint32_t* bm;
    IterRec* r;
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
    WarpStamp ws;
    ws.start(X);
    if (X.standalone_k >= 0) {
        bm = X.bm_in;
        r = X.rec;
        xform_scan_words(bm, X.V, X.bm_words, X.eidx_off, X.pieces, &r->npieces, tid >> 5, nth >> 5);
        ws.stop(X, tid >> 5, 0);
        return;
    } else {
        if (C->done) return;
        const unsigned it = C->it;
        if (X.trace && blockIdx.x == 0 && threadIdx.x == 0) X.rec[it].t_xf0 = global_timer();
        prepare_iteration(X, it, tid, nth);
        r = X.rec + it;
        if (r->mode == 0) return;
        if (r->nlist == r->nfront) {
            xform_scan_list((it & 1) ? X.flist[1] : X.flist[0], r->nfront, X.eidx_off, X.pieces, &r->npieces,
                            tid >> 5, nth >> 5);
            return;
        }
        bm = (it & 1) ? X.bm[1] : X.bm[0];
    }
    xform_scan_words(bm, X.V, X.bm_words, X.eidx_off, X.pieces, &r->npieces, tid >> 5, nth >> 5);
}

__global__ void __launch_bounds__(kXformThreads) k_xform_expand(const XformParams X) {
    RunCtl* C = X.ctl;
    unsigned n, k;
    unsigned* count;
    unsigned it = 0;
    if (X.standalone_k >= 0) {
        n = __ldcg(&X.rec[0].npieces);
        k = (unsigned)X.standalone_k;
        count = X.count_out;
    } else {
        if (C->done) return;
        it = C->it;
        const IterRec* r = X.rec + it;
        if (r->mode == 0) return;
        n = r->npieces;
        k = r->k;
        count = &X.rec[it].nchunks;
    }
    __shared__ uint32_t s_stage[kXformThreads / 32][kAppendStage];
    const unsigned long long gw = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    WarpStamp ws;
    ws.start(X);
    xform_expand_pieces(X.pieces, n, k, X.eidx, X.wb, X.clist, count, gw, nw, s_stage[threadIdx.x >> 5]);
    if (X.standalone_k >= 0) ws.stop(X, gw, 1);
    if (X.trace && X.standalone_k < 0) {
        __syncthreads();
        if (threadIdx.x == 0) atomicMax(&X.rec[it].t_xf1, global_timer());
    }
}

// The transformation as the paper's implementation schedules it (Section 4,
// "Parallelization"), for the load-balance study of Section 5.3 (Fig. 13):
// the vertex frontier is sliced into equal pieces of kStaticSliceWords
// bitmap words, each taken by the next free warp, which walks the whole
// edge-index row of every active vertex in its piece, 32 entries at a time
// (neither the pieces' bit counts nor the rows' lengths are considered).
// Every Wedge bitmap bit is set with an atomicOr; the one that finds it
// clear appends its entry to the list.  Standalone transformations only.
constexpr unsigned kStaticSliceWords = 8;  // 256 vertices per piece

__global__ void __launch_bounds__(kXformThreads) k_xform_static(const XformParams X) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long gw = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned k = (unsigned)X.standalone_k;
    const unsigned long long nslices = (X.bm_words + kStaticSliceWords - 1) / kStaticSliceWords;
    WarpStamp ws;
    ws.start(X);
    for (;;) {
        unsigned long long sl = 0;
        if (lane == 0) sl = atomicAdd(X.slice_ctr, 1u);
        sl = __shfl_sync(kFull, sl, 0);
        if (sl >= nslices) break;
        for (unsigned long long wi = sl * kStaticSliceWords; wi < (sl + 1) * kStaticSliceWords && wi < X.bm_words;
             ++wi) {
            uint32_t word = __ldg(X.bm_in + wi);
            if (wi == X.bm_words - 1 && (X.V & 31)) word &= (1u << (X.V & 31)) - 1u;
            for (; word; word &= word - 1) {
                const uint32_t u = (uint32_t)(wi * 32 + __ffs(word) - 1);
                const uint32_t rb = __ldg(X.eidx_off + u), re = __ldg(X.eidx_off + u + 1);
                for (uint32_t e0 = rb; e0 < re; e0 += 32) {
                    const uint32_t e = e0 + lane;
                    bool fresh = false;
                    uint32_t b = 0;
                    if (e < re) {
                        b = __ldg(X.eidx + e) >> k;
                        const uint32_t bit = 1u << (b & 31);
                        fresh = (atomicOr(X.wb + (b >> 5), bit) & bit) == 0;
                    }
                    const unsigned m = __ballot_sync(kFull, fresh);
                    if (m) {
                        const unsigned leader = __ffs(m) - 1;
                        unsigned slot = 0;
                        if (lane == leader) slot = atomicAdd(X.count_out, (unsigned)__popc(m));
                        slot = __shfl_sync(kFull, slot, leader);
                        if (fresh) X.clist[slot + __popc(m & ((1u << lane) - 1u))] = b;
                    }
                }
            }
        }
    }
    ws.stop(X, gw, 0);
}

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
    __shared__ unsigned s_n, s_row, s_lcnt;
    RunCtl* C = P.ctl;
    if (C->done) return;
    const unsigned it = C->it;
    if (P.rec[it].mode == 0) return;  // a dense iteration: the pull serves it
    const unsigned n = P.rec[it].npieces;
    if (threadIdx.x == 0) {
        s_F = 0;
        s_n = 0;
        s_row = 0;
        s_lcnt = 0;
        if (P.trace && blockIdx.x == 0) P.rec[it].t_pull0 = global_timer();
    }
    __syncthreads();
    uint32_t* next = P.bm[(it + 1) & 1];
    Stats st{0ull, 0u, 0u};
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
    finish_block<true>(P, it, st, &s_F, &s_n, &s_row, &s_lcnt, s_list, reinterpret_cast<float*>(s_list));
}

// Initial frontier: size, fullness and edge-index work (the transformation
// derives its pieces from the bitmap), then the decision for pull 0.
__global__ void k_frontier_stats(const uint32_t* __restrict__ bm, uint32_t V, const uint32_t* __restrict__ outdeg,
                                 const uint32_t* __restrict__ eidx_off, IterRec* rec, RunCtl* C,
                                 const __nv_bfloat16* mlp, GraphFeat gf) {
    __shared__ __align__(16) unsigned char dsm_bytes[kDecideSmemBytes];
    float* dsm = reinterpret_cast<float*>(dsm_bytes);
    __shared__ unsigned long long s_F;
    __shared__ unsigned s_n, s_row, s_last;
    if (threadIdx.x == 0) {
        s_F = 0;
        s_n = 0;
        s_row = 0;
    }
    __syncthreads();
    unsigned long long F = 0;
    unsigned n = 0, row = 0;
    const unsigned long long words = ((unsigned long long)V + 31) / 32;
    for (unsigned long long wi = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; wi < words;
         wi += (unsigned long long)gridDim.x * blockDim.x) {
        uint32_t word = bm[wi];
        if (wi == words - 1 && (V & 31)) word &= (1u << (V & 31)) - 1u;
        for (; word; word &= word - 1) {
            const uint32_t u = (uint32_t)(wi * 32 + __ffs(word) - 1);
            F += outdeg[u];
            n += 1;
            row += eidx_off[u + 1] - eidx_off[u];
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        F += __shfl_down_sync(kFull, F, d);
        n += __shfl_down_sync(kFull, n, d);
        row += __shfl_down_sync(kFull, row, d);
    }
    if ((threadIdx.x & 31) == 0 && n) {
        atomicAdd(&s_F, F);
        atomicAdd(&s_n, n);
        atomicAdd(&s_row, row);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_n) {
            atomicAdd(&rec->fullness, s_F);
            atomicAdd(&rec->nfront, s_n);
            atomicAdd(&rec->rowsum, s_row);
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

// Decision step (Section 3.4, Fig. 5), taken by the last pull block to
// finish (a block ticket): sums the pull blocks' slots into the record of
// the next iteration and takes the fullness decision (or the learned
// switch's).  Then the device loop's control: count this body execution and
// keep looping while the frontier is non-empty, never more than
// max_iters + 2 times.  `dsm` (the cost model's activations) lives in the
// block's record buffer, free once the block's own slices are done.
__device__ void decide_after_pull(const PullParams& P, unsigned it, unsigned nblocks, float* dsm) {
    __shared__ unsigned long long d_F;
    __shared__ unsigned d_n, d_row;
    IterRec* rec = P.rec;
    RunCtl* C = P.ctl;
    // the cost model's weights load while the slots are summed
    const bool stage = C->switch_mode == WEDGE_SWITCH_LEARNED && P.mlp != nullptr;
    if (stage) stage_model(P.mlp, dsm);
    if (threadIdx.x == 0) {
        d_F = 0;
        d_n = 0;
        d_row = 0;
    }
    __syncthreads();
    // the slots were written by other blocks of this launch: read through L2
    unsigned long long F = 0;
    unsigned n = 0, row = 0;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) {
        F += __ldcg(&P.bstat[b].F);
        n += __ldcg(&P.bstat[b].n);
        row += __ldcg(&P.bstat[b].row);
    }
    for (int d = 16; d > 0; d >>= 1) {
        F += __shfl_down_sync(kFull, F, d);
        n += __shfl_down_sync(kFull, n, d);
        row += __shfl_down_sync(kFull, row, d);
    }
    if ((threadIdx.x & 31) == 0 && n) {
        atomicAdd(&d_F, F);
        atomicAdd(&d_n, n);
        atomicAdd(&d_row, row);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        IterRec* r = rec + it + 1;
        r->fullness = d_F;
        r->nfront = d_n;
        r->rowsum = d_row;
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
                              uint32_t* bm0) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nroots; i += gridDim.x * blockDim.x) {
        const uint32_t v = roots[i], q = rq[i];
        const unsigned long long bit = 1ull << q;
        atomicOr(fb0 + v, bit);
        atomicOr(seen + v, bit);
        levels[(size_t)v * Q + q] = 0u;
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
__global__ void __launch_bounds__(kCW * 32) k_msbfs(const PullParams P, const XformParams X, unsigned* bar) {
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
        Stats st{0ull, 0u, 0u};
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
        const bool done = nf == 0 || nit >= C->max_iters;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            P.rec[nit].mode = sparse;
            P.rec[nit].k = C->k;
            C->it = nit;
            if (done) {
                C->done = 1;
                if (nf) C->status |= kStatusMaxIters;
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
                xform_scan_list((nit & 1) ? P.flist[1] : P.flist[0], nf, X.eidx_off, X.pieces, &P.rec[nit].npieces,
                                gw, nw);
            else
                xform_scan_words(next, X.V, words, X.eidx_off, X.pieces, &P.rec[nit].npieces, gw, nw);
        }
        if (!grid_sync(bar, &C->status)) break;
        if (sparse)
            xform_expand_pieces(X.pieces, __ldcg(&P.rec[nit].npieces), C->k, X.eidx, X.wb, X.clist,
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

__global__ void k_pr_init(uint32_t V, const uint32_t* __restrict__ outdeg, float* __restrict__ contrib,
                          unsigned long long* __restrict__ acc, RunCtl* C) {
    const float pr0 = 1.0f / (float)V;
    unsigned long long dang = 0;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t od = outdeg[v];
        contrib[v] = od ? pr0 / (float)od : 0.0f;
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
                           unsigned long long* __restrict__ acc, float* __restrict__ contrib,
                           float* __restrict__ out, RunCtl* C, unsigned t, int last, float base, float d) {
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
        if (last) reinterpret_cast<float4*>(out)[q] = o;
        else reinterpret_cast<float4*>(contrib)[q] = c;
    }
    // the tail of V mod 4 vertices
    for (unsigned long long v = 4 * nq + blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V; v += stride) {
        const unsigned long long a = acc[v];
        if ((__ldg(split_bm + (v >> 5)) >> (v & 31)) & 1u) acc[v] = 0ull;
        float o = 0.f, c = 0.f;
        pr_vertex(a, last ? 0u : outdeg[v], dv, base, d, last, o, c, dang);
        if (last) out[v] = o;
        else contrib[v] = c;
    }
    if (!last) block_add_u64(dang, &C->dangling[(t + 1) & 1]);
}

__global__ void k_ctl_init(RunCtl* C, RunCtl init) {
    if (threadIdx.x == 0) *C = init;
}

__global__ void k_clear_listed(const uint32_t* __restrict__ list, const uint32_t* __restrict__ count,
                               uint32_t* __restrict__ wb) {
    const unsigned n = *count;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        wb[list[i] >> 5] = 0u;
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
    WEDGE_TRY(dev_alloc(g, (void**)&g->wb, ((NC + 31) / 32 + 1) * 4));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->wb, 0, ((NC + 31) / 32 + 1) * 4, s));
    WEDGE_TRY(dev_alloc(g, (void**)&g->clist, (NC + 1) * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->pieces, (g->npieces_max + 1) * sizeof(uint2)));
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
    X.standalone_k = -1;
    X.trace = trace;
    X.wstat = nullptr;
    X.slice_ctr = nullptr;
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
        launch_xform(g, xform_params(g, 0), cs);
    }, &g->loop_exec[app]);
}

static wedge_status check_opts(const wedge_opts* o) {
    if (o->log2_coarsen > kMaxCoarsen) return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be <= 7");
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
            const uint64_t e = (uint64_t)r[t].nchunks << (5 + r[t].k);
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
    const uint64_t wb_words = (g->NC + 31) / 32 + 1;
    const bool sync = o.synchronous && app != kBFS;
    const bool push = o.sparse_push != 0;
    if (push && o.synchronous) return set_error(WEDGE_ERR_INVALID_ARG, "sparse_push and synchronous exclude each other");
    if (push && init.switch_mode == WEDGE_SWITCH_LEARNED) init.switch_mode = WEDGE_SWITCH_THRESHOLD;
    if (sync && !g->vals_sync) WEDGE_TRY(dev_alloc(g, (void**)&g->vals_sync, (uint64_t)g->V * 4));
    if (push) WEDGE_TRY(build_csr(g, s));
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
    const uint32_t* result = g->vals;
    if (push) {
        X.eidx_off = g->csr_off;
        X.pieces = g->push_pieces;
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
static wedge_status msbfs_enqueue(wedge_graph* g, uint32_t nroots, uint32_t Q, uint32_t* levels, const RunCtl& init,
                                  bool sssp, cudaStream_t s) {
    WEDGE_TRY_CUDA(cudaMemsetAsync(levels, 0xFF, (size_t)g->V * Q * 4, s));
    k_msbfs_clear<<<g->num_sms * 4, 256, 0, s>>>(g->V, g->ms_fb[0], g->ms_fb[1], g->ms_seen, g->bm[0], g->bm[1], g->wb,
                                                 (g->NC + 31) / 32 + 1, g->rec, g->ctl, init, g->ms_bar);
    k_msbfs_roots<<<(nroots + 255) / 256, 256, 0, s>>>(g->ms_roots, g->ms_roots + g->ms_cap, nroots, Q, g->ms_fb[0],
                                                       g->ms_seen, levels, g->bm[0]);
    PullParams P = pull_params(g, 0, kBFS);
    P.mlp = nullptr;
    P.visk = nullptr;  // per-query visits live in the seen masks
    P.decide = 0;      // the persistent launch takes its own decisions
    P.fb[0] = g->ms_fb[0];
    P.fb[1] = g->ms_fb[1];
    P.seen = g->ms_seen;
    P.levels = levels;
    P.Q = Q;
    XformParams X = xform_params(g, 0);
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
    const float base = (1.0f - damping) / (float)g->V;
    for (uint32_t t = 0; t < iters; ++t) {
        P.pr_iter = t;
        launch_pull_app(g, kPR, P, s);
        const int last = (t + 1 == iters);
        k_pr_apply<<<vb, 256, 0, s>>>(g->V, g->outdeg, g->split_bm, g->acc, g->contrib, g->rank, g->ctl, t, last, base,
                                      damping);
        count_launch();
    }
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
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev0, s));
    RunCtl init{};
    init.max_iters = 0xFFFFFFFFu;
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->rec, 0, 2 * sizeof(IterRec), s));
    k_ctl_init<<<1, 32, 0, s>>>(g->ctl, init);
    k_pr_init<<<g->num_sms * 8, 256, 0, s>>>(V, g->outdeg, g->contrib, g->acc, g->ctl);
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
    if (!g || !d_contrib || !d_sums) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    // a dense pull at iteration 0; the caller's zeros take the place of the
    // vertex step that clears split destinations between iterations
    k_standalone_prep<<<1, 32, 0, s>>>(g->rec, g->ctl, 0, 0, 0, nullptr, 0);
    PullParams P = pull_params(g, 0, kPR);
    P.contrib = d_contrib;
    P.acc = reinterpret_cast<unsigned long long*>(d_sums);
    P.pr_iter = 0;
    launch_pull_app(g, kPR, P, s);
    count_launch();
    WEDGE_TRY_CUDA(cudaGetLastError());
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
                              uint32_t nroots, uint32_t nqueries, uint32_t* d_levels, const wedge_opts* opts_in,
                              wedge_stats* stats, cudaStream_t s) {
    if (!g || !roots || !d_levels) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (sssp && !g->w && g->E) return set_error(WEDGE_ERR_INVALID_ARG, "SSSP needs edge weights");
    if (nqueries < 1 || nqueries > 64) return set_error(WEDGE_ERR_INVALID_ARG, "nqueries must be 1..64");
    if (nroots < 1 || nroots > (1u << 24)) return set_error(WEDGE_ERR_INVALID_ARG, "nroots must be 1..2^24");
    wedge_opts o;
    if (opts_in) o = *opts_in;
    else wedge_default_opts(sssp ? WEDGE_SSSP : WEDGE_BFS, &o);
    WEDGE_TRY(check_opts(&o));
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
    const uint32_t key[5] = {init.tau_bp, init.k, init.switch_mode, init.max_iters, sssp ? 1u : 0u};
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
        if (e == cudaSuccess) es = msbfs_enqueue(g, nroots, nqueries, d_levels, init, sssp, g->cap_stream);
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
        WEDGE_TRY(msbfs_enqueue(g, nroots, nqueries, d_levels, init, sssp, s));
    }
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev1, s));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost, s));
    g->last_stream = s;
    g->last_trace = false;
    g->last_push = false;
    if (!stats) return WEDGE_OK;
    return fill_stats(g, s, stats);
}
}  // namespace wedge

extern "C" {

wedge_status wedge_run_bfs_batch(wedge_graph_t g, const uint32_t* roots, const uint32_t* root_query, uint32_t nroots,
                                 uint32_t nqueries, uint32_t* d_levels, const wedge_opts* opts, wedge_stats* stats,
                                 wedge_stream_t stream) {
    return run_batch(g, false, roots, root_query, nroots, nqueries, d_levels, opts, stats, (cudaStream_t)stream);
}

wedge_status wedge_run_sssp_batch(wedge_graph_t g, const uint32_t* roots, const uint32_t* root_query,
                                  uint32_t nroots, uint32_t nqueries, uint32_t* d_dist, const wedge_opts* opts,
                                  wedge_stats* stats, wedge_stream_t stream) {
    return run_batch(g, true, roots, root_query, nroots, nqueries, d_dist, opts, stats, (cudaStream_t)stream);
}

wedge_status wedge_frontier_transform(wedge_graph_t g, const uint32_t* d_vertex_bitmap, uint32_t log2_coarsen,
                                      uint32_t* d_chunk_list, uint32_t* d_chunk_count, wedge_stream_t stream) {
    if (!g || !d_vertex_bitmap || !d_chunk_list || !d_chunk_count)
        return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (log2_coarsen > kMaxCoarsen) return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be <= 7");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->rec, 0, sizeof(IterRec), s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(d_chunk_count, 0, 4, s));
    XformParams X = xform_params(g, 0);
    X.bm_in = d_vertex_bitmap;
    X.clist = d_chunk_list;
    X.count_out = d_chunk_count;
    X.standalone_k = (int)log2_coarsen;
    launch_xform(g, X, s);
    k_clear_listed<<<g->num_sms * 4, 256, 0, s>>>(d_chunk_list, d_chunk_count, g->wb);
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
    if (log2_coarsen > kMaxCoarsen) return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be <= 7");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (!g->slice_ctr) WEDGE_TRY(dev_alloc(g, (void**)&g->slice_ctr, 16));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->rec, 0, sizeof(IterRec), s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(d_chunk_count, 0, 4, s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->slice_ctr, 0, 4, s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(d_warp_stats, 0, (size_t)nw * 8 * sizeof(uint64_t), s));
    XformParams X = xform_params(g, 0);
    X.bm_in = d_vertex_bitmap;
    X.clist = d_chunk_list;
    X.count_out = d_chunk_count;
    X.standalone_k = (int)log2_coarsen;
    X.wstat = reinterpret_cast<unsigned long long*>(d_warp_stats);
    X.slice_ctr = g->slice_ctr;
    if (schedule == 0) {
        launch_xform(g, X, s);
    } else {
        k_xform_static<<<g->xform_blocks, kXformThreads, 0, s>>>(X);
        count_launch();
    }
    k_clear_listed<<<g->num_sms * 4, 256, 0, s>>>(d_chunk_list, d_chunk_count, g->wb);
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
    if (log2_coarsen > kMaxCoarsen) return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be <= 7");
    if (iter + 2 >= g->rec_cap) return set_error(WEDGE_ERR_INVALID_ARG, "iter too large");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned sparse = d_chunk_list ? 1u : 0u;
    const unsigned cap = (unsigned)((g->NC + (1ull << log2_coarsen) - 1) >> log2_coarsen);
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
    for (uint32_t r : t->reserved)
        if (r) return set_error(WEDGE_ERR_INVALID_ARG, "reserved tuning fields must be zero");
    DeviceGuard dg(g->device);
    WEDGE_TRY_CUDA(cudaDeviceSynchronize());
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
                                              (g->NC + 31) / 32 + 1, g->rec, g->ctl, init, g->flist[0], g->visk,
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

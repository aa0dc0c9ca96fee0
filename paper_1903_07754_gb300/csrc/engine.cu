// The Wedge hot path on the device:
//   pull (dense over all chunks, or over the listed Wedge Frontier chunks) with
//   the frontier-fullness epilogue and the fullness decision,
//   frontier transformation (Sections 3.3, 3.4, 4),
//   run drivers for BFS, CC, SSSP and PageRank (Section 5).
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace wedge {

constexpr unsigned kFull = 0xFFFFFFFFu;
enum AppId { kBFS = 0, kCC = 1, kSSSP = 2, kPR = 3 };

// ------------------------------------------------------------------------
// Kernel parameter blocks
// ------------------------------------------------------------------------
struct PullParams {
    const uint32_t* src;
    const uint32_t* w;
    const uint2* cmeta;
    const uint32_t* vid;
    const uint32_t* outdeg;
    const uint32_t* eidx_off;
    unsigned long long E;
    unsigned long long NC;
    uint32_t* vals;             // BFS levels / CC labels / SSSP distances
    uint32_t* bm[2];            // vertex frontier bitmaps indexed by iteration parity
    const uint32_t* clist;      // Wedge Frontier list (sparse pulls)
    uint32_t* wb;               // Wedge Frontier bitmap, consumed words are zeroed
    uint2* pieces;              // transformation work produced for the next frontier
    IterRec* rec;
    RunCtl* ctl;
    const float* contrib;       // PageRank
    unsigned long long* acc;    // PageRank fixed-point in-edge sums
    unsigned int pr_iter;       // PageRank iteration (dangling slot bookkeeping)
    int decide;                 // elect a last block that takes the fullness decision
    int trace;
};

struct XformParams {
    const uint32_t* eidx;
    const uint2* pieces;
    uint32_t* wb;
    uint32_t* clist;
    IterRec* rec;
    RunCtl* ctl;
    uint32_t* bm_clear[2];      // run mode: bitmap cleared per parity (nullptr = none)
    unsigned long long bm_words;
    unsigned int* count_out;    // standalone mode: count destination (else rec[it].nchunks)
    int standalone_k;           // >= 0: standalone transformation at this coarsening
    int trace;
};

// ------------------------------------------------------------------------
// Application traits: the per-edge candidate and the combine operator
// ------------------------------------------------------------------------
template <int APP>
struct Traits;

template <>
struct Traits<kBFS> {  // found-a-parent flag, OR
    using T = uint32_t;
    static __device__ __forceinline__ T neutral() { return 0u; }
    static __device__ __forceinline__ T op(T a, T b) { return a | b; }
};
template <>
struct Traits<kCC> {  // label, min
    using T = uint32_t;
    static __device__ __forceinline__ T neutral() { return kInf; }
    static __device__ __forceinline__ T op(T a, T b) { return a < b ? a : b; }
};
template <>
struct Traits<kSSSP> {  // distance, min
    using T = uint32_t;
    static __device__ __forceinline__ T neutral() { return kInf; }
    static __device__ __forceinline__ T op(T a, T b) { return a < b ? a : b; }
};
template <>
struct Traits<kPR> {  // fixed-point contribution, sum
    using T = unsigned long long;
    static __device__ __forceinline__ T neutral() { return 0ull; }
    static __device__ __forceinline__ T op(T a, T b) { return a + b; }
};

template <int APP>
__device__ __forceinline__ typename Traits<APP>::T candidate(const PullParams& P, const uint32_t* cur,
                                                             uint32_t u, uint32_t w) {
    if constexpr (APP == kBFS) {
        return (__ldg(cur + (u >> 5)) >> (u & 31)) & 1u;
    } else if constexpr (APP == kCC) {
        return P.vals[u];
    } else if constexpr (APP == kSSSP) {
        const uint32_t d = P.vals[u];
        if (d == kInf) return kInf;
        const unsigned long long s = (unsigned long long)d + w;
        return s > kSat ? kSat : (uint32_t)s;
    } else {
        return __float2ull_rn(__ldg(P.contrib + u) * 0x1p62f);
    }
}

__device__ __forceinline__ bool set_bit(uint32_t* bm, uint32_t v) {
    const uint32_t bit = 1u << (v & 31);
    return (atomicOr(bm + (v >> 5), bit) & bit) == 0;
}

// Decision after pull it_next-1 for pull it_next (Section 3.4, Fig. 5):
// run by one thread once all blocks of the pull have published their sums.
__device__ void decide_next(IterRec* rec, RunCtl* C, unsigned it_next) {
    IterRec* r = rec + it_next;
    const unsigned long long F = __ldcg(&r->fullness);
    const unsigned nf = __ldcg(&r->nfront);
    unsigned sparse;
    if (C->switch_mode == WEDGE_SWITCH_ALWAYS_DENSE) sparse = 0;
    else if (C->switch_mode == WEDGE_SWITCH_ALWAYS_SPARSE) sparse = 1;
    else sparse = (F * 10000ull < (unsigned long long)C->tau_bp * C->E) ? 1u : 0u;
    r->mode = sparse;
    r->k = C->k;
    if (nf == 0) {
        C->done = 1;
    } else if (it_next >= C->max_iters) {
        C->done = 1;
        C->status |= kStatusMaxIters;
    }
    C->it = it_next;
}

// ------------------------------------------------------------------------
// Pull kernel (K1 dense / K4 sparse, with the K5 fullness epilogue)
//
// Work unit: a 32-edge chunk.  A warp processes a tile of four units; lane L
// holds edges 4*(L&7) .. 4*(L&7)+3 of unit L>>3 (one 16-byte load each of
// src, and of w for SSSP).  Dense pulls take units 0..NC-1 in order; sparse
// pulls expand list entry b into units b*2^k .. b*2^k+2^k-1.
// Destinations come from the chunk's head mask and first-destination index.
// A segmented scan over the 128 edges of the tile combines the candidates of
// each destination.  A segment that starts at its destination's first edge
// and ends right before the next destination's first edge holds all in-edges
// of that destination, so its lane is the only writer (plain store);
// other segments combine with atomics (min, or 64-bit add for PageRank).
// ------------------------------------------------------------------------
struct Stats {
    unsigned long long F;
    unsigned int n;
    unsigned int row;
};

template <int APP>
__device__ __forceinline__ void pull_tile(const PullParams& P, unsigned it, bool sparse, unsigned k,
                                          unsigned long long nunits, unsigned long long tile,
                                          const uint32_t* cur, uint32_t* next, Stats& st) {
    using Tr = Traits<APP>;
    using T = typename Tr::T;
    const unsigned lane = threadIdx.x & 31, g = lane >> 3, s = lane & 7;
    const unsigned long long j = tile * 4 + g;
    bool uvalid = j < nunits;
    unsigned long long c = 0;
    if (uvalid) {
        if (sparse) {
            const unsigned long long kmask = (1ull << k) - 1;
            const uint32_t b = P.clist[j >> k];
            c = ((unsigned long long)b << k) | (j & kmask);
            uvalid = c < P.NC;
            // the pull consumes the Wedge Frontier bitmap: zero its word
            if (uvalid && P.wb && s == 0 && (j & kmask) == 0) P.wb[b >> 5] = 0u;
        } else {
            c = j;
            uvalid = c < P.NC;
        }
    }
    const unsigned long long cprev = __shfl_up_sync(kFull, c, 8);
    const unsigned pvalid = __shfl_up_sync(kFull, (unsigned)uvalid, 8);
    const bool contig = g > 0 && pvalid && uvalid && c == cprev + 1;

    const unsigned long long p0 = c * 32 + 4 * s;
    uint2 meta = make_uint2(0u, 0u);
    unsigned next_head = 1u;  // head bit of position 32c+32 (1 past the end)
    int nvalid = 0;
    if (uvalid) {
        meta = __ldg(P.cmeta + c);
        if (s == 7 && c + 1 < P.NC) next_head = __ldg(&P.cmeta[c + 1].x) & 1u;
        const long long rem = (long long)P.E - (long long)p0;
        nvalid = rem >= 4 ? 4 : (rem > 0 ? (int)rem : 0);
    }
    uint32_t sv[4] = {0, 0, 0, 0}, wv[4] = {0, 0, 0, 0};
    if (nvalid == 4) {
        const uint4 q = __ldcs(reinterpret_cast<const uint4*>(P.src + p0));
        sv[0] = q.x; sv[1] = q.y; sv[2] = q.z; sv[3] = q.w;
        if constexpr (APP == kSSSP) {
            const uint4 r = __ldcs(reinterpret_cast<const uint4*>(P.w + p0));
            wv[0] = r.x; wv[1] = r.y; wv[2] = r.z; wv[3] = r.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (i < nvalid) {
                sv[i] = P.src[p0 + i];
                if constexpr (APP == kSSSP) wv[i] = P.w[p0 + i];
            }
    }
    const uint32_t heads = meta.x;
    T cand[4];
    bool hd[4], brk[4];
    uint32_t kid[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const unsigned idx = 4 * s + i;
        cand[i] = (i < nvalid) ? candidate<APP>(P, cur, sv[i], wv[i]) : Tr::neutral();
        hd[i] = (heads >> idx) & 1u;
        brk[i] = hd[i] || (idx == 0 && !contig);
        kid[i] = meta.y + __popc(heads & ((2u << idx) - 1u) & ~1u);
    }
    // in-lane segmented inclusive scan
    T inc[4];
    bool ish[4];
    T run = Tr::neutral();
    bool rsh = false;
    int first_brk = 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (brk[i]) {
            run = cand[i];
            rsh = hd[i];
            if (first_brk == 4) first_brk = i;
        } else {
            run = Tr::op(run, cand[i]);
        }
        inc[i] = run;
        ish[i] = rsh;
    }
    // cross-lane segmented scan of (has break, value, start-is-head)
    bool f = first_brk < 4;
    T v = run;
    bool sh = rsh;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned f2 = __shfl_up_sync(kFull, (unsigned)f, o);
        const T v2 = __shfl_up_sync(kFull, v, o);
        const unsigned sh2 = __shfl_up_sync(kFull, (unsigned)sh, o);
        if (lane >= (unsigned)o && !f) {
            v = Tr::op(v2, v);
            sh = sh2;
            f = f2;
        }
    }
    const T cv = __shfl_up_sync(kFull, v, 1);
    const bool csh = __shfl_up_sync(kFull, (unsigned)sh, 1);
    // what follows the lane's last edge
    const unsigned mypack = (unsigned)brk[0] | ((unsigned)hd[0] << 1) | ((nvalid > 0) << 2);
    const unsigned nx = __shfl_down_sync(kFull, mypack, 1);
    const bool nx_valid = lane < 31 && (nx & 4u);
    const bool nx_brk = nx & 1u, nx_hd = (nx >> 1) & 1u;

    uint32_t act_v[4];
    int nact = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i >= nvalid) break;
        bool end, end_head;
        if (i < 3) {
            if (i + 1 < nvalid) {
                end = brk[i + 1];
                end_head = hd[i + 1];
            } else {
                end = true;  // next position is past E
                end_head = true;
            }
        } else {
            end = !nx_valid || nx_brk;
            end_head = (s == 7) ? (next_head != 0) : (nx_valid ? nx_hd : true);
        }
        if (!end) continue;
        const T m = (i < first_brk) ? Tr::op(cv, inc[i]) : inc[i];
        const bool start_head = (i < first_brk) ? csh : ish[i];
        const bool excl = start_head && end_head;
        const uint32_t dv = __ldg(P.vid + kid[i]);
        if constexpr (APP == kBFS) {
            if (m && P.vals[dv] == kInf) {
                P.vals[dv] = it + 1;
                if (set_bit(next, dv)) act_v[nact++] = dv;
            }
        } else if constexpr (APP == kPR) {
            if (excl) P.acc[dv] = m;
            else if (m) atomicAdd(P.acc + dv, m);
        } else {
            if (m != kInf) {
                bool changed;
                if (excl) {
                    const uint32_t old = P.vals[dv];
                    changed = m < old;
                    if (changed) P.vals[dv] = m;
                } else {
                    changed = m < atomicMin(P.vals + dv, m);
                }
                if (changed && set_bit(next, dv)) act_v[nact++] = dv;
            }
        }
    }
    if constexpr (APP != kPR) {
        // frontier bookkeeping: fullness, size, edge-index work pieces
        uint32_t rb[4], rl[4];
        unsigned np = 0;
        for (int a = 0; a < nact; ++a) {
            const uint32_t u = act_v[a];
            rb[a] = __ldg(P.eidx_off + u);
            rl[a] = __ldg(P.eidx_off + u + 1) - rb[a];
            st.F += __ldg(P.outdeg + u);
            st.n += 1;
            st.row += rl[a];
            np += (rl[a] + 31u) >> 5;
        }
        unsigned incl = np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, o);
            if (lane >= (unsigned)o) incl += y;
        }
        const unsigned total = __shfl_sync(kFull, incl, 31);
        if (total) {
            unsigned base = 0;
            if (lane == 31) base = atomicAdd(&P.rec[it + 1].npieces, total);
            base = __shfl_sync(kFull, base, 31) + incl - np;
            for (int a = 0; a < nact; ++a)
                for (uint32_t q = 0; q < rl[a]; q += 32) {
                    const uint32_t len = rl[a] - q < 32u ? rl[a] - q : 32u;
                    P.pieces[base++] = make_uint2(rb[a] + q, len);
                }
        }
    }
}

template <int APP>
__global__ void __launch_bounds__(kPullThreads) k_pull(const PullParams P) {
    __shared__ unsigned long long s_F;
    __shared__ unsigned s_n, s_row, s_last;
    RunCtl* C = P.ctl;
    if (C->done) return;
    const unsigned it = C->it;
    const IterRec rin = P.rec[it];
    if (threadIdx.x == 0) {
        s_F = 0;
        s_n = 0;
        s_row = 0;
        if (P.trace && blockIdx.x == 0) P.rec[it].t_pull0 = global_timer();
        if constexpr (APP == kPR) {
            if (blockIdx.x == 0) C->dangling[(P.pr_iter + 1) & 1] = 0ull;
        }
    }
    __syncthreads();
    const bool sparse = rin.mode != 0;
    const unsigned k = rin.k;
    const unsigned long long nunits = sparse ? ((unsigned long long)rin.nchunks << k) : P.NC;
    const unsigned long long ntiles = (nunits + 3) / 4;
    const unsigned long long gw = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const uint32_t* cur = P.bm[it & 1];
    uint32_t* next = P.bm[(it + 1) & 1];
    Stats st{0ull, 0u, 0u};
    for (unsigned long long t = gw; t < ntiles; t += nw) pull_tile<APP>(P, it, sparse, k, nunits, t, cur, next, st);

    if constexpr (APP != kPR) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            st.F += __shfl_down_sync(kFull, st.F, o);
            st.n += __shfl_down_sync(kFull, st.n, o);
            st.row += __shfl_down_sync(kFull, st.row, o);
        }
        if ((threadIdx.x & 31) == 0 && st.n) {
            atomicAdd(&s_F, st.F);
            atomicAdd(&s_n, st.n);
            atomicAdd(&s_row, st.row);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_n) {
            atomicAdd(&P.rec[it + 1].fullness, s_F);
            atomicAdd(&P.rec[it + 1].nfront, s_n);
            atomicAdd(&P.rec[it + 1].rowsum, s_row);
        }
        s_last = 0;
        if (P.decide) {
            __threadfence();
            const unsigned ticket = atomicAdd(&C->ticket, 1u);
            s_last = ticket == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        decide_next(P.rec, C, it + 1);
        C->ticket = 0;
        if (P.trace) P.rec[it].t_pull1 = global_timer();
    }
}

// ------------------------------------------------------------------------
// Transformation (K2): expand the work pieces of the frontier's edge-index
// rows, set the Wedge Frontier bits (bit b = list entry b at coarsening k)
// and append every newly set bit to the Wedge Frontier list.  The bitmap
// removes duplicates (Section 4); only the first setter of a bit appends it.
// ------------------------------------------------------------------------
__device__ __forceinline__ void expand_pieces(const XformParams& X, unsigned n, unsigned k, unsigned* count) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned long long gw = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (unsigned long long base = gw * 32; base < n; base += nw * 32) {
        const unsigned long long idx = base + lane;
        const uint2 pc = idx < n ? X.pieces[idx] : make_uint2(0u, 0u);
        unsigned incl = pc.y;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, o);
            if (lane >= (unsigned)o) incl += y;
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
            bool fresh = false;
            uint32_t b = 0;
            if (act) {
                const uint32_t chunk = __ldg(X.eidx + st + (e - ex));
                b = chunk >> k;
                const uint32_t bit = 1u << (b & 31);
                fresh = (atomicOr(X.wb + (b >> 5), bit) & bit) == 0;
            }
            const unsigned m = __ballot_sync(kFull, fresh);
            if (m) {
                const unsigned leader = __ffs(m) - 1;
                unsigned slot = 0;
                if (lane == leader) slot = atomicAdd(count, (unsigned)__popc(m));
                slot = __shfl_sync(kFull, slot, leader);
                if (fresh) X.clist[slot + __popc(m & lt_mask)] = b;
            }
        }
    }
}

__global__ void __launch_bounds__(kXformThreads) k_transform(const XformParams X) {
    RunCtl* C = X.ctl;
    if (X.standalone_k >= 0) {
        expand_pieces(X, __ldcg(&X.rec[0].npieces), (unsigned)X.standalone_k, X.count_out);
        return;
    }
    if (C->done) return;
    const unsigned it = C->it;
    if (X.trace && blockIdx.x == 0 && threadIdx.x == 0) X.rec[it].t_xf0 = global_timer();
    // run bookkeeping: the bitmap that pull `it` fills must be clear, and so
    // must the record that pull `it` accumulates into
    uint32_t* clr = X.bm_clear[(it + 1) & 1];
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
    if (clr)
        for (unsigned long long i = tid; i < X.bm_words; i += nth) clr[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x < sizeof(IterRec) / 4)
        reinterpret_cast<unsigned*>(X.rec + it + 1)[threadIdx.x] = 0u;
    const IterRec r = X.rec[it];
    if (r.mode != 0) expand_pieces(X, r.npieces, r.k, &X.rec[it].nchunks);
    if (X.trace) {
        __syncthreads();
        if (threadIdx.x == 0) atomicMax(&X.rec[it].t_xf1, global_timer());
    }
}

// Vertex bitmap -> frontier size, fullness and work pieces (used for the
// initial frontier and by the standalone transformation entry point).
__global__ void k_frontier_scan(const uint32_t* __restrict__ bm, uint32_t V, const uint32_t* __restrict__ outdeg,
                                const uint32_t* __restrict__ eidx_off, uint2* __restrict__ pieces, IterRec* rec,
                                RunCtl* C, int decide) {
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
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            const uint32_t u = (uint32_t)(wi * 32 + b);
            const uint32_t rb = eidx_off[u], rl = eidx_off[u + 1] - rb;
            F += outdeg[u];
            n += 1;
            row += rl;
            const unsigned np = (rl + 31u) >> 5;
            if (np) {
                unsigned slot = atomicAdd(&rec->npieces, np);
                for (uint32_t q = 0; q < rl; q += 32) pieces[slot++] = make_uint2(rb + q, rl - q < 32u ? rl - q : 32u);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        F += __shfl_down_sync(kFull, F, o);
        n += __shfl_down_sync(kFull, n, o);
        row += __shfl_down_sync(kFull, row, o);
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
        s_last = 0;
        if (decide) {
            __threadfence();
            s_last = atomicAdd(&C->ticket, 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        decide_next(rec, C, 0);  // rec points at slot 0 for the initial frontier
        C->ticket = 0;
    }
}

// Run start: values, initial frontier F_0, records 0 and 1, control block.
__global__ void k_run_init(int app, uint32_t V, uint32_t root, uint32_t* vals, uint32_t* bm0, uint32_t* bm1,
                           uint32_t* wb, unsigned long long wb_words, IterRec* rec, RunCtl* C, RunCtl init) {
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
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
    }
}

// ------------------------------------------------------------------------
// PageRank vertex step (K6): pr = (1-d)/V + d*(acc + D/V); then either the
// next iteration's contributions and dangling mass, or the final ranks.
// ------------------------------------------------------------------------
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
    for (int o = 16; o > 0; o >>= 1) dang += __shfl_down_sync(kFull, dang, o);
    if ((threadIdx.x & 31) == 0 && dang) atomicAdd(&C->dangling[0], dang);
}

__global__ void k_pr_apply(uint32_t V, const uint32_t* __restrict__ outdeg, const uint32_t* __restrict__ split_bm,
                           unsigned long long* __restrict__ acc, float* __restrict__ contrib,
                           float* __restrict__ out, RunCtl* C, unsigned t, int last, float base, float d) {
    const float dv = __ull2float_rn(__ldcg(&C->dangling[t & 1])) * 0x1p-62f / (float)V;
    unsigned long long dang = 0;
    for (unsigned long long v = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; v < V;
         v += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long a = acc[v];
        if ((__ldg(split_bm + (v >> 5)) >> (v & 31)) & 1u) acc[v] = 0ull;
        const float s = __ull2float_rn(a) * 0x1p-62f + dv;
        const float pr = fmaf(d, s, base);
        if (last) {
            out[v] = pr;
        } else {
            const uint32_t od = outdeg[v];
            contrib[v] = od ? pr / (float)od : 0.0f;
            if (!od) dang += __float2ull_rn(pr * 0x1p62f);
        }
    }
    if (!last) {
        for (int o = 16; o > 0; o >>= 1) dang += __shfl_down_sync(kFull, dang, o);
        if ((threadIdx.x & 31) == 0 && dang) atomicAdd(&C->dangling[(t + 1) & 1], dang);
    }
}

__global__ void k_clear_listed(const uint32_t* __restrict__ list, const uint32_t* __restrict__ count,
                               uint32_t* __restrict__ wb) {
    const unsigned n = *count;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        wb[list[i] >> 5] = 0u;
}

__global__ void k_ctl_init(RunCtl* C, RunCtl init) {
    if (threadIdx.x == 0) *C = init;
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

__global__ void k_standalone_out(const IterRec* rec, unsigned iter, unsigned long long* fullness, uint32_t* nfront) {
    if (threadIdx.x == 0) {
        *fullness = rec[iter + 1].fullness;
        *nfront = rec[iter + 1].nfront;
    }
}

// ------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------
static int pull_grid(const wedge_graph* g) { return g->pull_blocks; }

template <int APP>
static void launch_pull(const PullParams& P, int blocks, cudaStream_t s) {
    k_pull<APP><<<blocks, kPullThreads, 0, s>>>(P);
    count_launch();
}

static void launch_pull_app(int app, const PullParams& P, int blocks, cudaStream_t s) {
    switch (app) {
        case kBFS: launch_pull<kBFS>(P, blocks, s); break;
        case kCC: launch_pull<kCC>(P, blocks, s); break;
        case kSSSP: launch_pull<kSSSP>(P, blocks, s); break;
        default: launch_pull<kPR>(P, blocks, s); break;
    }
}

wedge_status ensure_run_scratch(wedge_graph* g) {
    if (g->ctl) return WEDGE_OK;
    const uint64_t V = g->V, NC = g->NC;
    const uint64_t words = (V + 31) / 32;
    WEDGE_TRY(dev_alloc(g, (void**)&g->vals, V * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->bm[0], words * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->bm[1], words * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->wb, ((NC + 31) / 32 + 1) * 4));
    WEDGE_TRY_CUDA(cudaMemset(g->wb, 0, ((NC + 31) / 32 + 1) * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->clist, (NC + 1) * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->pieces, (g->npieces_max + 1) * sizeof(uint2)));
    g->rec_cap = kDefaultMaxIters + 2;
    WEDGE_TRY(dev_alloc(g, (void**)&g->rec, (uint64_t)g->rec_cap * sizeof(IterRec)));
    WEDGE_TRY(dev_alloc(g, (void**)&g->ctl, sizeof(RunCtl)));
    WEDGE_TRY_CUDA(cudaMemset(g->ctl, 0, sizeof(RunCtl)));
    WEDGE_TRY_CUDA(cudaMallocHost((void**)&g->h_ctl, sizeof(RunCtl)));
    WEDGE_TRY(dev_alloc(g, (void**)&g->contrib, V * 4));
    WEDGE_TRY(dev_alloc(g, (void**)&g->acc, V * 8));
    WEDGE_TRY_CUDA(cudaEventCreate(&g->ev0));
    WEDGE_TRY_CUDA(cudaEventCreate(&g->ev1));
    int per_sm = 0;
    WEDGE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pull<kSSSP>, kPullThreads, 0));
    if (per_sm < 1) per_sm = 1;
    g->pull_blocks = g->num_sms * per_sm;
    g->xform_blocks = g->num_sms * 4;
    return WEDGE_OK;
}

static PullParams pull_params(wedge_graph* g, int trace) {
    PullParams P{};
    P.src = g->src;
    P.w = g->w;
    P.cmeta = g->cmeta;
    P.vid = g->vid;
    P.outdeg = g->outdeg;
    P.eidx_off = g->eidx_off;
    P.E = g->E;
    P.NC = g->NC;
    P.vals = g->vals;
    P.bm[0] = g->bm[0];
    P.bm[1] = g->bm[1];
    P.clist = g->clist;
    P.wb = g->wb;
    P.pieces = g->pieces;
    P.rec = g->rec;
    P.ctl = g->ctl;
    P.contrib = g->contrib;
    P.acc = g->acc;
    P.decide = 1;
    P.trace = trace;
    return P;
}

static XformParams xform_params(wedge_graph* g, int trace) {
    XformParams X{};
    X.eidx = g->eidx;
    X.pieces = g->pieces;
    X.wb = g->wb;
    X.clist = g->clist;
    X.rec = g->rec;
    X.ctl = g->ctl;
    X.bm_clear[0] = g->bm[0];
    X.bm_clear[1] = g->bm[1];
    X.bm_words = ((uint64_t)g->V + 31) / 32;
    X.count_out = nullptr;
    X.standalone_k = -1;
    X.trace = trace;
    return X;
}

static wedge_status check_opts(const wedge_opts* o) {
    if (o->log2_coarsen > kMaxCoarsen) return set_error(WEDGE_ERR_INVALID_ARG, "log2_coarsen must be <= 7");
    if (o->switch_mode > WEDGE_SWITCH_ALWAYS_SPARSE) return set_error(WEDGE_ERR_INVALID_ARG, "bad switch_mode");
    if (o->reserved[0] || o->reserved[1] || o->reserved[2])
        return set_error(WEDGE_ERR_INVALID_ARG, "reserved option fields must be zero");
    return WEDGE_OK;
}

static wedge_status fill_stats(wedge_graph* g, cudaStream_t s, wedge_stats* stats) {
    WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    WEDGE_TRY_CUDA(cudaMemcpy(g->h_ctl, g->ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost));
    const uint32_t iters = g->h_ctl->it;
    g->last_iters = iters;
    if (stats) {
        std::vector<IterRec> r(iters + 1);
        if (iters) WEDGE_TRY_CUDA(cudaMemcpy(r.data(), g->rec, (size_t)iters * sizeof(IterRec), cudaMemcpyDeviceToHost));
        stats->iters = iters;
        stats->sparse_iters = 0;
        stats->edges_pulled = 0;
        stats->chunks_listed = 0;
        for (uint32_t t = 0; t < iters; ++t) {
            if (r[t].mode) {
                stats->sparse_iters++;
                stats->chunks_listed += r[t].nchunks;
                uint64_t e = (uint64_t)r[t].nchunks << (5 + r[t].k);
                stats->edges_pulled += e < g->E ? e : g->E;
            } else {
                stats->edges_pulled += g->E;
            }
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, g->ev0, g->ev1);
        stats->device_ms = ms;
    }
    if (g->h_ctl->status & kStatusMaxIters)
        return set_error(WEDGE_ERR_MAX_ITERS, "frontier still non-empty at max_iters");
    return WEDGE_OK;
}

// The loop: pull and transform alternate on the device; the host only polls
// the done flag after each batch of iterations (kernels after the last
// iteration return at once).
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
    const uint32_t max_iters = o.max_iters ? (o.max_iters < kDefaultMaxIters ? o.max_iters : kDefaultMaxIters)
                                           : kDefaultMaxIters;
    const int trace = o.trace ? 1 : 0;
    RunCtl init{};
    init.max_iters = max_iters;
    init.switch_mode = o.switch_mode == WEDGE_SWITCH_LEARNED ? WEDGE_SWITCH_THRESHOLD : o.switch_mode;
    init.tau_bp = o.tau_bp;
    init.k = o.log2_coarsen;
    init.E = g->E;
    const uint64_t wb_words = (g->NC + 31) / 32 + 1;
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev0, s));
    k_run_init<<<g->num_sms * 4, 256, 0, s>>>(app, g->V, root, g->vals, g->bm[0], g->bm[1], g->wb, wb_words,
                                              g->rec, g->ctl, init);
    k_frontier_scan<<<g->num_sms * 4, 256, 0, s>>>(g->bm[0], g->V, g->outdeg, g->eidx_off, g->pieces, g->rec,
                                                   g->ctl, 1);
    PullParams P = pull_params(g, trace);
    XformParams X = xform_params(g, trace);
    k_transform<<<g->xform_blocks, kXformThreads, 0, s>>>(X);
    count_launch(3);
    WEDGE_TRY_CUDA(cudaGetLastError());
    const int batch = 8;
    uint32_t launched = 0;
    for (;;) {
        for (int b = 0; b < batch; ++b) {
            launch_pull_app(app, P, pull_grid(g), s);
            k_transform<<<g->xform_blocks, kXformThreads, 0, s>>>(X);
            count_launch();
        }
        launched += batch;
        WEDGE_TRY_CUDA(cudaGetLastError());
        WEDGE_TRY_CUDA(cudaMemcpyAsync(g->h_ctl, g->ctl, sizeof(RunCtl), cudaMemcpyDeviceToHost, s));
        WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
        if (g->h_ctl->done || launched > max_iters + 2) break;
    }
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev1, s));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(out, g->vals, (uint64_t)g->V * 4, cudaMemcpyDefault, s));
    g->last_trace = trace;
    g->last_stream = s;
    return fill_stats(g, s, stats);
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
    (void)opts;
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t V = g->V;
    const int vb = g->num_sms * 8;
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev0, s));
    RunCtl init{};
    init.max_iters = 0xFFFFFFFFu;
    k_ctl_init<<<1, 32, 0, s>>>(g->ctl, init);
    count_launch();
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->rec, 0, 2 * sizeof(IterRec), s));
    k_pr_init<<<vb, 256, 0, s>>>(V, g->outdeg, g->contrib, g->acc, g->ctl);
    count_launch();
    PullParams P = pull_params(g, 0);
    P.decide = 0;
    const float base = (1.0f - damping) / (float)V;
    if (iters == 0) {
        // pr0 = 1/V everywhere
        std::vector<float> h(V, 1.0f / (float)V);
        WEDGE_TRY_CUDA(cudaMemcpyAsync(d_rank, h.data(), (uint64_t)V * 4, cudaMemcpyHostToDevice, s));
        WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    }
    for (uint32_t t = 0; t < iters; ++t) {
        P.pr_iter = t;
        launch_pull<kPR>(P, pull_grid(g), s);
        const int last = (t + 1 == iters);
        k_pr_apply<<<vb, 256, 0, s>>>(V, g->outdeg, g->split_bm, g->acc, g->contrib, g->contrib, g->ctl, t, last,
                                      base, damping);
        count_launch();
    }
    WEDGE_TRY_CUDA(cudaGetLastError());
    WEDGE_TRY_CUDA(cudaEventRecord(g->ev1, s));
    if (iters) WEDGE_TRY_CUDA(cudaMemcpyAsync(d_rank, g->contrib, (uint64_t)V * 4, cudaMemcpyDefault, s));
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
    return WEDGE_OK;
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
    k_frontier_scan<<<g->num_sms * 4, 256, 0, s>>>(d_vertex_bitmap, g->V, g->outdeg, g->eidx_off, g->pieces, g->rec,
                                                   g->ctl, 0);
    XformParams X{};
    X.eidx = g->eidx;
    X.pieces = g->pieces;
    X.wb = g->wb;
    X.clist = d_chunk_list;
    X.rec = g->rec;
    X.ctl = g->ctl;
    X.count_out = d_chunk_count;
    X.standalone_k = (int)log2_coarsen;
    k_transform<<<g->xform_blocks, kXformThreads, 0, s>>>(X);
    k_clear_listed<<<g->num_sms * 4, 256, 0, s>>>(d_chunk_list, d_chunk_count, g->wb);
    count_launch(3);
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
    P.vals = d_values;
    P.bm[iter & 1] = const_cast<uint32_t*>(d_cur_bitmap ? d_cur_bitmap : d_next_bitmap);
    P.bm[(iter + 1) & 1] = d_next_bitmap;
    P.clist = d_chunk_list ? d_chunk_list : g->clist;
    P.wb = nullptr;  // a caller's list has no library bitmap behind it
    P.decide = 0;
    launch_pull_app(app, P, pull_grid(g), s);
    k_standalone_out<<<1, 32, 0, s>>>(g->rec, iter, reinterpret_cast<unsigned long long*>(d_fullness), d_nfront);
    count_launch(2);
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

wedge_status wedge_get_trace(wedge_graph_t g, wedge_iter_record* out, uint32_t cap, uint32_t* n) {
    if (!g || !n || (!out && cap)) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(g->device);
    WEDGE_TRY_CUDA(cudaStreamSynchronize(g->last_stream));
    const uint32_t iters = g->last_iters;
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

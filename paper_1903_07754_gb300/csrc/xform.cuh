// The frontier transformation (Sections 3.3, 4; K2 and the compaction K3):
// its parameter block, the library's load-balanced scan and expansion, and
// the paper's static schedule with per-warp load-balance accounting
// (Section 5.3, Fig. 13).  Included by engine.cu after pull.cuh.
#pragma once

#include "common.cuh"

namespace wedge {

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
    int standalone;              // nonzero: a standalone transformation (not a run's)
    int standalone_k;            // ... at this precision (-2 .. 7)
    const uint32_t* eidx8;       // the edge index in 8-edge units (precisions k < 0)
    const uint32_t* eidx8_off;
    int trace;
    int direct;                  // run mode: rows of at most 32 entries may be expanded by the scan
    // load-balance accounting of a standalone transformation (nullptr: off):
    // per warp and kernel {start ns, end ns, busy SM cycles, SM id}
    unsigned long long* wstat;
    unsigned* slice_ctr;         // the paper's schedule: next frontier slice
    uint32_t* longs;             // long rows of the transformation (nullptr: none listed)
    unsigned* task_ctr;          // the expansion's next task (zeroed by the scan; nullptr: static tasks)
    // compressed edge index (zhdr == nullptr: the plain index)
    const uint2* zhdr;
    const uint32_t* zwords;
    const uint32_t* zbo;
    uint4* zpieces;
};


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
// Where the scan writes the pieces: plain pieces {first entry, length}, or,
// with the compressed edge index, {block header .x, .y, length, 0}.
// Rows longer than kLongRow entries are not cut into pieces by the scan
// (one warp writing a hub's thousands of pieces held the whole scan): they
// are listed, and their 32-entry units are spread over every warp of the
// expansion instead.
constexpr unsigned kLongRow = 32u * 64u;
constexpr unsigned kLongCap = 1024;  // long rows listed per transformation (more: pieces)

struct PieceOut {
    uint2* pieces;
    uint4* zpieces;         // non-null: compressed edge index
    const uint32_t* zbo;    // first block of each row
    const uint2* zhdr;      // block headers
    uint32_t* longs;        // non-null: long rows go to this list (kLongCap entries)
    unsigned* nlong;        // ... and its count
};

// The edge index a transformation at precision kk reads: chunk ids shifted
// by kk (kk >= 0; compressed when the graph's tuning asks for it), or
// 8-edge-unit ids shifted by kk + 2 (kk = -2, -1: entries of 8 or 16 edges).
struct IndexSel {
    const uint32_t* eoff;
    const uint32_t* ei;
    unsigned shift;
    bool z;
};

__device__ __forceinline__ IndexSel select_index(const XformParams& X, int kk) {
    IndexSel r;
    if (kk < 0) {
        r.eoff = X.eidx8_off;
        r.ei = X.eidx8;
        r.shift = (unsigned)(kk + 2);
        r.z = false;
    } else {
        r.eoff = X.eidx_off;
        r.ei = X.eidx;
        r.shift = (unsigned)kk;
        r.z = X.zhdr != nullptr;
    }
    return r;
}

__device__ __forceinline__ PieceOut piece_out(const XformParams& X, unsigned* nlong, bool z) {
    PieceOut po;
    po.pieces = X.pieces;
    po.zpieces = z ? X.zpieces : nullptr;
    po.zbo = X.zbo;
    po.zhdr = X.zhdr;
    po.longs = X.longs;
    po.nlong = nlong;
    return po;
}

// Reserves list slots for the long rows a lane holds (the vertices at the
// bits of `cand` in bitmap word wi), one atomic per warp; rows that find no
// slot (the list is full) stay pieces.  Returns the bits of the rows listed.
__device__ __forceinline__ uint32_t list_long_rows(const PieceOut& po, unsigned long long wi, uint32_t cand) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned nl = __popc(cand);
    unsigned incl = nl;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, incl, d);
        if (lane >= (unsigned)d) incl += y;
    }
    const unsigned total = __shfl_sync(kFull, incl, 31);
    if (!total) return 0u;
    unsigned base = 0;
    if (lane == 31) base = atomicAdd(po.nlong, total);
    base = __shfl_sync(kFull, base, 31);
    unsigned slot = base + incl - nl;
    uint32_t listed = 0;
    for (uint32_t c = cand; c; c &= c - 1, ++slot) {
        if (slot >= kLongCap) break;
        const unsigned bpos = __ffs(c) - 1;
        po.longs[slot] = (uint32_t)(wi * 32 + bpos);
        listed |= 1u << bpos;
    }
    return listed;
}

__device__ __forceinline__ void write_pieces(const PieceOut& po, unsigned slot0, unsigned total, uint32_t rb,
                                             uint32_t rl, uint32_t zb, unsigned excl) {
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
        const uint32_t z = __shfl_sync(kFull, zb, jx);
        const unsigned qi = i - __shfl_sync(kFull, excl, jx);
        const unsigned q = qi * 32u;
        if (i < total) {
            if (po.zpieces) {
                const uint2 h = __ldg(po.zhdr + z + qi);
                po.zpieces[slot0 + i] = make_uint4(h.x, h.y, min(32u, l - q), 0u);
            } else {
                po.pieces[slot0 + i] = make_uint2(b + q, min(32u, l - q));
            }
        }
    }
}

// Warp-level scan of bitmap words [gw*32, ...) step nw*32: pieces of the
// active vertices' edge-index rows, one reservation per warp on *npieces.
__device__ __forceinline__ void xform_scan_words(const uint32_t* bm, uint32_t V, unsigned long long words,
                                                 const uint32_t* __restrict__ eidx_off, const PieceOut& po,
                                                 unsigned* npieces, unsigned long long gw, unsigned long long nw) {
    const unsigned lane = threadIdx.x & 31;
    for (unsigned long long base = gw * 32; base < words; base += nw * 32) {
        const unsigned long long wi = base + lane;
        uint32_t word = wi < words ? __ldcg(bm + wi) : 0u;
        if (wi == words - 1 && (V & 31)) word &= (1u << (V & 31)) - 1u;
        uint32_t cand = 0;  // active vertices with long rows
        unsigned np = 0;
        for (uint32_t w = word; w; w &= w - 1) {
            const unsigned bpos = __ffs(w) - 1;
            const uint32_t u = (uint32_t)(wi * 32 + bpos);
            const uint32_t len = __ldg(eidx_off + u + 1) - __ldg(eidx_off + u);
            if (po.longs && len > kLongRow) cand |= 1u << bpos;
            else np += (len + 31u) >> 5;
        }
        // rows that went to the long list; the others stay pieces
        const uint32_t longmask = (po.longs && __any_sync(kFull, cand != 0)) ? list_long_rows(po, wi, cand) : 0u;
        for (uint32_t c = cand & ~longmask; c; c &= c - 1) {
            const uint32_t u = (uint32_t)(wi * 32 + __ffs(c) - 1);
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
            uint32_t rb = 0, rl = 0, zb = 0;
            if (rem) {
                const unsigned bpos = __ffs(rem) - 1;
                const uint32_t u = (uint32_t)(wi * 32 + bpos);
                rem &= rem - 1;
                rb = __ldg(eidx_off + u);
                rl = ((longmask >> bpos) & 1u) ? 0u : __ldg(eidx_off + u + 1) - rb;
                if (po.zpieces) zb = __ldg(po.zbo + u);
            }
            const unsigned p = (rl + 31u) >> 5;
            unsigned pi = p;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned y = __shfl_up_sync(kFull, pi, d);
                if (lane >= (unsigned)d) pi += y;
            }
            const unsigned rt = __shfl_sync(kFull, pi, 31);
            write_pieces(po, slot + done, rt, rb, rl, zb, pi - p);
            done += rt;
        }
    }
}

// Same as xform_scan_words over an explicit list of n frontier vertices.
__device__ __forceinline__ void xform_scan_list(const uint32_t* list, unsigned n,
                                                const uint32_t* __restrict__ eidx_off, const PieceOut& po,
                                                unsigned* npieces, unsigned long long gw, unsigned long long nw) {
    const unsigned lane = threadIdx.x & 31;
    for (unsigned long long base = gw * 32; base < n; base += nw * 32) {
        const unsigned long long i = base + lane;
        uint32_t rb = 0, rl = 0, zb = 0;
        uint32_t u = 0;
        if (i < n) {
            u = __ldcg(list + i);
            rb = __ldg(eidx_off + u);
            rl = __ldg(eidx_off + u + 1) - rb;
            if (po.zpieces) zb = __ldg(po.zbo + u);
        }
        if (po.longs) {
            const bool lg = rl > kLongRow;
            const unsigned lm = __ballot_sync(kFull, lg);
            if (lm) {
                unsigned base = 0;
                if (lane == 0) base = atomicAdd(po.nlong, (unsigned)__popc(lm));
                base = __shfl_sync(kFull, base, 0);
                const unsigned slot = base + __popc(lm & ((1u << lane) - 1u));
                if (lg && slot < kLongCap) {
                    po.longs[slot] = u;
                    rl = 0;
                }
            }
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
        write_pieces(po, slot, total, rb, rl, zb, incl - np);
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

// One round of 32 entries (lane: entry b, act = it holds one), in two
// halves so that a warp keeps two rounds' atomics in flight:
//  round_issue: Wedge bitmap bits set with one atomicOr per run of lanes on
//    a word (neighbouring lanes often share a word: always for a hub's row
//    at coarse precision);
//  round_finish: within a run the first lane holding an entry owns it, fresh
//    if the word did not have its bit before; fresh entries are staged (or
//    appended) to the list.
struct Round {
    uint32_t b, bit, old;
    unsigned rs, re;
    bool act;
};

__device__ __forceinline__ Round round_issue(uint32_t b, bool act, uint32_t* wb) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    Round r;
    r.b = b;
    r.act = act;
    const uint32_t word = b >> 5;
    r.bit = act ? 1u << (b & 31) : 0u;
    const uint32_t wprev = __shfl_up_sync(kFull, word, 1);
    const unsigned starts = __ballot_sync(kFull, lane == 0 || word != wprev);
    r.rs = 31 - __clz(starts & (lt_mask | (1u << lane)));      // run start
    const unsigned above = starts & ~(lt_mask | (1u << lane));
    r.re = above ? (unsigned)__ffs(above) - 2 : 31u;           // run end
    uint32_t bits = r.bit;
#pragma unroll
    for (unsigned d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, bits, d);
        if (lane >= r.rs + d) bits |= y;
    }
    r.old = 0;
    if (lane == r.re && act) r.old = atomicOr(wb + word, bits);
    return r;
}

__device__ __forceinline__ void round_finish(const Round& r, uint32_t* list, unsigned* count, uint32_t* stage,
                                             unsigned& staged) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const uint32_t old = __shfl_sync(kFull, r.old, r.re);
    const unsigned run = (r.re == 31 ? kFull : ((2u << r.re) - 1u)) & ~((1u << r.rs) - 1u);
    const unsigned same = __match_any_sync(kFull, r.b) & run;
    const bool fresh = r.act && (unsigned)(__ffs(same) - 1) == lane && !(old & r.bit);
    const unsigned m = __ballot_sync(kFull, fresh);
    if (m && stage) {
        const unsigned nm = __popc(m);
        if (staged + nm > kAppendStage) {
            flush_staged(list, count, stage, staged);
            staged = 0;
        }
        if (fresh) stage[staged + __popc(m & lt_mask)] = r.b;
        staged += nm;
    } else if (m) {
        const unsigned leader = __ffs(m) - 1;
        unsigned slot = 0;
        if (lane == leader) slot = atomicAdd(count, (unsigned)__popc(m));
        slot = __shfl_sync(kFull, slot, leader);
        if (fresh) list[slot + __popc(m & lt_mask)] = r.b;
    }
}

// Entry value x of a compressed block's lane: the first entry (i == 0) or
// the packed difference i (w bits at bit (i-1)*w of the block's words).
__device__ __forceinline__ uint32_t z_raw(bool act, unsigned i, uint32_t hx, uint32_t hy,
                                          const uint32_t* __restrict__ zwords) {
    const unsigned w = hx >> 27;
    if (!act) return 0u;
    if (i == 0) return hx & 0x7FFFFFFu;
    if (!w) return 0u;
    const unsigned bit = (i - 1) * w, j = bit >> 5, r = bit & 31u;
    unsigned long long two = __ldg(zwords + hy + j);
    if (r + w > 32u) two |= (unsigned long long)__ldg(zwords + hy + j + 1) << 32;
    return (uint32_t)(two >> r) & ((1u << w) - 1u);
}

// Inclusive sum of x over runs of lanes with equal `key` (the lanes of one
// block), plus `carry` on the run that starts at lane 0 when that run
// continues a block from the previous round (cont).
__device__ __forceinline__ uint32_t z_scan(uint32_t x, unsigned key, bool cont, uint32_t carry) {
    const unsigned lane = threadIdx.x & 31;
    const unsigned kprev = __shfl_up_sync(kFull, key, 1);
    const unsigned heads = __ballot_sync(kFull, lane == 0 || key != kprev);
    const unsigned rs = 31 - __clz(heads & ((2u << lane) - 1u));
#pragma unroll
    for (unsigned d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= rs + d) x += y;
    }
    if (rs == 0 && cont) x += carry;
    return x;
}

// Warp-level expansion of n pieces (and of the long rows): with Z, the
// pieces are compressed blocks {header .x, .y, length, 0}, and each lane
// decodes its entry, the block's first entry plus the prefix sum of the
// packed differences over the block's lanes (a block cut by a round
// boundary carries its last decoded entry into the next round).  The next
// round's entries are loaded before the current round's atomics.
// SRC: kSrcPieces (pieces_v: uint2 pieces), kSrcZPieces (uint4 pieces of
// the compressed index) or kSrcRows (pieces_v: a frontier list whose every
// edge-index row, start eidx_off[u], has at most 32 entries: each row is
// one piece).
constexpr int kSrcPieces = 0, kSrcZPieces = 1, kSrcRows = 2;

template <int SRC>
__device__ __forceinline__ void xform_expand_pieces(const void* pieces_v, unsigned n, unsigned k,
                                                    const uint32_t* __restrict__ eidx, uint32_t* wb, uint32_t* list,
                                                    unsigned* count, unsigned long long gw, unsigned long long nw,
                                                    uint32_t* stage = nullptr, const uint32_t* longs = nullptr,
                                                    const uint32_t* s_lpre = nullptr, unsigned nlong = 0,
                                                    const uint32_t* __restrict__ eidx_off = nullptr,
                                                    const uint32_t* __restrict__ zbo = nullptr,
                                                    const uint2* __restrict__ zhdr = nullptr,
                                                    unsigned* task_ctr = nullptr) {
    unsigned staged = 0;  // warp-uniform
    const unsigned lane = threadIdx.x & 31;
    // 32-bit arithmetic: n < 2^32 pieces, nw < 2^32 warps
    const unsigned per = n / (unsigned)nw;
    const unsigned ppt = per >= 32 ? 32u : (per < 1 ? 1u : per);
    // tasks of ppt pieces: warp gw takes task gw first; when there are more
    // tasks than warps the rest come from *task_ctr (zeroed by the scan) as
    // warps become free, else task gw + nw, gw + 2nw, ...  (A small frontier
    // then costs no counter atomics: every warp would hit the one address.)
    const unsigned long long ntasks = ppt == 1 ? n : (n - 1) / ppt + 1;  // n >= 1 when ppt > 1
    const bool dyn = task_ctr != nullptr && ntasks > nw;
    unsigned long long task = gw;
    for (bool first = true;; first = false) {
        if (!first) {
            if (dyn) {
                unsigned t = 0;
                if (lane == 0) t = atomicAdd(task_ctr, 1u);
                task = nw + __shfl_sync(kFull, t, 0);
            } else {
                task += nw;
            }
        }
        if (task >= ntasks) break;
        const unsigned long long base = task * ppt;
        const unsigned long long idx = base + lane;
        const bool have = lane < ppt && idx < n;
        uint2 pc;        // plain, rows: {first entry, length}; Z: {header .x, header .y}
        unsigned plen;   // piece length
        if constexpr (SRC == kSrcZPieces) {
            const uint4 z = have ? __ldcg(static_cast<const uint4*>(pieces_v) + idx) : make_uint4(0u, 0u, 0u, 0u);
            pc = make_uint2(z.x, z.y);
            plen = z.z;
        } else if constexpr (SRC == kSrcRows) {
            pc = make_uint2(0u, 0u);
            if (have) {
                const uint32_t u = __ldcg(static_cast<const uint32_t*>(pieces_v) + idx);
                pc.x = __ldg(eidx_off + u);
                pc.y = __ldg(eidx_off + u + 1) - pc.x;
            }
            plen = pc.y;
        } else {
            pc = have ? __ldcg(static_cast<const uint2*>(pieces_v) + idx) : make_uint2(0u, 0u);
            plen = pc.y;
        }
        unsigned incl = plen;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, d);
            if (lane >= (unsigned)d) incl += y;
        }
        const unsigned total = __shfl_sync(kFull, incl, 31);
        const unsigned excl = incl - plen;
        // a task holds at most 32 pieces of at most 32 entries: anything else
        // is a corrupt piece, skipped rather than walked (its lengths' sum
        // could wrap the round counter below)
        if (total > 32u * 32u) continue;
        // entry value of every lane in the round starting at e0 (Z: decoded,
        // `carry` = the previous round's lane-31 value)
        auto fetch = [&](unsigned e0, uint32_t carry) -> uint32_t {
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
            if constexpr (SRC == kSrcZPieces) {
                const unsigned i = e - ex;
                const unsigned hy = __shfl_sync(kFull, pc.y, jx);
                const unsigned i_lane0 = __shfl_sync(kFull, i, 0);  // by every lane
                return z_scan(z_raw(act, i, st, hy, eidx), jx, i_lane0 > 0, carry);
            } else {
                return act ? __ldg(eidx + st + (e - ex)) : 0u;
            }
        };
        // round r's atomics are issued before round r - 1's results are used
        uint32_t x = fetch(0, 0u);
        Round pend;
        for (unsigned e0 = 0; e0 < total; e0 += 32) {
            const bool act = e0 + lane < total;
            const Round cur = round_issue(act ? x >> k : 0xFFFFFFFFu, act, wb);
            uint32_t xn = 0;
            if (e0 + 32 < total) xn = fetch(e0 + 32, __shfl_sync(kFull, x, 31));
            if (e0) round_finish(pend, list, count, stage, staged);
            pend = cur;
            x = xn;
        }
        if (total) round_finish(pend, list, count, stage, staged);
    }
    // long rows: the scan's list (`longs`) holds their vertices and the
    // block's table s_lpre the exclusive prefix of their 32-entry unit
    // counts; unit t of the concatenation goes to warp t mod nw
    const unsigned long long lunits = nlong ? s_lpre[nlong] : 0ull;
    Round lpend;
    for (unsigned long long t = gw; t < lunits; t += nw) {
        unsigned lo = 0, hi = nlong;  // s_lpre[lo] <= t < s_lpre[hi]
        while (hi - lo > 1) {
            const unsigned mid = (lo + hi) >> 1;
            if (s_lpre[mid] <= t) lo = mid;
            else hi = mid;
        }
        const uint32_t u = __ldcg(longs + lo);
        const unsigned q = (unsigned)(t - s_lpre[lo]);
        const uint32_t rb = __ldg(eidx_off + u), len = __ldg(eidx_off + u + 1) - rb;
        const unsigned n_u = min(32u, len - q * 32u);
        const bool act = lane < n_u;
        uint32_t x;
        if constexpr (SRC == kSrcZPieces) {
            const uint2 h = __ldg(zhdr + __ldg(zbo + u) + q);
            x = z_scan(z_raw(act, lane, h.x, h.y, eidx), 0u, false, 0u);
        } else {
            x = act ? __ldg(eidx + rb + q * 32u + lane) : 0u;
        }
        const Round cur = round_issue(act ? x >> k : 0xFFFFFFFFu, act, wb);
        if (t != gw) round_finish(lpend, list, count, stage, staged);
        lpend = cur;
    }
    if (gw < lunits) round_finish(lpend, list, count, stage, staged);
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

// A run's transformation skips the pieces when the frontier is listed
// completely, every row has at most 32 entries (one piece each; the pull
// recorded the longest, in the chunk index) and the plain chunk index serves
// the precision (k >= 0): the scan kernel then expands the listed rows
// itself, up to 32 rows per warp task, and the expansion kernel has nothing
// to do.  Both kernels evaluate this on the same record.
__device__ __forceinline__ bool xform_direct(const XformParams& X, const IterRec* r, const IndexSel& ix,
                                             unsigned long long nw) {
    return X.direct && !ix.z && (int)r->k >= 0 && r->nlist == r->nfront && r->rowmax <= 32u &&
           (unsigned long long)r->nfront <= 32ull * nw;
}

__global__ void __launch_bounds__(kXformThreads) k_xform_scan(const XformParams X) {
    RunCtl* C = X.ctl;
    const uint32_t* bm;
    IterRec* r;
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
    WarpStamp ws;
    ws.start(X);
    if (X.task_ctr && tid == 0) *X.task_ctr = 0u;  // the expansion after this kernel takes tasks from it
    if (X.standalone) {
        bm = X.bm_in;
        r = X.rec;
        const IndexSel ix = select_index(X, X.standalone_k);
        xform_scan_words(bm, X.V, X.bm_words, ix.eoff, piece_out(X, &r->nlong, ix.z), &r->npieces, tid >> 5,
                         nth >> 5);
        ws.stop(X, tid >> 5, 0);
        return;
    }
    if (C->done) return;
    const unsigned it = C->it;
    if (X.trace && blockIdx.x == 0 && threadIdx.x == 0) X.rec[it].t_xf0 = global_timer();
    prepare_iteration(X, it, tid, nth);
    r = X.rec + it;
    if (r->mode == 0) return;
    const IndexSel ix = select_index(X, (int)r->k);
    if (xform_direct(X, r, ix, nth >> 5)) {
        __shared__ uint32_t s_stage[kXformThreads / 32][kAppendStage];
        xform_expand_pieces<kSrcRows>((it & 1) ? X.flist[1] : X.flist[0], r->nfront, ix.shift, ix.ei, X.wb, X.clist,
                                      &X.rec[it].nchunks, tid >> 5, nth >> 5, s_stage[threadIdx.x >> 5], nullptr,
                                      nullptr, 0, ix.eoff);
        return;
    }
    if (r->nlist == r->nfront) {
        xform_scan_list((it & 1) ? X.flist[1] : X.flist[0], r->nfront, ix.eoff, piece_out(X, &r->nlong, ix.z),
                        &r->npieces, tid >> 5, nth >> 5);
        return;
    }
    bm = (it & 1) ? X.bm[1] : X.bm[0];
    xform_scan_words(bm, X.V, X.bm_words, ix.eoff, piece_out(X, &r->nlong, ix.z), &r->npieces, tid >> 5, nth >> 5);
}

__global__ void __launch_bounds__(kXformThreads) k_xform_expand(const XformParams X) {
    RunCtl* C = X.ctl;
    unsigned n;
    int k;
    unsigned* count;
    unsigned it = 0;
    unsigned nlong;
    if (X.standalone) {
        n = __ldcg(&X.rec[0].npieces);
        nlong = __ldcg(&X.rec[0].nlong);
        k = X.standalone_k;
        count = X.count_out;
    } else {
        if (C->done) return;
        it = C->it;
        const IterRec* r = X.rec + it;
        if (r->mode == 0) return;
        if (xform_direct(X, r, select_index(X, (int)r->k), ((unsigned long long)gridDim.x * blockDim.x) >> 5)) {
            if (X.trace && threadIdx.x == 0) atomicMax(&X.rec[it].t_xf1, global_timer());
            return;  // the scan kernel expanded the rows
        }
        n = r->npieces;
        nlong = r->nlong;
        k = (int)r->k;
        count = &X.rec[it].nchunks;
    }
    const IndexSel ix = select_index(X, k);
    if (!X.longs) nlong = 0;
    if (nlong > kLongCap) nlong = kLongCap;
    __shared__ uint32_t s_stage[kXformThreads / 32][kAppendStage];
    // the long rows' table: the exclusive prefix of their unit counts (each
    // thread sums a run of kLongCap / blockDim entries)
    __shared__ uint32_t s_lpre[kLongCap + 1];
    __shared__ uint32_t s_part[kXformThreads / 32];
    if (nlong) {
        constexpr unsigned per = kLongCap / kXformThreads;
        const unsigned r0 = threadIdx.x * per;
        uint32_t sum = 0, cnt[per];
#pragma unroll
        for (unsigned j = 0; j < per; ++j) {
            cnt[j] = 0;
            if (r0 + j < nlong) {
                const uint32_t u = __ldcg(X.longs + r0 + j);
                cnt[j] = (__ldg(ix.eoff + u + 1) - __ldg(ix.eoff + u) + 31u) >> 5;
            }
            sum += cnt[j];
        }
        const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        uint32_t incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, d);
            if (lane >= (unsigned)d) incl += y;
        }
        if (lane == 31) s_part[warp] = incl;
        __syncthreads();
        uint32_t wbase = 0;
        for (unsigned w = 0; w < warp; ++w) wbase += s_part[w];
        uint32_t run = wbase + incl - sum;
#pragma unroll
        for (unsigned j = 0; j < per; ++j) {
            if (r0 + j <= nlong) s_lpre[r0 + j] = run;
            run += cnt[j];
        }
        if (threadIdx.x == kXformThreads - 1 && nlong == kLongCap) s_lpre[kLongCap] = run;
        __syncthreads();
    }
    const unsigned long long gw = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    WarpStamp ws;
    ws.start(X);
    if (ix.z)
        xform_expand_pieces<kSrcZPieces>(X.zpieces, n, ix.shift, X.zwords, X.wb, X.clist, count, gw, nw,
                                  s_stage[threadIdx.x >> 5], X.longs, s_lpre, nlong, ix.eoff, X.zbo, X.zhdr, X.task_ctr);
    else
        xform_expand_pieces<kSrcPieces>(X.pieces, n, ix.shift, ix.ei, X.wb, X.clist, count, gw, nw,
                                   s_stage[threadIdx.x >> 5], X.longs, s_lpre, nlong, ix.eoff, nullptr, nullptr,
                                   X.task_ctr);
    if (X.standalone) ws.stop(X, gw, 1);
    if (X.trace && !X.standalone) {
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
    const IndexSel ix = select_index(X, X.standalone_k);
    const unsigned k = ix.shift;
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
                const uint32_t rb = __ldg(ix.eoff + u), re = __ldg(ix.eoff + u + 1);
                for (uint32_t e0 = rb; e0 < re; e0 += 32) {
                    const uint32_t e = e0 + lane;
                    bool fresh = false;
                    uint32_t b = 0;
                    if (e < re) {
                        b = __ldg(ix.ei + e) >> k;
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

}  // namespace wedge

// Graph object: validation, upload, and the device-side build of the per-chunk
// metadata and of the edge index (Sections 3.3 and 4: a CSR keyed by source
// whose entries are Wedge Frontier positions).  Runs once per graph, off the
// timed path.
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace wedge {

// ------------------------------------------------------------------------
// Exclusive scan of uint32 (device, multi-level reduce-then-scan)
// ------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* total) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t block_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t s = (lane < nw) ? warp_sums[lane] : 0;
        uint32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, si, o);
            if (lane >= o) si += y;
        }
        warp_sums[lane] = si - s;
        if (lane == 31) block_total = si;
    }
    __syncthreads();
    const uint32_t base = warp_sums[warp];
    *total = block_total;
    __syncthreads();
    return base + incl - x;
}

// Scans n + 1 items (item n is 0), writing out[0..n]; per-block totals to sums.
__global__ void k_scan_tiles(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, uint64_t n,
                             uint32_t* __restrict__ sums) {
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t local = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        uint64_t idx = base + i;
        v[i] = (idx < n) ? in[idx] : 0u;
        local += v[i];
    }
    uint32_t total;
    uint32_t pre = block_exclusive_scan(local, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        uint64_t idx = base + i;
        if (idx <= n) out[idx] = pre;
        pre += v[i];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, uint64_t n, const uint32_t* __restrict__ offs) {
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    const uint32_t add = offs[blockIdx.x];
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        uint64_t idx = base + i;
        if (idx <= n) out[idx] += add;
    }
}

static wedge_status scan_rec(const uint32_t* in, uint32_t* out, uint64_t n, cudaStream_t s) {
    const uint64_t items = n + 1;
    const uint64_t nb = (items + kScanTile - 1) / kScanTile;
    uint32_t* sums = nullptr;
    uint32_t* offs = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&sums, nb * 4));
    WEDGE_TRY(dev_alloc(nullptr, (void**)&offs, (nb + 1) * 4));
    k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
    count_launch();
    wedge_status st = WEDGE_OK;
    if (nb > 1) {
        st = scan_rec(sums, offs, nb, s);
        if (st == WEDGE_OK) {
            k_scan_add<<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, offs);
            count_launch();
        }
    }
    cudaError_t e = cudaGetLastError();
    dev_free_async(sums, s);  // stream-ordered: after the kernels above
    dev_free_async(offs, s);
    if (e != cudaSuccess) return cuda_error(e, "scan launch");
    return st;
}

wedge_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t*, cudaStream_t s) {
    return scan_rec(in, out, n, s);
}

size_t scan_tmp_words(uint64_t) { return 0; }

// ------------------------------------------------------------------------
// Build kernels
// ------------------------------------------------------------------------
__global__ void k_outdeg(const uint32_t* __restrict__ src, uint64_t E, uint32_t* __restrict__ outdeg) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < E;
         p += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&outdeg[src[p]], 1u);
}

__global__ void k_nz_flags(const uint32_t* __restrict__ off, uint32_t V, uint32_t* __restrict__ flag) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V;
         v += (uint64_t)gridDim.x * blockDim.x)
        flag[v] = off[v + 1] > off[v] ? 1u : 0u;
}

// vid, head bits and the destination index of each chunk's first position.
__global__ void k_chunk_meta(const uint32_t* __restrict__ off, uint32_t V, const uint32_t* __restrict__ knz,
                             uint32_t* __restrict__ vid, uint2* __restrict__ cmeta,
                             uint32_t* __restrict__ split_bm) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t b = off[v], e = off[v + 1];
        if (e == b) continue;
        const uint32_t k = knz[v];
        vid[k] = (uint32_t)v;
        atomicOr(&cmeta[b >> 5].x, 1u << (b & 31));
        for (uint32_t c = (b + 31) >> 5; c <= (e - 1) >> 5; ++c) cmeta[c].y = k;
        if ((b >> kSliceShift) != ((e - 1) >> kSliceShift)) atomicOr(&split_bm[v >> 5], 1u << (v & 31));
    }
}

// One warp per chunk: the sources that appear in the chunk, each counted once
// (__match_any_sync groups equal sources; the lowest lane of a group keeps it).
// COUNT: one 64-bit atomic per distinct source and chunk adds the row entry
// (low word) and the group's size, the source's edges in the chunk (high
// word: its out-degree once summed); row entries stay below NC < 2^32.
// Otherwise the group's lane appends the chunk to the source's row at the
// row's cursor.
template <bool COUNT>
__global__ void k_eidx_pass(const uint32_t* __restrict__ src, uint64_t E, uint64_t NC,
                            unsigned long long* __restrict__ counts, uint32_t* __restrict__ cursor,
                            uint32_t* __restrict__ eidx) {
    const unsigned lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c = warp; c < NC; c += nwarps) {
        const uint64_t p = c * 32 + lane;
        const bool valid = p < E;
        const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid);
        if (!valid) continue;
        const uint32_t s = src[p];
        const unsigned same = __match_any_sync(vmask, s);
        if ((unsigned)(__ffs(same) - 1) != lane) continue;
        if (COUNT) {
            atomicAdd(&counts[s], ((unsigned long long)__popc(same) << 32) | 1ull);
        } else {
            const uint32_t pos = atomicAdd(&cursor[s], 1u);
            eidx[pos] = (uint32_t)c;
        }
    }
}

// The edge index at the paper's finer precisions (Section 3.4, "Frontier
// Precision"): row u lists, once each, the 8-edge units (position >> 3)
// holding u's out-edges.  One warp per 32 positions (four units); the
// sources of each unit are made distinct with __match_any_sync on (source,
// unit).  COUNT: one atomic per distinct source and unit on its row length;
// otherwise the unit is appended to the row at the row's cursor.
template <bool COUNT>
__global__ void k_eidx8_pass(const uint32_t* __restrict__ src, uint64_t E, uint64_t NC, uint32_t* __restrict__ cnt,
                             uint32_t* __restrict__ eidx8) {
    const unsigned lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c = warp; c < NC; c += nwarps) {
        const uint64_t p = c * 32 + lane;
        const bool valid = p < E;
        const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid);
        if (!valid) continue;
        const uint32_t s = src[p];
        const unsigned same = __match_any_sync(vmask, ((unsigned long long)s << 2) | (lane >> 3));
        if ((unsigned)(__ffs(same) - 1) != lane) continue;
        if (COUNT) {
            atomicAdd(&cnt[s], 1u);
        } else {
            const uint32_t pos = atomicAdd(&cnt[s], 1u);
            eidx8[pos] = (uint32_t)(p >> 3);
        }
    }
}

// Row lengths (low words) and out-degrees (high words) of the count pass.
__global__ void k_split_counts(const unsigned long long* __restrict__ counts, uint32_t V,
                               uint32_t* __restrict__ rowlen, uint32_t* __restrict__ outdeg) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long c = counts[v];
        rowlen[v] = (uint32_t)c;
        outdeg[v] = (uint32_t)(c >> 32);
    }
}

// Metadata past the last chunk reads as "a new destination starts here".
__global__ void k_meta_pad(uint2* __restrict__ cmeta, uint64_t NC, uint64_t len) {
    for (uint64_t c = NC + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < len;
         c += (uint64_t)gridDim.x * blockDim.x)
        cmeta[c] = make_uint2(1u, 0u);
}

__global__ void k_pieces_total(const uint32_t* __restrict__ rowlen, uint32_t V,
                               unsigned long long* __restrict__ total) {
    unsigned long long local = 0;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V;
         v += (uint64_t)gridDim.x * blockDim.x)
        local += (rowlen[v] + 31u) >> 5;
    for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xFFFFFFFFu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(total, local);
}

__global__ void k_max_u32(const uint32_t* __restrict__ a, uint32_t n, unsigned* __restrict__ out) {
    unsigned m = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, a[i]);
    for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_down_sync(0xFFFFFFFFu, m, d));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__global__ void k_rowlen_from_off(const uint32_t* __restrict__ eoff, uint32_t V, uint32_t* __restrict__ rowlen) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V;
         v += (uint64_t)gridDim.x * blockDim.x)
        rowlen[v] = eoff[v + 1] - eoff[v];
}

// Input checks: offsets non-decreasing, sources < V, and for a caller's edge
// index: offsets non-decreasing and entries < NC.  Any violation sets a bit
// in *bad so that creation fails with INVALID_ARG before a kernel indexes
// with the bad value.
__global__ void k_validate(const uint32_t* __restrict__ off, const uint32_t* __restrict__ src, uint32_t V,
                           uint64_t E, const uint32_t* __restrict__ eoff, const uint32_t* __restrict__ eidx,
                           uint64_t elen, uint64_t NC, unsigned* bad) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    unsigned flag = 0;
    for (uint64_t v = tid; v < V; v += nth) {
        if (off[v] > off[v + 1]) flag |= 1u;
        if (eoff && eoff[v] > eoff[v + 1]) flag |= 4u;
    }
    // src is 16-byte aligned (checked on entry): four sources per load
    const uint4* src4 = reinterpret_cast<const uint4*>(src);
    for (uint64_t q = tid; q < E / 4; q += nth) {
        const uint4 x = src4[q];
        if (x.x >= V || x.y >= V || x.z >= V || x.w >= V) flag |= 2u;
    }
    for (uint64_t p = (E & ~3ull) + tid; p < E; p += nth)
        if (src[p] >= V) flag |= 2u;
    for (uint64_t i = tid; eidx && i < elen; i += nth)
        if (eidx[i] >= NC) flag |= 8u;
    if (flag) atomicOr(bad, flag);
}

// Out-edges of the push/pull hybrid: every in-edge position p (destination
// from the chunk's head mask and vid, as in the pull) is appended to its
// source's CSR row; one atomic per distinct source and warp.
__global__ void k_csr_fill(const uint32_t* __restrict__ src, const uint32_t* __restrict__ w, uint64_t E,
                           uint64_t NC, const uint2* __restrict__ cmeta, const uint32_t* __restrict__ vid,
                           uint32_t* __restrict__ cursor, uint32_t* __restrict__ dst_out,
                           uint32_t* __restrict__ src_out, uint32_t* __restrict__ w_out) {
    const unsigned lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; c < NC; c += nw) {
        const uint64_t p = c * 32 + lane;
        const bool valid = p < E;
        const uint32_t u = valid ? src[p] : 0xFFFFFFFFu;
        const uint2 meta = cmeta[c];
        const uint32_t kid = meta.y + __popc(meta.x & ((2u << lane) - 1u) & ~1u);
        const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
        const unsigned same = __match_any_sync(0xFFFFFFFFu, u) & vm;
        if (!valid) continue;
        const unsigned leader = __ffs(same) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&cursor[u], (unsigned)__popc(same));
        base = __shfl_sync(same, base, leader);
        const uint32_t pos = base + __popc(same & ((1u << lane) - 1u));
        dst_out[pos] = vid[kid];
        src_out[pos] = u;
        if (w_out) w_out[pos] = w[p];
    }
}

__global__ void k_kid_of(const uint32_t* __restrict__ vid, uint32_t NZ, uint32_t* __restrict__ kid_of) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < NZ; i += (uint64_t)gridDim.x * blockDim.x)
        kid_of[vid[i]] = (uint32_t)i;
}

static unsigned grid_for(uint64_t n, int threads, int sms) {
    uint64_t b = (n + threads - 1) / threads;
    uint64_t cap = (uint64_t)sms * 32;
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

static wedge_status upload(wedge_graph* g, const uint32_t* p, uint64_t n, uint32_t** own,
                           const uint32_t** use, cudaStream_t s, const char* name, bool need_align) {
    if (n == 0) {
        WEDGE_TRY(dev_alloc(g, (void**)own, 16));
        *use = *own;
        return WEDGE_OK;
    }
    if (!p) return set_error(WEDGE_ERR_INVALID_ARG, std::string(name) + " is NULL");
    PtrKind k = classify(p);
    if (k == PtrKind::Device) {
        if (need_align && (reinterpret_cast<uintptr_t>(p) & 15))
            return set_error(WEDGE_ERR_INVALID_ARG, std::string(name) + " must be 16-byte aligned");
        *use = p;
        return WEDGE_OK;
    }
    WEDGE_TRY(dev_alloc(g, (void**)own, n * 4));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(*own, p, n * 4, cudaMemcpyHostToDevice, s));
    *use = *own;
    return WEDGE_OK;
}

static void free_graph(wedge_graph* g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    dev_free(g->off_own);
    dev_free(g->src_own);
    dev_free(g->w_own);
    dev_free(g->outdeg);
    dev_free(g->csr_off);
    dev_free(g->csr_dst);
    dev_free(g->csr_src);
    dev_free(g->csr_w);
    dev_free(g->kid_of);
    dev_free(g->push_pieces);
    dev_free(g->vid);
    dev_free(g->cmeta);
    if (g->eidx_off_owned) dev_free(g->eidx_off);
    if (g->eidx_owned) dev_free(g->eidx);
    dev_free(g->vals);
    dev_free(g->vals_sync);
    dev_free(g->bm[0]);
    dev_free(g->bm[1]);
    dev_free(g->wb);
    dev_free(g->clist);
    dev_free(g->pieces);
    dev_free(g->longs);
    dev_free(g->xf_task);
    dev_free(g->flist[0]);
    dev_free(g->flist[1]);
    dev_free(g->visk);
    dev_free(g->bstat);
    dev_free(g->rec);
    dev_free(g->ctl);
    pinned_small_free(g->h_ctl);
    dev_free(g->contrib);
    dev_free(g->pr_perm);
    dev_free(g->pr_src);
    dev_free(g->acc);
    dev_free(g->rank);
    dev_free(g->split_bm);
    dev_free(g->mlp_bf16);
    dev_free(g->snap_vals);
    dev_free(g->snap_visk);
    dev_free(g->ms_fb[0]);
    dev_free(g->ms_fb[1]);
    dev_free(g->ms_seen);
    dev_free(g->ms_roots);
    dev_free(g->ms_bar);
    dev_free(g->slice_ctr);
    dev_free(g->zhdr);
    dev_free(g->eidx8);
    dev_free(g->eidx8_off);
    dev_free(g->zwords);
    dev_free(g->zbo);
    dev_free(g->zpieces);
    if (g->ms_exec) cudaGraphExecDestroy(g->ms_exec);
    for (auto& e : g->loop_exec)
        if (e) cudaGraphExecDestroy(e);
    for (auto& e : g->loop_exec_push)
        if (e) cudaGraphExecDestroy(e);
    if (g->pr_exec) cudaGraphExecDestroy(g->pr_exec);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
}

static wedge_status validate(wedge_graph* g, cudaStream_t s) {
    unsigned* d_bad = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&d_bad, 4));
    unsigned bad = 0;
    cudaError_t e = cudaMemsetAsync(d_bad, 0, 4, s);
    if (e == cudaSuccess) {
        const bool user_index = !g->eidx_off_owned || !g->eidx_owned;
        k_validate<<<grid_for(g->E > g->V ? g->E : g->V, 256, g->num_sms), 256, 0, s>>>(
            g->off, g->src, g->V, g->E, user_index ? g->eidx_off : nullptr, user_index ? g->eidx : nullptr,
            user_index ? g->eidx_len : 0, g->NC, d_bad);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free_async(d_bad, s);
    if (e != cudaSuccess) return cuda_error(e, "validation");
    if (bad & 1u) return set_error(WEDGE_ERR_INVALID_ARG, "offsets must be non-decreasing");
    if (bad & 2u) return set_error(WEDGE_ERR_INVALID_ARG, "a source id is >= V");
    if (bad & 4u) return set_error(WEDGE_ERR_INVALID_ARG, "edge index offsets must be non-decreasing");
    if (bad & 8u) return set_error(WEDGE_ERR_INVALID_ARG, "an edge index entry is >= ceil(E/32)");
    return WEDGE_OK;
}

static wedge_status build(wedge_graph* g, const uint32_t* user_eoff, const uint32_t* user_eidx, cudaStream_t s) {
    const uint32_t V = g->V;
    const uint64_t E = g->E, NC = g->NC;
    const int sms = g->num_sms;
    uint32_t* tmp = nullptr;   // V+1 words of scratch
    WEDGE_TRY(dev_alloc(nullptr, (void**)&tmp, ((uint64_t)V + 1) * 4));
    struct Free {
        uint32_t* p;
        cudaStream_t s;
        ~Free() { dev_free_async(p, s); }
    } free_tmp{tmp, s};

    WEDGE_TRY(validate(g, s));  // CSC only: no index yet
    WEDGE_TRY(dev_alloc(g, (void**)&g->outdeg, (uint64_t)V * 4));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->outdeg, 0, (uint64_t)V * 4, s));
    if (E && user_eoff) {  // otherwise the edge-index counting pass counts them
        k_outdeg<<<grid_for(E, 256, sms), 256, 0, s>>>(g->src, E, g->outdeg);
        count_launch();
    }

    // vertices with in-degree > 0 and their order
    uint32_t* knz = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&knz, ((uint64_t)V + 1) * 4));
    struct Free2 {
        uint32_t* p;
        cudaStream_t s;
        ~Free2() { dev_free_async(p, s); }
    } free_knz{knz, s};
    k_nz_flags<<<grid_for(V, 256, sms), 256, 0, s>>>(g->off, V, tmp);
    count_launch();
    WEDGE_TRY(exclusive_scan_u32(tmp, knz, V, nullptr, s));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(&g->NZ, knz + V, 4, cudaMemcpyDeviceToHost, s));
    WEDGE_TRY_CUDA(cudaStreamSynchronize(s));

    WEDGE_TRY(dev_alloc(g, (void**)&g->vid, (uint64_t)(g->NZ ? g->NZ : 1) * 4));
    g->meta_len = (NC + kTileC - 1) / kTileC * kTileC + kTileC + kMetaPad;
    WEDGE_TRY(dev_alloc(g, (void**)&g->cmeta, g->meta_len * sizeof(uint2)));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->cmeta, 0, g->meta_len * sizeof(uint2), s));
    k_meta_pad<<<grid_for(g->meta_len - NC, 256, sms), 256, 0, s>>>(g->cmeta, NC, g->meta_len);
    count_launch();
    const uint64_t bm_words = ((uint64_t)V + 31) / 32;
    WEDGE_TRY(dev_alloc(g, (void**)&g->split_bm, bm_words * 4));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->split_bm, 0, bm_words * 4, s));
    k_chunk_meta<<<grid_for(V, 256, sms), 256, 0, s>>>(g->off, V, knz, g->vid, g->cmeta, g->split_bm);
    count_launch();

    // edge index
    if (user_eoff) {
        PtrKind k = classify(user_eoff);
        if (k == PtrKind::Device) {
            g->eidx_off = const_cast<uint32_t*>(user_eoff);
        } else {
            g->eidx_off_owned = true;
            WEDGE_TRY(dev_alloc(g, (void**)&g->eidx_off, ((uint64_t)V + 1) * 4));
            WEDGE_TRY_CUDA(
                cudaMemcpyAsync(g->eidx_off, user_eoff, ((uint64_t)V + 1) * 4, cudaMemcpyHostToDevice, s));
        }
        uint32_t len = 0;
        WEDGE_TRY_CUDA(cudaMemcpyAsync(&len, g->eidx_off + V, 4, cudaMemcpyDeviceToHost, s));
        WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
        g->eidx_len = len;
        if (len > E) return set_error(WEDGE_ERR_INVALID_ARG, "edge index longer than E");
        if (len && !user_eidx) return set_error(WEDGE_ERR_INVALID_ARG, "eidx is NULL");
        if (len) {
            if (classify(user_eidx) == PtrKind::Device) {
                g->eidx = const_cast<uint32_t*>(user_eidx);
            } else {
                WEDGE_TRY(dev_alloc(g, (void**)&g->eidx, (uint64_t)len * 4));
                WEDGE_TRY_CUDA(cudaMemcpyAsync(g->eidx, user_eidx, (uint64_t)len * 4, cudaMemcpyHostToDevice, s));
                g->eidx_owned = true;
            }
        } else {
            WEDGE_TRY(dev_alloc(g, (void**)&g->eidx, 16));
        }
        // eidx_off came from the caller: only free what we allocated
        {
            const bool o1 = g->eidx_off_owned, o2 = g->eidx_owned;
            g->eidx_off_owned = false;  // tells validate() to check the caller's index
            wedge_status vs = validate(g, s);
            g->eidx_off_owned = o1;
            g->eidx_owned = o2;
            WEDGE_TRY(vs);
        }
        k_rowlen_from_off<<<grid_for(V, 256, sms), 256, 0, s>>>(g->eidx_off, V, tmp);
        count_launch();
    } else {
        g->eidx_owned = true;
        g->eidx_off_owned = true;
        WEDGE_TRY(dev_alloc(g, (void**)&g->eidx_off, ((uint64_t)V + 1) * 4));
        WEDGE_TRY_CUDA(cudaMemsetAsync(tmp, 0, ((uint64_t)V + 1) * 4, s));
        const unsigned eg = grid_for(NC * 32, 256, sms);
        if (NC) {
            unsigned long long* counts = nullptr;
            WEDGE_TRY(dev_alloc(nullptr, (void**)&counts, (uint64_t)V * 8));
            cudaError_t e = cudaMemsetAsync(counts, 0, (uint64_t)V * 8, s);
            if (e == cudaSuccess) {
                k_eidx_pass<true><<<eg, 256, 0, s>>>(g->src, E, NC, counts, nullptr, nullptr);
                k_split_counts<<<grid_for(V, 256, sms), 256, 0, s>>>(counts, V, tmp, g->outdeg);
                count_launch(2);
                e = cudaGetLastError();
            }
            dev_free_async(counts, s);
            if (e != cudaSuccess) return cuda_error(e, "edge index count");
        }
        WEDGE_TRY(exclusive_scan_u32(tmp, g->eidx_off, V, nullptr, s));
        uint32_t len = 0;
        WEDGE_TRY_CUDA(cudaMemcpyAsync(&len, g->eidx_off + V, 4, cudaMemcpyDeviceToHost, s));
        WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
        g->eidx_len = len;
        WEDGE_TRY(dev_alloc(g, (void**)&g->eidx, (uint64_t)(len ? len : 1) * 4));
        // cursor = eidx_off; fill rows
        WEDGE_TRY_CUDA(cudaMemcpyAsync(knz, g->eidx_off, ((uint64_t)V + 1) * 4, cudaMemcpyDeviceToDevice, s));
        if (NC) {
            k_eidx_pass<false><<<eg, 256, 0, s>>>(g->src, E, NC, nullptr, knz, g->eidx);
            count_launch();
        }
    }
    // largest out-degree (a statistic of the learned switch's features)
    {
        unsigned* d_max = nullptr;
        WEDGE_TRY(dev_alloc(nullptr, (void**)&d_max, 4));
        cudaError_t e = cudaMemsetAsync(d_max, 0, 4, s);
        if (e == cudaSuccess) {
            k_max_u32<<<grid_for(V, 256, sms), 256, 0, s>>>(g->outdeg, V, d_max);
            count_launch();
            e = cudaMemcpyAsync(&g->max_outdeg, d_max, 4, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        dev_free_async(d_max, s);
        if (e != cudaSuccess) return cuda_error(e, "max out-degree");
    }
    // work pieces bound: sum ceil(|row| / 32); and sum ceil(outdeg / 32),
    // which also bounds the pieces of the 8-edge-unit index (a row there
    // lists at most one unit per out-edge)
    unsigned long long* d_total = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&d_total, 16));
    WEDGE_TRY_CUDA(cudaMemsetAsync(d_total, 0, 16, s));
    k_pieces_total<<<grid_for(V, 256, sms), 256, 0, s>>>(tmp, V, d_total);
    k_pieces_total<<<grid_for(V, 256, sms), 256, 0, s>>>(g->outdeg, V, d_total + 1);
    count_launch(2);
    unsigned long long total[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(total, d_total, 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free_async(d_total, s);
    if (e != cudaSuccess) return cuda_error(e, "edge index build");
    g->npieces_max = total[0];
    g->npieces_outdeg_bound = total[1];
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

// The 8-edge-unit edge index, built on the first run or transformation at
// a finer precision than one 32-edge chunk.
wedge_status build_eidx8(wedge_graph* g, cudaStream_t s) {
    if (g->eidx8) return WEDGE_OK;
    const uint32_t V = g->V;
    const uint64_t E = g->E, NC = g->NC;
    const int sms = g->num_sms;
    uint32_t* cnt = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&cnt, ((uint64_t)V + 1) * 4));
    struct Free {
        uint32_t* p;
        cudaStream_t s;
        ~Free() { dev_free_async(p, s); }
    } free_cnt{cnt, s};
    WEDGE_TRY(dev_alloc(g, (void**)&g->eidx8_off, ((uint64_t)V + 1) * 4));
    WEDGE_TRY_CUDA(cudaMemsetAsync(cnt, 0, ((uint64_t)V + 1) * 4, s));
    const unsigned eg = grid_for(NC * 32, 256, sms);
    if (NC) {
        k_eidx8_pass<true><<<eg, 256, 0, s>>>(g->src, E, NC, cnt, nullptr);
        count_launch();
    }
    WEDGE_TRY(exclusive_scan_u32(cnt, g->eidx8_off, V, nullptr, s));
    uint32_t len = 0;
    WEDGE_TRY_CUDA(cudaMemcpyAsync(&len, g->eidx8_off + V, 4, cudaMemcpyDeviceToHost, s));
    WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    WEDGE_TRY(dev_alloc(g, (void**)&g->eidx8, (uint64_t)(len ? len : 1) * 4));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(cnt, g->eidx8_off, ((uint64_t)V + 1) * 4, cudaMemcpyDeviceToDevice, s));
    if (NC) {
        k_eidx8_pass<false><<<eg, 256, 0, s>>>(g->src, E, NC, cnt, g->eidx8);
        count_launch();
    }
    // work pieces bound: sum ceil(|row| / 32)
    k_rowlen_from_off<<<grid_for(V, 256, sms), 256, 0, s>>>(g->eidx8_off, V, cnt);
    unsigned long long* d_total = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&d_total, 8));
    WEDGE_TRY_CUDA(cudaMemsetAsync(d_total, 0, 8, s));
    k_pieces_total<<<grid_for(V, 256, sms), 256, 0, s>>>(cnt, V, d_total);
    count_launch(2);
    unsigned long long total = 0;
    cudaError_t e = cudaMemcpyAsync(&total, d_total, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free_async(d_total, s);
    if (e != cudaSuccess) return cuda_error(e, "8-edge edge index build");
    g->eidx8_len = len;
    g->npieces8_max = total;
    return WEDGE_OK;
}

wedge_status build_csr(wedge_graph* g, cudaStream_t s) {
    if (g->csr_off) return WEDGE_OK;
    const uint32_t V = g->V;
    const uint64_t E = g->E;
    const int sms = g->num_sms;
    uint32_t* cursor = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&cursor, ((uint64_t)V + 1) * 4));
    struct Free {
        uint32_t* p;
        cudaStream_t s;
        ~Free() { dev_free_async(p, s); }
    } free_cursor{cursor, s};
    uint32_t* off = nullptr;
    WEDGE_TRY(dev_alloc(g, (void**)&off, ((uint64_t)V + 1) * 4));
    wedge_status st = exclusive_scan_u32(g->outdeg, off, V, nullptr, s);
    if (st == WEDGE_OK) st = dev_alloc(g, (void**)&g->csr_dst, (E ? E : 1) * 4);
    if (st == WEDGE_OK) st = dev_alloc(g, (void**)&g->csr_src, (E ? E : 1) * 4);
    if (st == WEDGE_OK && g->w) st = dev_alloc(g, (void**)&g->csr_w, (E ? E : 1) * 4);
    if (st == WEDGE_OK) st = dev_alloc(g, (void**)&g->kid_of, (uint64_t)V * 4);
    unsigned long long* d_total = nullptr;
    if (st == WEDGE_OK) st = dev_alloc(nullptr, (void**)&d_total, 8);
    if (st != WEDGE_OK) {
        dev_free_async(off, s);
        return st;
    }
    g->csr_off = off;  // from here on freed with the graph
    cudaError_t e = cudaMemcpyAsync(cursor, off, ((uint64_t)V + 1) * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_total, 0, 8, s);
    if (e == cudaSuccess) {
        if (g->NC)
            k_csr_fill<<<grid_for(g->NC * 32, 256, sms), 256, 0, s>>>(g->src, g->w, E, g->NC, g->cmeta, g->vid, cursor,
                                                                     g->csr_dst, g->csr_src, g->csr_w);
        if (g->NZ) k_kid_of<<<grid_for(g->NZ, 256, sms), 256, 0, s>>>(g->vid, g->NZ, g->kid_of);
        k_pieces_total<<<grid_for(V, 256, sms), 256, 0, s>>>(g->outdeg, V, d_total);
        count_launch(3);
        unsigned long long total = 0;
        e = cudaMemcpyAsync(&total, d_total, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        g->npieces_push_max = total;
    }
    dev_free_async(d_total, s);
    if (e != cudaSuccess) return cuda_error(e, "out-edge CSR build");
    WEDGE_TRY(dev_alloc(g, (void**)&g->push_pieces, (g->npieces_push_max ? g->npieces_push_max : 1) * sizeof(uint2)));
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

}  // namespace wedge

using namespace wedge;

extern "C" {

wedge_status wedge_graph_create(uint32_t V, uint64_t E, const uint32_t* d_offsets, const uint32_t* d_src,
                                const uint32_t* d_w, const uint32_t* d_eidx_off, const uint32_t* d_eidx,
                                uint32_t chunk_edges, wedge_stream_t stream, wedge_graph_t* out) {
    if (!out) return set_error(WEDGE_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (V == 0) return set_error(WEDGE_ERR_INVALID_ARG, "V must be >= 1");
    if (E >= 0xFFFFFF00ull) return set_error(WEDGE_ERR_INVALID_ARG, "E must be < 2^32 - 256");
    if (chunk_edges != kChunk) return set_error(WEDGE_ERR_INVALID_ARG, "chunk_edges must be 32");
    if (!d_offsets) return set_error(WEDGE_ERR_INVALID_ARG, "offsets is NULL");
    if (!d_eidx_off && d_eidx) return set_error(WEDGE_ERR_INVALID_ARG, "eidx given without eidx_off");
    cudaStream_t s = (cudaStream_t)stream;
    wedge_graph* g = new wedge_graph();
    cudaGetDevice(&g->device);
    int sms = 0, smem = 0;  // two attributes: far cheaper than the whole property set
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, g->device);
    if (e != cudaSuccess) {
        delete g;
        return cuda_error(e, "cudaDeviceGetAttribute");
    }
    g->num_sms = sms;
    g->smem_per_sm = (size_t)smem;
    g->V = V;
    g->E = E;
    g->NC = (E + kChunk - 1) / kChunk;
    wedge_status st = upload(g, d_offsets, (uint64_t)V + 1, &g->off_own, &g->off, s, "offsets", false);
    if (st == WEDGE_OK) st = upload(g, d_src, E, &g->src_own, &g->src, s, "src", true);
    if (st == WEDGE_OK && d_w) st = upload(g, d_w, E, &g->w_own, &g->w, s, "w", true);
    if (st == WEDGE_OK) {
        // the offsets must describe E edges
        uint32_t first = 1, last = 0;
        cudaError_t e1 = cudaMemcpyAsync(&first, g->off, 4, cudaMemcpyDeviceToHost, s);
        cudaError_t e2 = cudaMemcpyAsync(&last, g->off + V, 4, cudaMemcpyDeviceToHost, s);
        cudaError_t e3 = cudaStreamSynchronize(s);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
            st = cuda_error(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "offsets readback");
        else if (first != 0 || last != E)
            st = set_error(WEDGE_ERR_INVALID_ARG, "offsets[0] must be 0 and offsets[V] must be E");
    }
    if (st == WEDGE_OK) st = build(g, d_eidx_off, d_eidx, s);
    if (st == WEDGE_OK) st = ensure_run_scratch(g, s);
    if (st == WEDGE_OK) {  // ready for runs on any stream
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(e, "graph creation");
    }
    if (st != WEDGE_OK) {
        free_graph(g);
        return st;
    }
    *out = g;
    return WEDGE_OK;
}

wedge_status wedge_graph_destroy(wedge_graph_t g) {
    if (!g) return set_error(WEDGE_ERR_INVALID_ARG, "graph is NULL");
    free_graph(g);
    return WEDGE_OK;
}

wedge_status wedge_graph_get_info(wedge_graph_t g, wedge_graph_info* out) {
    if (!g || !out) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    out->V = g->V;
    out->nz_dst = g->NZ;
    out->E = g->E;
    out->nchunks = g->NC;
    out->eidx_len = g->eidx_len;
    out->device_bytes = g->device_bytes;
    out->device = g->device;
    out->eidx_bytes = ((uint64_t)g->V + 1) * 4 + g->eidx_len * 4;
    out->eidx_z_bytes = g->zpieces ? g->z_bytes : 0;
    out->eidx_z_blocks = g->zpieces ? g->zblocks : 0;
    out->eidx_z_words = g->zpieces ? g->zwords_len : 0;
    return WEDGE_OK;
}

wedge_status wedge_graph_copy_edge_index_z(wedge_graph_t g, uint32_t* d_zbo, uint32_t* d_zhdr, uint32_t* d_zwords,
                                           wedge_stream_t stream) {
    if (!g || !d_zbo || !d_zhdr || !d_zwords) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (!g->zpieces) return set_error(WEDGE_ERR_INVALID_ARG, "the compressed edge index is not built");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    WEDGE_TRY_CUDA(cudaMemcpyAsync(d_zbo, g->zbo, ((uint64_t)g->V + 1) * 4, cudaMemcpyDeviceToDevice, s));
    if (g->zblocks)
        WEDGE_TRY_CUDA(cudaMemcpyAsync(d_zhdr, g->zhdr, g->zblocks * sizeof(uint2), cudaMemcpyDeviceToDevice, s));
    if (g->zwords_len)
        WEDGE_TRY_CUDA(cudaMemcpyAsync(d_zwords, g->zwords, g->zwords_len * 4, cudaMemcpyDeviceToDevice, s));
    return WEDGE_OK;
}

wedge_status wedge_graph_copy_edge_index(wedge_graph_t g, uint32_t* d_eidx_off, uint32_t* d_eidx,
                                         wedge_stream_t stream) {
    if (!g || !d_eidx_off || (!d_eidx && g->eidx_len)) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(g->device);
    cudaStream_t s = (cudaStream_t)stream;
    WEDGE_TRY_CUDA(cudaMemcpyAsync(d_eidx_off, g->eidx_off, ((uint64_t)g->V + 1) * 4, cudaMemcpyDefault, s));
    if (g->eidx_len)
        WEDGE_TRY_CUDA(cudaMemcpyAsync(d_eidx, g->eidx, g->eidx_len * 4, cudaMemcpyDefault, s));
    return WEDGE_OK;
}

}  // extern "C"

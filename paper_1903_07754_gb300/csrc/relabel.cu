// Degree-ordered relabelling of a CSC graph (not in the paper: a locality
// step before graph creation).  The pulls gather one value per in-edge,
// indexed by the edge's source; when the sources with the most out-edges
// get the smallest ids their values share cache lines, so more of the
// gathers hit L1 and L2.  New ids follow descending out-degree, ties by
// ascending old id; every destination keeps its in-edges in their original
// order with the sources renamed.  Results of runs on the relabelled graph
// are brought back to the original ids with wedge_permute_rows (levels,
// distances, ranks, batched rows) and wedge_cc_labels_to_original
// (component labels, which name the smallest member id).
#include <initializer_list>

#include "common.cuh"

namespace wedge {

wedge_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* tkeys, uint32_t* tvals, uint64_t n,
                              int key_bits, int num_sms, cudaStream_t s, bool* in_tmp);

namespace {

constexpr unsigned kPieceEdges = 1024;  // in-edges copied by one warp task
constexpr uint32_t kPrHubDegree = 1;     // PageRank's order ranks vertices of at least this out-degree

unsigned grid_of(uint64_t n, int threads, int sms) {
    const uint64_t b = (n + threads - 1) / threads;
    const uint64_t cap = (uint64_t)sms * 8;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

// Offsets non-decreasing and sources < V (flag bits 1 and 2); out-degrees
// counted for the valid sources.
__global__ void k_rl_check_count(const uint32_t* __restrict__ off, const uint32_t* __restrict__ src, uint32_t V,
                                 uint64_t E, uint32_t* __restrict__ deg, unsigned* bad) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    unsigned flag = 0;
    for (uint64_t v = tid; v < V; v += nth)
        if (off[v] > off[v + 1]) flag |= 1u;
    for (uint64_t p = tid; p < E; p += nth) {
        const uint32_t u = src[p];
        if (u < V) atomicAdd(deg + u, 1u);
        else flag |= 2u;
    }
    if (flag) atomicOr(bad, flag);
}

// Sort keys: ascending key = descending out-degree; values: old ids.
__global__ void k_rl_keys(const uint32_t* __restrict__ deg, uint32_t V, uint32_t kmax, uint32_t* __restrict__ key,
                          uint32_t* __restrict__ val) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
        key[v] = kmax - deg[v];
        val[v] = (uint32_t)v;
    }
}

// new_of_old, the new in-degrees and each new vertex's copy-task count.
__global__ void k_rl_place(const uint32_t* __restrict__ old_of_new, const uint32_t* __restrict__ off, uint32_t V,
                           uint32_t* __restrict__ new_of_old, uint32_t* __restrict__ indeg,
                           uint32_t* __restrict__ ntask) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < V; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t o = old_of_new[i];
        new_of_old[o] = (uint32_t)i;
        const uint32_t d = off[o + 1] - off[o];
        indeg[i] = d;
        ntask[i] = (d + kPieceEdges - 1) / kPieceEdges;
    }
}

// task_dst[t] = the new vertex whose in-edges task t copies.
__global__ void k_rl_task_dst(const uint32_t* __restrict__ tofs, uint32_t V, uint32_t* __restrict__ task_dst) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < V; i += (uint64_t)gridDim.x * blockDim.x)
        for (uint32_t t = tofs[i]; t < tofs[i + 1]; ++t) task_dst[t] = (uint32_t)i;
}

// One warp per task: up to kPieceEdges in-edges of new vertex i, in their
// original order, sources renamed (weights carried along).
__global__ void k_rl_copy(const uint32_t* __restrict__ off, const uint32_t* __restrict__ src,
                          const uint32_t* __restrict__ w, const uint32_t* __restrict__ old_of_new,
                          const uint32_t* __restrict__ new_of_old, const uint32_t* __restrict__ new_off,
                          const uint32_t* __restrict__ tofs, const uint32_t* __restrict__ task_dst, uint32_t V,
                          uint32_t* __restrict__ nsrc, uint32_t* __restrict__ nw) {
    const unsigned lane = threadIdx.x & 31;
    const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t ntasks = tofs[V];
    for (uint64_t t = w0; t < ntasks; t += nwarps) {
        const uint32_t i = task_dst[t];
        const uint32_t o = old_of_new[i];
        const uint32_t j = (uint32_t)(t - tofs[i]) * kPieceEdges;
        const uint32_t b_old = off[o] + j, b_new = new_off[i] + j;
        const uint32_t d = off[o + 1] - off[o];
        const uint32_t n = d - j < kPieceEdges ? d - j : kPieceEdges;
        for (uint32_t q = lane; q < n; q += 32) {
            nsrc[b_new + q] = __ldg(new_of_old + src[b_old + q]);
            if (w) nw[b_new + q] = w[b_old + q];
        }
    }
}

// out[v * width + c] = in[new_of_old[v] * width + c]
__global__ void k_rl_rows(const uint32_t* __restrict__ new_of_old, uint32_t V, uint32_t width,
                          const uint32_t* __restrict__ in, uint32_t* __restrict__ out) {
    const uint64_t n = (uint64_t)V * width;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = x / width, c = x - v * width;
        out[x] = in[(uint64_t)new_of_old[v] * width + c];
    }
}

__global__ void k_rl_fill(uint32_t* p, uint32_t V, uint32_t x) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x)
        p[v] = x;
}

// Smallest old id per component: m[label of new vertex i] <- old id of i
// (labels >= V, which no CC run produces, are skipped).  Most vertices of
// a warp share a label (the giant component), so each distinct label of a
// warp takes one atomicMin with the warp's minimum for it.
__global__ void k_rl_label_min(const uint32_t* __restrict__ labels, const uint32_t* __restrict__ old_of_new,
                               uint32_t V, uint32_t* __restrict__ m) {
    const unsigned lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); i0 < V; i0 += stride) {
        const uint64_t i = i0 + lane;
        uint32_t l = 0xFFFFFFFFu, o = 0xFFFFFFFFu;
        if (i < V) {
            l = labels[i];
            o = old_of_new[i];
        }
        const bool valid = l < V;
        unsigned todo = __ballot_sync(kFull, valid);
        while (todo) {  // warp-uniform: one distinct label per round
            const unsigned src = __ffs(todo) - 1;
            const uint32_t lab = __shfl_sync(kFull, l, src);
            const bool mine = valid && l == lab;
            const uint32_t lo = __reduce_min_sync(kFull, mine ? o : 0xFFFFFFFFu);
            if (lane == src) atomicMin(m + lab, lo);
            todo &= ~__ballot_sync(kFull, mine);
        }
    }
}

__global__ void k_rl_label_out(const uint32_t* __restrict__ labels, const uint32_t* __restrict__ old_of_new,
                               uint32_t V, const uint32_t* __restrict__ m, uint32_t* __restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < V; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t l = labels[i];
        out[old_of_new[i]] = l < V ? m[l] : l;
    }
}

int device_sms(int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev);
    return (int)e;
}

struct Scratch {
    void* p[8] = {};
    cudaStream_t s;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void* q : p) dev_free_async(q, s);
    }
};

bool all_device(std::initializer_list<const void*> ps) {
    for (const void* p : ps)
        if (p && classify(p) != PtrKind::Device) return false;
    return true;
}

// PageRank's ranking keys: vertices of out-degree >= dmin first, by
// descending out-degree; all others after them in id order (one shared
// key, the sort is stable).
__global__ void k_rl_hub_keys(const uint32_t* __restrict__ deg, uint32_t V, uint32_t kmax, uint32_t dmin,
                              uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V; v += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t dg = deg[v];
        key[v] = dg >= dmin ? kmax - dg : kmax;
        val[v] = (uint32_t)v;
    }
}

// pr_src[e] = perm[src[e]], 16-byte loads and stores (tail by words).
__global__ void k_rl_rename(const uint32_t* __restrict__ src, uint64_t E, const uint32_t* __restrict__ perm,
                            uint32_t* __restrict__ out) {
    const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t n4 = E / 4;
    for (uint64_t q = tid; q < n4; q += nth) {
        const uint4 s = reinterpret_cast<const uint4*>(src)[q];
        reinterpret_cast<uint4*>(out)[q] = make_uint4(__ldg(perm + s.x), __ldg(perm + s.y), __ldg(perm + s.z),
                                                      __ldg(perm + s.w));
    }
    for (uint64_t p = 4 * n4 + tid; p < E; p += nth) out[p] = __ldg(perm + src[p]);
}

// perm[old_of_new[i]] = i
__global__ void k_rl_invert(const uint32_t* __restrict__ old_of_new, uint32_t V, uint32_t* __restrict__ perm) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < V; i += (uint64_t)gridDim.x * blockDim.x)
        perm[old_of_new[i]] = (uint32_t)i;
}

}  // namespace

// PageRank gathers one contribution per in-edge, indexed by the source;
// stored in the order of descending out-degree (the ranking the relabelling
// above gives), the most gathered contributions share cache lines.  Only
// the gathers move: destinations, the chunk metadata and every result stay
// in the graph's own ids, and the sums are the same exact fixed-point sums.
wedge_status build_pr_order(wedge_graph* g, cudaStream_t s) {
    if (g->pr_src) return WEDGE_OK;
    const uint32_t V = g->V;
    const uint64_t E = g->E;
    const int sms = g->num_sms;
    uint32_t* perm = nullptr;
    uint32_t* psrc = nullptr;
    WEDGE_TRY(dev_alloc(g, (void**)&perm, (uint64_t)V * 4));
    wedge_status st = dev_alloc(g, (void**)&psrc, (E ? E : 4) * 4);
    if (st != WEDGE_OK) {
        dev_free(perm);
        return st;
    }
    Scratch sc(s);
    for (int i = 0; i < 4 && st == WEDGE_OK; ++i) st = dev_alloc(nullptr, &sc.p[i], (uint64_t)V * 4);
    if (st == WEDGE_OK) {
        uint32_t *key = (uint32_t*)sc.p[0], *val = (uint32_t*)sc.p[1], *tkey = (uint32_t*)sc.p[2],
                 *tval = (uint32_t*)sc.p[3];
        int bits = 0;
        while (bits < 32 && (E >> bits)) ++bits;
        const uint32_t kmax = bits >= 32 ? 0xFFFFFFFFu : (uint32_t)((1ull << bits) - 1);
        k_rl_hub_keys<<<grid_of(V, 256, sms), 256, 0, s>>>(g->outdeg, V, kmax, kPrHubDegree, key, val);
        count_launch();
        bool in_tmp = false;
        st = radix_sort_pairs(key, val, tkey, tval, V, bits, sms, s, &in_tmp);
        if (st == WEDGE_OK) {
            k_rl_invert<<<grid_of(V, 256, sms), 256, 0, s>>>(in_tmp ? tval : val, V, perm);
            if (E) k_rl_rename<<<grid_of((E + 3) / 4, 256, sms), 256, 0, s>>>(g->src, E, perm, psrc);
            count_launch(2);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_error(e, "PageRank gather order");
        }
    }
    if (st != WEDGE_OK) {
        dev_free(perm);
        dev_free(psrc);
        return st;
    }
    g->pr_perm = perm;
    g->pr_src = psrc;
    return WEDGE_OK;
}

}  // namespace wedge

using namespace wedge;

extern "C" {

wedge_status wedge_csc_relabel_by_degree(uint32_t V, uint64_t E, const uint32_t* d_offsets, const uint32_t* d_src,
                                         const uint32_t* d_w, uint32_t* d_new_offsets, uint32_t* d_new_src,
                                         uint32_t* d_new_w, uint32_t* d_new_of_old, uint32_t* d_old_of_new,
                                         wedge_stream_t stream) {
    if (V == 0) return set_error(WEDGE_ERR_INVALID_ARG, "V must be >= 1");
    if (E >= 0xFFFFFF00ull) return set_error(WEDGE_ERR_INVALID_ARG, "E must be < 2^32 - 256");
    if (!d_offsets || !d_new_offsets || !d_new_of_old || (E && (!d_src || !d_new_src)))
        return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if ((d_w != nullptr) != (d_new_w != nullptr))
        return set_error(WEDGE_ERR_INVALID_ARG, "w and new_w must both be given or both be NULL");
    if (!all_device({d_offsets, d_src, d_w, d_new_offsets, d_new_src, d_new_w, d_new_of_old, d_old_of_new}))
        return set_error(WEDGE_ERR_INVALID_ARG, "every array must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0;
    if (int e = device_sms(&sms)) return cuda_error((cudaError_t)e, "cudaDeviceGetAttribute");
    Scratch sc(s);
    uint32_t *deg, *key, *val, *tkey, *tval, *tofs, *task_dst;
    unsigned* bad;
    const uint64_t V1 = (uint64_t)V + 1;
    WEDGE_TRY(dev_alloc(nullptr, &sc.p[0], V1 * 4));
    WEDGE_TRY(dev_alloc(nullptr, &sc.p[1], V1 * 4));
    WEDGE_TRY(dev_alloc(nullptr, &sc.p[2], V1 * 4));
    WEDGE_TRY(dev_alloc(nullptr, &sc.p[3], V1 * 4));
    WEDGE_TRY(dev_alloc(nullptr, &sc.p[4], V1 * 4));
    WEDGE_TRY(dev_alloc(nullptr, &sc.p[5], V1 * 4));
    WEDGE_TRY(dev_alloc(nullptr, &sc.p[6], (V1 + E / kPieceEdges + 1) * 4));
    WEDGE_TRY(dev_alloc(nullptr, &sc.p[7], 4));
    deg = (uint32_t*)sc.p[0];
    key = (uint32_t*)sc.p[1];
    val = (uint32_t*)sc.p[2];
    tkey = (uint32_t*)sc.p[3];
    tval = (uint32_t*)sc.p[4];
    tofs = (uint32_t*)sc.p[5];
    task_dst = (uint32_t*)sc.p[6];
    bad = (unsigned*)sc.p[7];
    WEDGE_TRY_CUDA(cudaMemsetAsync(deg, 0, V1 * 4, s));
    WEDGE_TRY_CUDA(cudaMemsetAsync(bad, 0, 4, s));
    const uint64_t nmax = E > V ? E : V;
    k_rl_check_count<<<grid_of(nmax, 256, sms), 256, 0, s>>>(d_offsets, d_src, V, E, deg, bad);
    count_launch();
    uint32_t h[3] = {1, 0, 0};
    WEDGE_TRY_CUDA(cudaMemcpyAsync(&h[0], d_offsets, 4, cudaMemcpyDeviceToHost, s));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(&h[1], d_offsets + V, 4, cudaMemcpyDeviceToHost, s));
    WEDGE_TRY_CUDA(cudaMemcpyAsync(&h[2], bad, 4, cudaMemcpyDeviceToHost, s));
    WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    if (h[0] != 0 || h[1] != E) return set_error(WEDGE_ERR_INVALID_ARG, "offsets[0] must be 0 and offsets[V] must be E");
    if (h[2] & 1u) return set_error(WEDGE_ERR_INVALID_ARG, "offsets must be non-decreasing");
    if (h[2] & 2u) return set_error(WEDGE_ERR_INVALID_ARG, "a source id is >= V");
    // descending out-degree (<= E), stable: ties keep ascending old ids
    int bits = 0;
    while (bits < 32 && (E >> bits)) ++bits;
    const uint32_t kmax = bits >= 32 ? 0xFFFFFFFFu : (uint32_t)((1ull << bits) - 1);
    k_rl_keys<<<grid_of(V, 256, sms), 256, 0, s>>>(deg, V, kmax, key, val);
    count_launch();
    bool in_tmp = false;
    WEDGE_TRY(radix_sort_pairs(key, val, tkey, tval, V, bits, sms, s, &in_tmp));
    const uint32_t* sorted = in_tmp ? tval : val;
    uint32_t* indeg = in_tmp ? val : tval;   // free again after the sort
    uint32_t* ntask = deg;                   // out-degrees are no longer needed
    if (d_old_of_new)
        WEDGE_TRY_CUDA(cudaMemcpyAsync(d_old_of_new, sorted, (uint64_t)V * 4, cudaMemcpyDeviceToDevice, s));
    k_rl_place<<<grid_of(V, 256, sms), 256, 0, s>>>(sorted, d_offsets, V, d_new_of_old, indeg, ntask);
    count_launch();
    WEDGE_TRY(exclusive_scan_u32(indeg, d_new_offsets, V, nullptr, s));
    WEDGE_TRY(exclusive_scan_u32(ntask, tofs, V, nullptr, s));
    k_rl_task_dst<<<grid_of(V, 256, sms), 256, 0, s>>>(tofs, V, task_dst);
    count_launch();
    if (E) {
        k_rl_copy<<<(unsigned)sms * 8, 256, 0, s>>>(d_offsets, d_src, d_w, sorted, d_new_of_old, d_new_offsets, tofs,
                                                   task_dst, V, d_new_src, d_new_w);
        count_launch();
    }
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

wedge_status wedge_permute_rows(uint32_t V, uint32_t width, const uint32_t* d_new_of_old, const uint32_t* d_in,
                                uint32_t* d_out, wedge_stream_t stream) {
    if (V == 0 || width == 0) return set_error(WEDGE_ERR_INVALID_ARG, "V and width must be >= 1");
    if (!d_new_of_old || !d_in || !d_out) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (d_in == d_out) return set_error(WEDGE_ERR_INVALID_ARG, "in and out must not be the same array");
    if (!all_device({d_new_of_old, d_in, d_out})) return set_error(WEDGE_ERR_INVALID_ARG, "arrays must be device memory");
    int sms = 0;
    if (int e = device_sms(&sms)) return cuda_error((cudaError_t)e, "cudaDeviceGetAttribute");
    k_rl_rows<<<grid_of((uint64_t)V * width, 256, sms), 256, 0, (cudaStream_t)stream>>>(d_new_of_old, V, width, d_in,
                                                                                        d_out);
    count_launch();
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

wedge_status wedge_cc_labels_to_original(uint32_t V, const uint32_t* d_old_of_new, const uint32_t* d_labels,
                                         uint32_t* d_scratch, uint32_t* d_out, wedge_stream_t stream) {
    if (V == 0) return set_error(WEDGE_ERR_INVALID_ARG, "V must be >= 1");
    if (!d_old_of_new || !d_labels || !d_scratch || !d_out) return set_error(WEDGE_ERR_INVALID_ARG, "NULL argument");
    if (d_out == d_labels || d_scratch == d_labels || d_scratch == d_out)
        return set_error(WEDGE_ERR_INVALID_ARG, "labels, scratch and out must be distinct arrays");
    if (!all_device({d_old_of_new, d_labels, d_scratch, d_out}))
        return set_error(WEDGE_ERR_INVALID_ARG, "arrays must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0;
    if (int e = device_sms(&sms)) return cuda_error((cudaError_t)e, "cudaDeviceGetAttribute");
    k_rl_fill<<<grid_of(V, 256, sms), 256, 0, s>>>(d_scratch, V, 0xFFFFFFFFu);
    k_rl_label_min<<<grid_of(V, 256, sms), 256, 0, s>>>(d_labels, d_old_of_new, V, d_scratch);
    k_rl_label_out<<<grid_of(V, 256, sms), 256, 0, s>>>(d_labels, d_old_of_new, V, d_scratch, d_out);
    count_launch(3);
    WEDGE_TRY_CUDA(cudaGetLastError());
    return WEDGE_OK;
}

}  // extern "C"

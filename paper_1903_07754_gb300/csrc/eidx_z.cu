// The compressed edge index (Section 4 names in-memory compression of the
// edge index as a way to cut the transformation's memory traffic).
//
// Layout.  Each row of the edge index (the chunks holding a source's
// out-edges) is put in ascending order and cut into blocks of up to 32
// entries, the transformation's work pieces.  A block stores its first
// entry and the differences between consecutive entries, every difference
// in the same number of bits w (the fewest that hold the block's largest),
// packed little-endian into 32-bit words that start at a word boundary:
//   zhdr[b] = {first entry | w << 27, index of the block's first word}
//   zwords[]  the packed differences
//   zbo[u]    index of row u's first block (rows keep eidx_off's lengths)
// Entries are below NC < 2^27, so the first entry and w share one word.
// Decoding entry i of a block: the first entry plus the sum of differences
// 1..i, a prefix sum across the warp's lanes.
#include "common.cuh"

namespace wedge {

wedge_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* tkeys, uint32_t* tvals, uint64_t n,
                              int key_bits, int num_sms, cudaStream_t s, bool* in_tmp);

namespace {

unsigned grid_of(uint64_t n, int threads, int sms) {
    const uint64_t b = (n + threads - 1) / threads;
    const uint64_t cap = (uint64_t)sms * 8;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 32 && (maxval >> b)) ++b;
    return b;
}

// (entry, row) pairs in the index's order: one warp per row.
__global__ void k_z_pairs(const uint32_t* __restrict__ eoff, const uint32_t* __restrict__ eidx, uint32_t V,
                          uint32_t* __restrict__ ent, uint32_t* __restrict__ row) {
    const unsigned lane = threadIdx.x & 31;
    const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = w0; u < V; u += nw) {
        const uint32_t b = eoff[u], e = eoff[u + 1];
        for (uint32_t i = b + lane; i < e; i += 32) {
            ent[i] = eidx[i];
            row[i] = (uint32_t)u;
        }
    }
}

// Blocks per row: ceil(len / 32).
__global__ void k_z_nblocks(const uint32_t* __restrict__ eoff, uint32_t V, uint32_t* __restrict__ nb) {
    for (uint64_t u = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; u < V; u += (uint64_t)gridDim.x * blockDim.x)
        nb[u] = (eoff[u + 1] - eoff[u] + 31u) >> 5;
}

// Row of block b: the last u with zbo[u] <= b (zbo non-decreasing, V+1 long).
__device__ __forceinline__ uint32_t z_row_of(const uint32_t* __restrict__ zbo, uint32_t V, uint32_t b) {
    uint32_t lo = 0, hi = V;  // zbo[lo] <= b < zbo[hi]
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (__ldg(zbo + mid) <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

// One warp per block: its entries (sorted rows), their differences, the
// width w; WORDS: the block's word count, else its header and packed bits
// (ORed into zeroed words).
template <bool WORDS>
__global__ void k_z_blocks(const uint32_t* __restrict__ eoff, const uint32_t* __restrict__ sorted,
                           const uint32_t* __restrict__ zbo, uint32_t V, uint64_t nblocks,
                           uint32_t* __restrict__ words_or_off, uint2* __restrict__ zhdr,
                           uint32_t* __restrict__ zwords) {
    const unsigned lane = threadIdx.x & 31;
    const uint64_t w0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t b = w0; b < nblocks; b += nw) {
        const uint32_t u = z_row_of(zbo, V, (uint32_t)b);
        const uint32_t q = (uint32_t)b - __ldg(zbo + u);
        const uint32_t r0 = __ldg(eoff + u) + 32u * q, r1 = __ldg(eoff + u + 1);
        const uint32_t n = min(32u, r1 - r0);
        const uint32_t x = lane < n ? sorted[r0 + lane] : 0u;
        const uint32_t xp = __shfl_up_sync(kFull, x, 1);
        const uint32_t d = (lane > 0 && lane < n) ? x - xp : 0u;
        unsigned m = d;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
        const unsigned w = m ? 32u - __clz(m) : 0u;
        const unsigned nwords = (unsigned)(((n - 1) * w + 31u) >> 5);
        if (WORDS) {
            if (lane == 0) words_or_off[b] = nwords;
        } else {
            const uint32_t woff = words_or_off[b];
            const uint32_t first = __shfl_sync(kFull, x, 0);
            if (lane == 0) zhdr[b] = make_uint2(first | (w << 27), woff);
            if (lane > 0 && lane < n && w) {
                const unsigned bit = (lane - 1) * w;
                const unsigned j = bit >> 5, r = bit & 31u;
                atomicOr(zwords + woff + j, d << r);
                if (r + w > 32u) atomicOr(zwords + woff + j + 1, d >> (32u - r));
            }
        }
    }
}

}  // namespace

wedge_status build_eidx_z(wedge_graph* g, cudaStream_t s) {
    if (g->zpieces) return WEDGE_OK;  // allocated last: the index is complete
    for (void** p : {(void**)&g->zhdr, (void**)&g->zwords, (void**)&g->zbo}) {  // a build that failed midway
        dev_free(*p);
        *p = nullptr;
    }
    const uint32_t V = g->V;
    const uint64_t len = g->eidx_len;
    const int sms = g->num_sms;
    if (g->NC >= (1ull << 27)) return set_error(WEDGE_ERR_NOT_SUPPORTED, "compressed edge index needs NC < 2^27");
    // rows in ascending order: stable sorts by entry, then by row
    uint32_t* buf[4] = {nullptr, nullptr, nullptr, nullptr};
    struct Free {
        uint32_t** b;
        cudaStream_t s;
        ~Free() {
            for (int i = 0; i < 4; ++i) dev_free_async(b[i], s);
        }
    } guard{buf, s};
    for (int i = 0; i < 4; ++i) WEDGE_TRY(dev_alloc(nullptr, (void**)&buf[i], (len ? len : 1) * 4));
    uint32_t* sorted = buf[0];
    if (len) {
        k_z_pairs<<<grid_of((uint64_t)V * 32, 256, sms), 256, 0, s>>>(g->eidx_off, g->eidx, V, buf[0], buf[1]);
        count_launch();
        bool t1 = false, t2 = false;
        WEDGE_TRY(radix_sort_pairs(buf[0], buf[1], buf[2], buf[3], len, bits_for(g->NC ? g->NC - 1 : 0), sms, s, &t1));
        uint32_t* ent = t1 ? buf[2] : buf[0];
        uint32_t* row = t1 ? buf[3] : buf[1];
        uint32_t* ent_t = t1 ? buf[0] : buf[2];
        uint32_t* row_t = t1 ? buf[1] : buf[3];
        WEDGE_TRY(radix_sort_pairs(row, ent, row_t, ent_t, len, bits_for(V - 1), sms, s, &t2));
        sorted = t2 ? ent_t : ent;
    }
    // blocks per row and their offsets
    WEDGE_TRY(dev_alloc(g, (void**)&g->zbo, ((uint64_t)V + 1) * 4));
    uint32_t* nbv = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&nbv, ((uint64_t)V + 1) * 4));
    k_z_nblocks<<<grid_of(V, 256, sms), 256, 0, s>>>(g->eidx_off, V, nbv);
    count_launch();
    wedge_status st = exclusive_scan_u32(nbv, g->zbo, V, nullptr, s);
    dev_free_async(nbv, s);
    WEDGE_TRY(st);
    uint32_t nblocks = 0;
    WEDGE_TRY_CUDA(cudaMemcpyAsync(&nblocks, g->zbo + V, 4, cudaMemcpyDeviceToHost, s));
    WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    g->zblocks = nblocks;
    // words per block, their offsets, then headers and packed differences
    uint32_t* wcount = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&wcount, ((uint64_t)nblocks + 1) * 4));
    struct Free1 {
        uint32_t* p;
        cudaStream_t s;
        ~Free1() { dev_free_async(p, s); }
    } free_wc{wcount, s};
    WEDGE_TRY(dev_alloc(g, (void**)&g->zhdr, ((uint64_t)nblocks + 1) * sizeof(uint2)));
    if (nblocks) {
        k_z_blocks<true><<<grid_of((uint64_t)nblocks * 32, 256, sms), 256, 0, s>>>(
            g->eidx_off, sorted, g->zbo, V, nblocks, wcount, nullptr, nullptr);
        count_launch();
    }
    uint32_t* woff = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&woff, ((uint64_t)nblocks + 1) * 4));
    struct Free2 {
        uint32_t* p;
        cudaStream_t s;
        ~Free2() { dev_free_async(p, s); }
    } free_wo{woff, s};
    WEDGE_TRY(exclusive_scan_u32(wcount, woff, nblocks, nullptr, s));
    uint32_t nwords = 0;
    WEDGE_TRY_CUDA(cudaMemcpyAsync(&nwords, woff + nblocks, 4, cudaMemcpyDeviceToHost, s));
    WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    g->zwords_len = nwords;
    WEDGE_TRY(dev_alloc(g, (void**)&g->zwords, ((uint64_t)nwords + 2) * 4));
    WEDGE_TRY_CUDA(cudaMemsetAsync(g->zwords, 0, ((uint64_t)nwords + 2) * 4, s));
    if (nblocks) {
        k_z_blocks<false><<<grid_of((uint64_t)nblocks * 32, 256, sms), 256, 0, s>>>(
            g->eidx_off, sorted, g->zbo, V, nblocks, woff, g->zhdr, g->zwords);
        count_launch();
    }
    WEDGE_TRY(dev_alloc(g, (void**)&g->zpieces, (g->npieces_max + 1) * sizeof(uint4)));
    WEDGE_TRY_CUDA(cudaGetLastError());
    WEDGE_TRY_CUDA(cudaStreamSynchronize(s));
    g->z_bytes = (uint64_t)nblocks * sizeof(uint2) + (uint64_t)nwords * 4 + ((uint64_t)V + 1) * 4;
    return WEDGE_OK;
}

}  // namespace wedge

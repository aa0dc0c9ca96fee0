// Stable LSD radix sort of (key, value) uint32 pairs on the device, 8-bit
// digits: per pass a digit histogram per block, an exclusive scan of the
// (digit, block) counts, and a scatter in which each block ranks its
// segment's items in input order (warp ranks from eight ballots on the
// digit's bits, block ranks from per-warp digit counts).  Used off the
// timed path to order the edge index's rows before compressing them.
#include <utility>

#include "common.cuh"

namespace wedge {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kDigits = 256;

__device__ __forceinline__ unsigned digit_of(uint32_t key, int shift) { return (key >> shift) & 0xFFu; }

// Lanes of the warp whose digit equals this lane's (eight ballots).
__device__ __forceinline__ unsigned digit_peers(unsigned d, bool valid) {
    unsigned peers = __ballot_sync(kFull, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const unsigned m = __ballot_sync(kFull, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? m : ~m;
    }
    return peers;
}

// counts[d * nblocks + b] = items of block b's segment with digit d.
__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t* __restrict__ keys, uint64_t n,
                                                            uint64_t seg, int shift, uint32_t* __restrict__ counts) {
    __shared__ unsigned h[kSortWarps][kDigits];
    for (int i = threadIdx.x; i < kSortWarps * kDigits; i += blockDim.x) (&h[0][0])[i] = 0u;
    __syncthreads();
    const uint64_t b0 = blockIdx.x * seg, b1 = b0 + seg < n ? b0 + seg : n;
    unsigned* mine = h[threadIdx.x >> 5];
    for (uint64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(mine + digit_of(keys[i], shift), 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x) {
        unsigned s = 0;
        for (int w = 0; w < kSortWarps; ++w) s += h[w][d];
        counts[(uint64_t)d * gridDim.x + blockIdx.x] = s;
    }
}

// Scatter of block b's segment, 256 items per round in input order.
__global__ void __launch_bounds__(kSortThreads)
    k_sort_scatter(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t n, uint64_t seg,
                   int shift, const uint32_t* __restrict__ offs, uint32_t* __restrict__ okeys,
                   uint32_t* __restrict__ ovals) {
    __shared__ unsigned wcnt[kSortWarps][kDigits];  // this round's counts per warp (then their prefix)
    __shared__ unsigned run[kDigits];               // next output slot of each digit
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kDigits; i += blockDim.x) (&wcnt[0][0])[i] = 0u;
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x) run[d] = offs[(uint64_t)d * gridDim.x + blockIdx.x];
    __syncthreads();
    const uint64_t b0 = blockIdx.x * seg, b1 = b0 + seg < n ? b0 + seg : n;
    for (uint64_t base = b0; base < b1; base += blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        const bool valid = i < b1;
        const uint32_t k = valid ? keys[i] : 0u;
        const uint32_t v = valid ? vals[i] : 0u;
        const unsigned d = digit_of(k, shift);
        const unsigned peers = digit_peers(d, valid);
        const unsigned wrank = __popc(peers & ((1u << lane) - 1u));
        if (valid && wrank == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        // per digit: exclusive prefix over the warps, then advance the slot
        for (int dd = threadIdx.x; dd < kDigits; dd += blockDim.x) {
            unsigned s = run[dd];
            for (int w = 0; w < kSortWarps; ++w) {
                const unsigned c = wcnt[w][dd];
                wcnt[w][dd] = s;
                s += c;
            }
            run[dd] = s;
        }
        __syncthreads();
        if (valid) {
            const unsigned pos = wcnt[warp][d] + wrank;
            okeys[pos] = k;
            ovals[pos] = v;
        }
        __syncthreads();
        for (int ii = threadIdx.x; ii < kSortWarps * kDigits; ii += blockDim.x) (&wcnt[0][0])[ii] = 0u;
        __syncthreads();
    }
}

}  // namespace

// Sorts n pairs by key (the low key_bits bits; higher bits must be zero),
// stably.  keys/vals are the input; tkeys/tvals scratch of n entries each.
// On return *in_tmp says which pair of buffers holds the result.  n < 2^32.
wedge_status radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* tkeys, uint32_t* tvals, uint64_t n,
                              int key_bits, int num_sms, cudaStream_t s, bool* in_tmp) {
    *in_tmp = false;
    if (n <= 1 || key_bits <= 0) return WEDGE_OK;
    if (n >= (1ull << 32)) return set_error(WEDGE_ERR_NOT_SUPPORTED, "radix sort of 2^32 items or more");
    const uint64_t per = 4096;
    uint64_t nb = (n + per - 1) / per;
    const uint64_t cap = (uint64_t)num_sms * 4;
    if (nb > cap) nb = cap;
    const uint64_t seg = (n + nb - 1) / nb;
    uint32_t* counts = nullptr;
    uint32_t* offs = nullptr;
    WEDGE_TRY(dev_alloc(nullptr, (void**)&counts, (kDigits * nb + 1) * 4));
    wedge_status st = dev_alloc(nullptr, (void**)&offs, (kDigits * nb + 1) * 4);
    if (st != WEDGE_OK) {
        dev_free(counts);
        return st;
    }
    uint32_t *ik = keys, *iv = vals, *ok = tkeys, *ov = tvals;
    for (int shift = 0; shift < key_bits && st == WEDGE_OK; shift += 8) {
        k_sort_hist<<<(unsigned)nb, kSortThreads, 0, s>>>(ik, n, seg, shift, counts);
        st = exclusive_scan_u32(counts, offs, kDigits * nb, nullptr, s);
        if (st != WEDGE_OK) break;
        k_sort_scatter<<<(unsigned)nb, kSortThreads, 0, s>>>(ik, iv, n, seg, shift, offs, ok, ov);
        count_launch(2);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_error(e, "radix sort pass");
        std::swap(ik, ok);
        std::swap(iv, ov);
        *in_tmp = !*in_tmp;
    }
    dev_free_async(counts, s);
    dev_free_async(offs, s);
    return st;
}

}  // namespace wedge

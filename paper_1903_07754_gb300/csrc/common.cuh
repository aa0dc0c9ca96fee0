// Internal definitions shared by the translation units of libwedge.so.
//
// Device layout of a graph object (all library-owned unless noted):
//   off[V+1], src[E], w[E]   CSC in-edges (borrowed, or owned copies of host input)
//   outdeg[V]                out-degree of every vertex
//   vid[NZ]                  ids of the vertices with in-degree > 0, ascending
//   cmeta[NC]                per 32-edge chunk c: .x = head mask (bit i set iff
//                            position 32c+i is the first in-edge of its
//                            destination), .y = index into vid of the
//                            destination of position 32c
//   eidx_off[V+1], eidx[]    edge index (Sections 3.3, 4): row u lists the
//                            chunks that hold u's out-edges, once each
//   npieces_max              sum over u of ceil(|row u| / 32)
//   csr_off[V+1], csr_dst[E], csr_src[E], csr_w[E], kid_of[V]
//                            out-edges (CSR) for the push/pull hybrid, built on
//                            its first run: edge j leaves csr_src[j] for
//                            csr_dst[j]; kid_of[v] = index of v in vid
// The head mask plus vid let a warp find the destination of each of its
// edges from the chunk alone, the role the paper gives to Vector-Sparse
// (Section 2.2): no search in off[] on the hot path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/wedge.h"

#define WEDGE_VERSION_STRING "wedge-gb300 0.1"

namespace wedge {

constexpr unsigned kFull = 0xFFFFFFFFu;  // all lanes of a warp
constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr uint32_t kSat = 0xFFFFFFFEu;
constexpr uint32_t kChunk = 32;
constexpr uint32_t kMaxCoarsen = 7;
constexpr uint32_t kDefaultMaxIters = 1u << 20;
constexpr int kXformThreads = 256;
constexpr int kFixedShift = 62;  // PageRank fixed point: 1.0 == 2^62

// Pull geometry.  A warp processes a slice of kSliceC chunks (kEPL edges per
// lane); a block has kCW such consumer warps plus one producer warp that
// streams tiles of kTileC chunks into kStages shared-memory stages with 1D
// bulk copies (dense pulls).
constexpr int kEPL = 8;
constexpr int kSliceE = 32 * kEPL;          // 256 edges
constexpr int kSliceC = kSliceE / 32;       // 8 chunks
constexpr int kCW = 8;
constexpr int kPullThreads = (kCW + 1) * 32;
constexpr int kTileC = kCW * kSliceC;       // 64 chunks per stage
constexpr int kTileE = kTileC * 32;         // 2048 edges per stage
constexpr int kStages = 4;
constexpr int kMetaPad = 2;                 // chunk metadata entries copied past a tile
constexpr int kSliceShift = 8;              // log2(kSliceE)
// Segment records a pull warp buffers at a time (a slice makes one per
// destination segment, up to kSliceE; more take further passes).  The less
// shared memory the pulls take, the more of the unified L1 caches gathers.
#ifndef WEDGE_REC_CAP
#define WEDGE_REC_CAP 64
#endif
constexpr int kRecCap = WEDGE_REC_CAP;
static_assert(kRecCap % 32 == 0 && kRecCap <= kSliceE, "record buffer");

// Per-iteration record (device).  Slot t describes frontier F_t and pull t.
struct IterRec {
    unsigned long long fullness;  // sum outdeg over F_t (written by pull t-1)
    unsigned int nfront;          // |F_t|
    unsigned int npieces;         // transformation work pieces for F_t
    unsigned int nchunks;         // Wedge Frontier entries for pull t
    unsigned int mode;            // 0 dense, 1 sparse (decided after pull t-1)
    unsigned int k;               // coarsening used by pull t
    unsigned int rowsum;          // sum |eidx row| over F_t
    unsigned long long t_pull0, t_pull1;    // globaltimer stamps of pull t
    unsigned long long t_xf0, t_xf1;        // and of the transformation for t
    unsigned int nlist;           // F_t vertices written to the frontier list
                                  // (the list is complete iff nlist == nfront)
    unsigned int nlong;           // F_t's long edge-index rows listed for the transformation
    unsigned int rowmax;          // max |eidx row| over F_t
    unsigned int pad_;
};
static_assert(sizeof(IterRec) == 80, "IterRec layout");
constexpr int kListCap = 1024;  // frontier-list entries a pull block stages in shared memory
constexpr int kMaxPullBlocks = 4096;

// What one pull block found: written to its own slot (no shared counter),
// summed by the pull's last block when it takes the decision.
struct BlockStat {
    unsigned long long F;  // sum of out-degrees of the vertices it activated
    unsigned int n;        // vertices it activated
    unsigned int row;      // their edge-index row lengths
    unsigned int lcnt;     // vertices it staged for the next frontier list (> kListCap: overflow)
    unsigned int rowmax;   // the longest of their edge-index rows
};

// Run control block (device).
struct RunCtl {
    unsigned int it;          // iteration about to be pulled
    unsigned int done;        // 1 once the frontier is empty or max_iters hit
    unsigned int ticket;      // last-block election in the pull
    unsigned int status;      // kStatus* bits
    unsigned int max_iters;
    unsigned int switch_mode; // wedge_switch
    unsigned int tau_bp;
    unsigned int k;           // coarsening for sparse iterations
    unsigned long long E;
    unsigned long long dangling[2];  // PageRank: fixed-point dangling mass
    unsigned int loops;              // loop-body executions (bounds the device loop)
    unsigned int pad_;
};
constexpr unsigned int kStatusMaxIters = 1u;
constexpr unsigned int kStatusLevelOverflow = 4u;  // 8-bit batched levels: a level of 255 or more was needed

}  // namespace wedge

struct wedge_graph {
    int device = 0;
    uint32_t V = 0;
    uint64_t E = 0;
    uint64_t NC = 0;
    uint32_t NZ = 0;
    uint64_t eidx_len = 0;
    uint64_t npieces_max = 0;
    const uint32_t* off = nullptr;
    const uint32_t* src = nullptr;
    const uint32_t* w = nullptr;
    // owned
    uint32_t* off_own = nullptr;
    uint32_t* src_own = nullptr;
    uint32_t* w_own = nullptr;
    uint32_t* outdeg = nullptr;
    uint32_t* vid = nullptr;
    uint2* cmeta = nullptr;
    uint32_t* eidx_off = nullptr;
    uint32_t* eidx = nullptr;
    bool eidx_owned = false;
    bool eidx_off_owned = false;
    // scratch for runs
    uint32_t* vals = nullptr;      // V values of the current run
    uint32_t* vals_sync = nullptr; // synchronous CC/SSSP runs: the second value buffer
    uint32_t* bm[2] = {nullptr, nullptr};  // vertex frontier bitmaps
    uint32_t* wb = nullptr;        // Wedge Frontier bitmap, ceil(NC/32) words
    uint32_t* clist = nullptr;     // Wedge Frontier list, NC entries
    uint2* pieces = nullptr;       // transformation work pieces
    uint32_t* longs = nullptr;     // the transformation's long rows (kLongCap entries)
    unsigned* xf_task = nullptr;   // the expansion's task counter
    uint32_t* flist[2] = {nullptr, nullptr};  // frontier vertex lists by iteration parity
    uint32_t* visk = nullptr;      // BFS: visited destinations by index into vid, ceil(NZ/32)+1 words
    wedge::BlockStat* bstat = nullptr;  // per-block results of the last pull
    wedge::IterRec* rec = nullptr; // per-iteration records
    uint32_t rec_cap = 0;
    wedge::RunCtl* ctl = nullptr;
    wedge::RunCtl* h_ctl = nullptr;  // pinned mirror
    // PageRank scratch
    float* contrib = nullptr;               // pr(u)/outdeg(u), at position pr_perm[u]
    // PageRank's gather order: pr_perm[u] = u's rank by descending
    // out-degree (ties by id), pr_src[e] = pr_perm[src[e]]; built on the
    // first PageRank call
    uint32_t* pr_perm = nullptr;
    uint32_t* pr_src = nullptr;
    unsigned long long* acc = nullptr;
    float* rank = nullptr;
    uint32_t* split_bm = nullptr;  // destinations whose in-edges cross a pull slice boundary
    uint64_t meta_len = 0;         // cmeta entries allocated (NC rounded up plus padding)
    // device loop graphs (one per frontier application) and the PageRank graph
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t loop_exec[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t loop_exec_push[3] = {nullptr, nullptr, nullptr};
    // push/pull hybrid (the comparison engine): out-edges, built on first use
    uint32_t* csr_off = nullptr;
    uint32_t* csr_dst = nullptr;
    uint32_t* csr_src = nullptr;
    uint32_t* csr_w = nullptr;
    uint32_t* kid_of = nullptr;
    uint2* push_pieces = nullptr;
    uint64_t npieces_push_max = 0;
    bool last_push = false;
    bool loop_failed = false;
    cudaGraphExec_t pr_exec = nullptr;
    uint32_t pr_exec_iters = 0;
    float pr_exec_damping = -1.f;
    int pull_smem = 0;
    // learned switch
    void* mlp_bf16 = nullptr;        // cost model weights (BF16)
    bool has_model = false;
    float band_lo = 0.f, band_hi = 3.0e38f;  // fullness / E where the model is evaluated
    uint32_t max_outdeg = 0;
    uint32_t* snap_vals = nullptr;   // candidate-timing trace: value snapshot
    uint32_t* snap_visk = nullptr;   // candidate-timing trace: visited-bitmap snapshot
    // batched BFS
    unsigned long long* ms_fb[2] = {nullptr, nullptr};
    unsigned long long* ms_seen = nullptr;
    uint32_t* ms_roots = nullptr;    // roots then their query ids
    uint32_t ms_cap = 0;
    unsigned* ms_bar = nullptr;
    int ms_blocks = 0;
    int ms_occ = 0;                  // resident blocks per SM of the batched BFS kernel
    int ms_occ_sssp = 0;             // ... and of the batched SSSP kernel
    cudaGraphExec_t ms_exec = nullptr;
    uint32_t ms_exec_q = 0, ms_exec_n = 0;
    void* ms_exec_levels = nullptr;
    uint32_t ms_exec_key[5] = {0, 0, 0, 0, 0};  // tau, k, switch, max_iters, SSSP
    bool ms_graph_failed = false;
    uint64_t device_bytes = 0;
    int num_sms = 0;
    size_t smem_per_sm = 0;
    int pull_blocks = 0;
    int pull_blocks_app[4] = {0, 0, 0, 0};     // direct-load pulls
    int pull_blocks_tma[4] = {0, 0, 0, 0};     // bulk-copy staged dense pulls
    wedge_tuning tuning{};
    // edge index in 8-edge units (the finer precisions; built on first use)
    uint32_t* eidx8_off = nullptr;
    uint32_t* eidx8 = nullptr;
    uint64_t eidx8_len = 0, npieces8_max = 0;
    uint64_t npieces_outdeg_bound = 0;  // sum ceil(outdeg / 32): bounds the pieces of either index
    uint64_t wb_words = 0;          // Wedge bitmap words allocated
    uint64_t clist_cap = 0;         // Wedge list entries allocated
    uint64_t pieces_cap = 0;        // work pieces allocated
    // compressed edge index (built when the tuning asks for it; eidx_z.cu)
    uint2* zhdr = nullptr;          // per block: {first entry | width << 27, first word}
    uint32_t* zwords = nullptr;     // packed differences
    uint32_t* zbo = nullptr;        // V+1: first block of each row
    uint4* zpieces = nullptr;       // the transformation's pieces in compressed mode
    uint64_t zblocks = 0, zwords_len = 0, z_bytes = 0;
    int xform_blocks = 0;
    unsigned* slice_ctr = nullptr;  // load-balance study: the paper's schedule's slice counter
    uint32_t last_iters = 0;
    bool last_trace = false;
    cudaStream_t last_stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace wedge {

// ---- error handling (api.cu) ----
wedge_status set_error(wedge_status s, const std::string& msg);
wedge_status cuda_error(cudaError_t e, const char* what);
void count_launch(uint64_t n = 1);

// ---- the push/pull hybrid's out-edges, built on its first run (graph_build.cu) ----
wedge_status build_csr(wedge_graph* g, cudaStream_t s);

#define WEDGE_TRY_CUDA(expr)                                      \
    do {                                                          \
        cudaError_t e_ = (expr);                                  \
        if (e_ != cudaSuccess) return ::wedge::cuda_error(e_, #expr); \
    } while (0)

#define WEDGE_TRY(expr)                      \
    do {                                     \
        wedge_status s_ = (expr);            \
        if (s_ != WEDGE_OK) return s_;       \
    } while (0)

// Allocation helper that records the bytes owned by g.
wedge_status dev_alloc(wedge_graph* g, void** p, size_t bytes);
void dev_free(void* p);
void dev_free_async(void* p, cudaStream_t s);
wedge_status trim_pools(int device);
void* pinned_small_alloc(size_t bytes);  // at most 256 bytes; nullptr on failure
void pinned_small_free(void* p);

// Exclusive scan of n uint32 values into out[0..n] (out[n] = total), on the
// device, using tmp scratch of scan_tmp_words(n) words.  Totals must fit in
// 32 bits.
size_t scan_tmp_words(uint64_t n);
wedge_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* tmp,
                                cudaStream_t s);

// Engine (engine.cu)
wedge_status ensure_run_scratch(wedge_graph* g, cudaStream_t s);

// The compressed edge index (eidx_z.cu), built once on request.
wedge_status build_eidx_z(wedge_graph* g, cudaStream_t s);
// The edge index in 8-edge units (graph_build.cu), built once on request.
wedge_status build_eidx8(wedge_graph* g, cudaStream_t s);
// PageRank's gather order (relabel.cu), built once on request.
wedge_status build_pr_order(wedge_graph* g, cudaStream_t s);

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Kind of memory a pointer refers to, as seen from the graph's device.
enum class PtrKind { Device, Host, Invalid };
PtrKind classify(const void* p);

__device__ __forceinline__ unsigned int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned long long global_timer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace wedge

/*
 * wedge.h - C ABI of the GB300 Wedge engine (libwedge.so).
 *
 * Wedge (Grossman & Kozyrakis, "A New Frontier for Pull-Based Graph
 * Processing", arXiv 1903.07754) is a pull-only graph engine.  Each
 * iteration pulls values along in-edges and produces the traditional
 * source-oriented vertex frontier (Section 3.1, Requirement 1).  When that
 * frontier is sparse enough (the fullness threshold, Section 3.4) it is
 * transformed into the Wedge Frontier: the set of edge groups ("chunks") of
 * the destination-sorted in-edge array that hold an edge from an active
 * source (Sections 3.3, 4), and the next iteration pulls only over those
 * chunks; otherwise it pulls over all edges.
 *
 * Conventions for every entry point:
 *  - Graph layout (Section 2.2): CSC.  offsets[V+1] (uint32) and src[E]
 *    (uint32): the in-edges of v are src[offsets[v] .. offsets[v+1]) (any
 *    order within a destination); w[E] (uint32, SSSP only) in the same
 *    order.  E < 2^32-256.  wedge_graph_create checks offsets and source
 *    ids on the device and rejects malformed input.
 *  - A chunk is 32 consecutive CSC positions: chunk c holds positions
 *    32c .. 32c+31 (the last one may be short).  With precision k
 *    (log2_coarsen, 0..7) one Wedge Frontier bit / list entry b stands for
 *    the 2^k chunks b*2^k .. b*2^k + 2^k - 1, i.e. 32*2^k edges
 *    (Section 3.4, "Frontier Precision").  k may also be -1 or -2, passed
 *    as uint32 (0xFFFFFFFF, 0xFFFFFFFE): entries of 16 or 8 consecutive
 *    positions (b*16 .., b*8 ..), the paper's finer settings; the first use
 *    builds an edge index in 8-edge units (4 bytes per distinct source and
 *    unit) and grows the Wedge bitmap and list to 8-edge entries.
 *    NC = ceil(E/32); a list at precision k holds up to ceil(E / (32*2^k))
 *    entries.
 *  - Vertex bitmaps are uint32 words, bit (v & 31) of word v >> 5, with
 *    ceil(V/32) words.
 *  - Pointers: arguments named d_* may point to device memory of the graph's
 *    device or, where stated, to host memory.  Device pointers are BORROWED:
 *    the caller keeps them valid until the stream work that uses them has
 *    finished (for the CSC arrays given to wedge_graph_create: until
 *    wedge_graph_destroy).  The library OWNS the edge index it builds, the
 *    per-chunk metadata and all scratch.  src and w device arrays must be
 *    16-byte aligned.
 *  - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *    Work is enqueued asynchronously on it unless stated otherwise.  A graph
 *    object is not thread-safe: calls that use the same graph must be
 *    ordered (same stream, or synchronised by the caller).
 *  - Errors: every call returns a wedge_status; on failure wedge_last_error()
 *    gives a message (per calling thread).  Nothing aborts or exits.
 *  - Unreached BFS levels and SSSP distances are 0xFFFFFFFF; finite SSSP
 *    distances saturate at 0xFFFFFFFE.
 */
#ifndef WEDGE_H
#define WEDGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WEDGE_OK = 0,
    WEDGE_ERR_INVALID_ARG = 1,   /* bad pointer, size, id or option */
    WEDGE_ERR_OUT_OF_MEMORY = 2, /* a device or pinned allocation failed */
    WEDGE_ERR_CUDA = 3,          /* a CUDA call failed (message has the code) */
    WEDGE_ERR_TIMEOUT = 4,       /* a bounded device wait gave up */
    WEDGE_ERR_NOT_SUPPORTED = 5, /* feature unavailable in this build/device */
    WEDGE_ERR_MAX_ITERS = 6      /* the frontier was still non-empty at max_iters */
} wedge_status;

typedef struct wedge_graph* wedge_graph_t; /* opaque, library-owned */
typedef void* wedge_stream_t;              /* cudaStream_t */

typedef enum { WEDGE_BFS = 0, WEDGE_CC = 1, WEDGE_SSSP = 2, WEDGE_PR = 3 } wedge_app;

/* How the next iteration is chosen after each pull (Section 3.4):
 *  THRESHOLD: Wedge Frontier iff fullness * 10^4 < tau_bp * E, where
 *             fullness = sum of out-degrees of the produced frontier
 *             (Section 5.2, "Frontier Fullness Threshold").
 *  LEARNED:   a small MLP cost model picks dense or sparse-with-k; falls back
 *             to THRESHOLD when no model is loaded.
 *  ALWAYS_DENSE / ALWAYS_SPARSE: never / always transform. */
typedef enum {
    WEDGE_SWITCH_THRESHOLD = 0,
    WEDGE_SWITCH_LEARNED = 1,
    WEDGE_SWITCH_ALWAYS_DENSE = 2,
    WEDGE_SWITCH_ALWAYS_SPARSE = 3
} wedge_switch;

typedef struct {
    uint32_t tau_bp;       /* fullness threshold in basis points of E (100 = 1%) */
    uint32_t log2_coarsen; /* k: one Wedge bit per 32 * 2^k edges, 0..7, or -1 / -2
                            * (as uint32) for 16 / 8 edges; batched runs list whole
                            * chunks (-1 / -2 act as 0 there) */
    uint32_t switch_mode;  /* wedge_switch */
    uint32_t max_iters;    /* 0 = default (2^20) */
    uint32_t trace;        /* nonzero: keep per-iteration records for wedge_get_trace */
    uint32_t synchronous;  /* CC/SSSP: nonzero = every pull reads the values of the
                            * previous iteration (double buffer, host-driven loop)
                            * instead of the in-place updates that let values
                            * move several hops per iteration (Section 5.2,
                            * "Frontier Precision"); iteration counts and traces
                            * then follow the synchronous definition exactly.
                            * BFS is level-synchronous either way. */
    uint32_t sparse_push;  /* nonzero: the push/pull hybrid instead of Wedge - a
                            * comparison engine, the analogue of the push-based and
                            * hybrid systems the paper measures against (Section
                            * 5.4; push vs. pull: Section 2.1): iterations the
                            * fullness test finds sparse push
                            * over the frontier's out-edges (an out-edge CSR is
                            * built on the graph's first such run: about 8E + 16V
                            * bytes more, 12E + 16V with weights), dense ones
                            * pull over all edges.
                            * log2_coarsen is ignored; LEARNED acts as THRESHOLD;
                            * not with `synchronous`. */
    uint32_t reserved[1];  /* must be zero */
} wedge_opts;

/* Defaults from the paper's tuned settings (Section 5.2, "Frontier Fullness
 * Threshold" and "Frontier Precision"): BFS tau = 1% with 8 edge vectors per
 * bit, CC/SSSP tau = 20% with 4 vectors per bit.  A vector holds up to 4
 * edges of one destination (Section 2.2), so a bit covers up to 32 / 16
 * edges: k = 0 (one 32-edge chunk) for BFS, k = -1 (16-edge entries) for CC
 * and SSSP. */
void wedge_default_opts(wedge_app app, wedge_opts* out);

typedef struct {
    uint32_t iters;           /* pull iterations executed */
    uint32_t sparse_iters;    /* of which pulled over a Wedge Frontier (hybrid: pushed) */
    uint64_t edges_pulled;    /* CSC positions loaded by the pulls (hybrid: plus the
                               * out-edges pushed, the fullness of pushed frontiers) */
    uint64_t chunks_listed;   /* Wedge Frontier entries over the run */
    double device_ms;         /* stream time of the run (CUDA events) */
} wedge_stats;

/* One record per iteration t of the last run (when opts.trace was set). */
typedef struct {
    uint64_t fullness;  /* sum of out-degrees of the frontier F_t pulled at t */
    uint32_t nfront;    /* |F_t| */
    uint32_t mode;      /* 0 = dense pull, 1 = pull over the Wedge Frontier */
    uint32_t log2_coarsen; /* precision of the entries (as in wedge_opts) */
    uint32_t nchunks;   /* Wedge Frontier entries pulled at t (mode 1) */
    uint32_t rowsum;    /* sum over F_t of edge-index row lengths (chunks at k=0) */
    uint32_t npieces;   /* work pieces handed to the transformation (0 when it
                         * expanded the listed rows directly: frontier listed
                         * completely, every row <= 32 entries, k >= 0) */
    uint64_t t_pull_ns; /* device time of the pull (globaltimer), 0 if unknown */
    uint64_t t_xform_ns;/* device time of the transformation feeding t */
} wedge_iter_record;

/* Builds a graph object on the current CUDA device.
 *  V >= 1 vertices, E >= 0 edges; d_offsets (V+1), d_src (E) and d_w (E, or
 *  NULL when the graph has no weights) in CSC layout (see above).  They may
 *  be host or device pointers; host arrays are copied into library-owned
 *  device memory, device arrays are borrowed.
 *  d_eidx_off / d_eidx: the edge index of Sections 3.3 and 4 (a CSR keyed by
 *  source whose row u lists, once each, the chunks holding u's out-edges,
 *  in any order), or both NULL to have the library build it on the device.
 *  A caller's index is checked for non-decreasing offsets and entries
 *  < NC; rows that list the wrong chunks give wrong results, not faults.
 *  chunk_edges must be 32.
 *  The weights are not read here: device weights only have to be in place
 *  (stream-ordered) before the first SSSP run and the first run with
 *  `sparse_push`, so their upload may overlap the graph's construction.
 *  Synchronises `stream` before returning.  Errors: INVALID_ARG (sizes,
 *  NULL arrays, unaligned device src/w, chunk_edges != 32), OUT_OF_MEMORY,
 *  CUDA. */
wedge_status wedge_graph_create(uint32_t V, uint64_t E, const uint32_t* d_offsets,
                                const uint32_t* d_src, const uint32_t* d_w,
                                const uint32_t* d_eidx_off, const uint32_t* d_eidx,
                                uint32_t chunk_edges, wedge_stream_t stream, wedge_graph_t* out);

/* Kernel schedule of a graph's pulls (chosen by an autotuner; results do
 * not depend on it).
 *  dense_loader: 0 = each warp streams its 256-edge slice with 16-byte
 *                loads that bypass L1 (default: L1 stays free for the
 *                gathered vertex values);
 *                1 = a producer warp per block stages 2048-edge tiles in
 *                shared memory with 1D bulk copies (TMA) through a 4-stage
 *                mbarrier pipeline.
 *  blocks_per_sm: pull blocks per SM, 0 = as many as fit.
 *  edge_index:   0 = the transformation reads the plain edge index (4
 *                bytes per entry);
 *                1 = it reads the compressed edge index (Section 4 names
 *                in-memory compression of the index as a way to cut the
 *                transformation's memory traffic): each row in ascending
 *                order, cut into blocks of up to 32 entries that store the
 *                first entry and the differences between consecutive
 *                entries at the block's fewest bits.  Built on the device
 *                the first time it is asked for (synchronously; about
 *                8 bytes per block of 32 entries plus the packed bits, see
 *                wedge_graph_info.eidx_z_bytes); needs ceil(E/32) < 2^27.
 *                Batched runs, the push/pull hybrid and the paper's
 *                transformation schedule keep the plain index.
 * Changing it drops the graph's cached device-loop graphs. */
typedef struct {
    uint32_t dense_loader;
    uint32_t blocks_per_sm;
    uint32_t edge_index;
    uint32_t reserved[5]; /* must be zero */
} wedge_tuning;

wedge_status wedge_graph_set_tuning(wedge_graph_t g, const wedge_tuning* t);
wedge_status wedge_graph_get_tuning(wedge_graph_t g, wedge_tuning* out);

/* Frees everything the library owns for g (waits for the device first). */
wedge_status wedge_graph_destroy(wedge_graph_t g);

typedef struct {
    uint32_t V;
    uint32_t nz_dst;      /* vertices with in-degree > 0 */
    uint64_t E;
    uint64_t nchunks;     /* NC = ceil(E/32) */
    uint64_t eidx_len;    /* edge-index entries */
    uint64_t device_bytes;/* device memory owned by the object */
    int device;
    uint64_t eidx_bytes;  /* the plain edge index: 4(V+1) + 4 * eidx_len */
    uint64_t eidx_z_bytes;/* the compressed edge index (block headers, packed
                           * differences, first block of each row); 0 until
                           * built (wedge_tuning.edge_index) */
    uint64_t eidx_z_blocks;/* its blocks (0 until built) */
    uint64_t eidx_z_words; /* its packed 32-bit words (0 until built) */
} wedge_graph_info;

wedge_status wedge_graph_get_info(wedge_graph_t g, wedge_graph_info* out);

/* Copies the edge index (eidx_off[V+1], eidx[eidx_len]) into device
 * buffers provided by the caller. */
wedge_status wedge_graph_copy_edge_index(wedge_graph_t g, uint32_t* d_eidx_off, uint32_t* d_eidx,
                                         wedge_stream_t stream);

/* Copies the compressed edge index (built by wedge_graph_set_tuning with
 * edge_index = 1) into device buffers of the caller: d_zbo[V+1] (first block
 * of each row; row u's blocks hold its eidx_len entries in ascending order,
 * 32 per block, the last one ragged), d_zhdr[2 * eidx_z_blocks] (per block:
 * first entry | w << 27, index of its first word) and
 * d_zwords[eidx_z_words] (entry i >= 1 of a block minus entry i-1, in w
 * bits at bit (i-1)*w of the block's words, little-endian).
 * Errors: INVALID_ARG (NULL, index not built), CUDA. */
wedge_status wedge_graph_copy_edge_index_z(wedge_graph_t g, uint32_t* d_zbo, uint32_t* d_zhdr, uint32_t* d_zwords,
                                           wedge_stream_t stream);

/* The frontier transformation (Sections 3.3, 4): from the vertex frontier
 * d_vertex_bitmap (ceil(V/32) words, device) to the Wedge Frontier at
 * precision log2_coarsen, written as a list of entries b (each standing for
 * chunks b*2^k .. b*2^k+2^k-1, or for 16 / 8 positions at k = -1 / -2) into
 * d_chunk_list (device, capacity ceil(E / (32*2^k))) with the count in
 * *d_chunk_count (device).  Entries are
 * distinct; their order is unspecified.  Errors: INVALID_ARG, CUDA. */
wedge_status wedge_frontier_transform(wedge_graph_t g, const uint32_t* d_vertex_bitmap,
                                      uint32_t log2_coarsen, uint32_t* d_chunk_list,
                                      uint32_t* d_chunk_count, wedge_stream_t stream);

/* Load balance of the frontier transformation (Section 4, "Parallelization";
 * Section 5.3 and Fig. 13, which measure the time threads spend idle at the
 * transformation's barrier).  Runs the transformation of
 * wedge_frontier_transform (same arguments and output) under one of two
 * schedules and records, for every warp of the launch and each kernel, the
 * warp's start and end on the device's global timer and its busy SM cycles:
 *  schedule 0: the library's (wedge_frontier_transform): kernel 0 cuts the
 *              active vertices' edge-index rows into pieces of at most 32
 *              entries, kernel 1 expands them with the pieces balanced over
 *              the warps;
 *  schedule 1: the paper's: the vertex frontier is cut into equal pieces of
 *              256 vertices, each taken by the next free warp, which walks
 *              every row of its piece's active vertices (kernel 0 only;
 *              kernel 1's records stay zero).
 * d_warp_stats (device): 8 uint64 per warp w, {start ns, end ns, busy SM
 * cycles, SM id} of kernel 0 at [8w .. 8w+3] and of kernel 1 at
 * [8w+4 .. 8w+7].  A warp is busy from its start to the end of its last
 * piece and idle from then to the end of the kernel (the barrier).
 * *n_warps (host) = the launch's warps; with d_warp_stats = NULL only
 * *n_warps is set.  cap_warps: warps d_warp_stats holds (>= *n_warps).
 * Errors: INVALID_ARG (NULL, schedule > 1, cap_warps too small,
 * log2_coarsen > 7), CUDA. */
wedge_status wedge_frontier_transform_profile(wedge_graph_t g, const uint32_t* d_vertex_bitmap,
                                              uint32_t log2_coarsen, uint32_t schedule, uint32_t* d_chunk_list,
                                              uint32_t* d_chunk_count, uint64_t* d_warp_stats, uint32_t cap_warps,
                                              uint32_t* n_warps, wedge_stream_t stream);

/* The frontier transformation without any memory allocation.  The paper has
 * no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (a framework that owns all device memory through its own pool,
 * latency-critical loops, deployments whose device footprint is fixed at
 * load time).  It needs no graph object: the caller passes the edge index
 * (d_eidx_off[V+1], d_eidx: chunk ids of each source's out-edges, as built
 * by wedge_graph_create or given to it), the vertex bitmap, and the output
 * list (capacity ceil(ceil(E/32) / 2^k)) and count, all device memory.
 * Output: as wedge_frontier_transform (distinct entries, unspecified order).
 * The duplicate-removing bitmap lives in a fixed 4 MiB device array that
 * every GPU loading the library holds until the process exits; graphs with
 * ceil(ceil(E/32) / 2^k) > 2^25 are rejected with INVALID_ARG.  The first call
 * on a device looks up that array's address; make that first call before
 * any stream capture.  All calls on a device share the array (each clears
 * the part it uses), so calls that overlap on the GPU race.
 * Errors: INVALID_ARG, NOT_SUPPORTED (device index >= 64), CUDA. */
wedge_status wedge_frontier_transform_noalloc(uint32_t V, uint64_t E, const uint32_t* d_eidx_off,
                                              const uint32_t* d_eidx, const uint32_t* d_vertex_bitmap,
                                              uint32_t log2_coarsen, uint32_t* d_chunk_list,
                                              uint32_t* d_chunk_count, wedge_stream_t stream);

/* One pull iteration of BFS, CC or SSSP (Sections 2.1, 3.2, 5):
 *  d_values (V, device) is updated in place: BFS levels, CC labels or SSSP
 *  distances.  iter is the iteration number (BFS gives level iter+1 to newly
 *  reached vertices).  d_cur_bitmap: the frontier consumed (BFS only; NULL
 *  otherwise).  d_chunk_list / d_chunk_count: the Wedge Frontier to pull
 *  over at coarsening log2_coarsen, or d_chunk_list = NULL for a dense pull
 *  over all edges; entries must be distinct, entries >= ceil(E/(32*2^k)) are
 *  ignored and the count is clamped to ceil(E/(32*2^k)).  Outputs: bits of the vertices whose value changed are
 *  ORed into d_next_bitmap (device, ceil(V/32) words; the caller zeroes it),
 *  *d_fullness (device uint64) = sum of their out-degrees, *d_nfront
 *  (device) = their number.
 *  CC and SSSP update values in place with atomic minima, so a value may
 *  move more than one hop in an iteration (Section 5.2, "Frontier
 *  Precision"); the fixed point reached is the same.  Errors: INVALID_ARG,
 *  CUDA. */
wedge_status wedge_pull_iterate(wedge_graph_t g, wedge_app app, uint32_t* d_values, uint32_t iter,
                                const uint32_t* d_cur_bitmap, const uint32_t* d_chunk_list,
                                const uint32_t* d_chunk_count, uint32_t log2_coarsen,
                                uint32_t* d_next_bitmap, uint64_t* d_fullness, uint32_t* d_nfront,
                                wedge_stream_t stream);

/* Whole applications (Section 5, "Applications"), each iterating pull,
 * fullness decision and transformation on the device until the frontier
 * is empty.  Outputs may be device or host pointers (host: copied back
 * before the call returns).  opts may be NULL for wedge_default_opts.
 * stats (host, may be NULL): when given, the call synchronises the stream
 * and fills it.  Errors: INVALID_ARG (root >= V, no weights for SSSP),
 * MAX_ITERS, TIMEOUT, CUDA. */
wedge_status wedge_run_bfs(wedge_graph_t g, uint32_t root, uint32_t* d_level,
                           const wedge_opts* opts, wedge_stats* stats, wedge_stream_t stream);
/* CC labels: smallest vertex id of the component; the graph must be
 * symmetric (every edge present in both directions) for HCC to give
 * components. */
wedge_status wedge_run_cc(wedge_graph_t g, uint32_t* d_label, const wedge_opts* opts,
                          wedge_stats* stats, wedge_stream_t stream);
wedge_status wedge_run_sssp(wedge_graph_t g, uint32_t root, uint32_t* d_dist,
                            const wedge_opts* opts, wedge_stats* stats, wedge_stream_t stream);
/* PageRank (named in Section 1; no frontier): pr0 = 1/V and `iters` times
 * pr'(v) = (1-d)/V + d * (sum_{u->v} pr(u)/outdeg(u) + D/V), D = rank of
 * vertices with out-degree 0.  FP32 values; in-edge sums are accumulated
 * exactly in 64-bit fixed point (2^-62 units), so results do not depend
 * on the schedule.  The pulls gather the contributions in the order of
 * descending out-degree (built on the graph's first PageRank call: 4E + 4V
 * bytes, a device radix sort of V keys), so the most gathered ones share
 * cache lines; results are in the graph's own vertex ids. */
wedge_status wedge_run_pr(wedge_graph_t g, float* d_rank, uint32_t iters, float damping,
                          const wedge_opts* opts, wedge_stats* stats, wedge_stream_t stream);
/* The in-edge pass of one PageRank iteration on its own (the dense pull of
 * Sections 2.1 and 3.2 with PageRank's sum): on return
 *   d_sums[v] = sum over in-edges (u, v) of round(d_contrib[u] * 2^62),
 * an exact 64-bit fixed-point sum (1.0 = 2^62) that does not depend on the
 * schedule.  d_contrib: V floats (device), finite, >= 0, and small enough
 * that every sum stays below 4.0 (pr(u)/outdeg(u) always is); not checked.
 * d_sums: V uint64 (device), must hold zeros on entry; vertices without
 * in-edges keep 0.  Runs the pull of wedge_run_pr (the contributions are
 * first copied into its gather order, in library memory that a concurrent
 * wedge_run_pr on the same graph also uses).  Asynchronous on stream.
 * Errors: INVALID_ARG, OUT_OF_MEMORY (first call), CUDA. */
wedge_status wedge_pr_pull(wedge_graph_t g, const float* d_contrib, uint64_t* d_sums, wedge_stream_t stream);
/* PageRank's gather order: d_order[v] (device, V uint32) = the position of
 * vertex v's contribution in the array the pulls gather from (v's rank by
 * descending out-degree, ties by id; built on first use).  Stream-ordered.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
wedge_status wedge_pr_order(wedge_graph_t g, uint32_t* d_order, wedge_stream_t stream);
/* wedge_pr_pull on contributions already in the gather order:
 * d_contrib[d_order[u]] holds u's contribution.  The pull of wedge_run_pr
 * alone, with no copy; same sums, conditions and errors as wedge_pr_pull. */
wedge_status wedge_pr_pull_ordered(wedge_graph_t g, const float* d_contrib, uint64_t* d_sums,
                                   wedge_stream_t stream);
/* ---- Learned switch (not in the paper) --------------------------------
 * A cost model replaces the fixed fullness threshold and the fixed
 * precision of Section 3.4: before each pull it predicts ln(milliseconds)
 * of the iteration under each candidate (dense pull; Wedge Frontier at
 * k = 0..4) and the lowest prediction wins (WEDGE_SWITCH_LEARNED).  Model:
 * 12 features -> 64 ReLU -> 64 ReLU -> 1; parameters as one FP32 array of
 * WEDGE_MLP_PARAMS floats laid out W1[64][12] | b1[64] | W2[64][64] | b2[64]
 * | w3[64] | b3.  Features (per candidate): log2(|F|+1)/32,
 * log2(fullness+1)/32, fullness/E, log2(edge-index row sum+1)/32, log2(V)/32,
 * log2(E)/32, (E/V)/64, log2(1+max/mean out-degree)/16, t/(t+8), app (BFS 0,
 * CC 0.5, SSSP 1), is_sparse, k/4. */
#define WEDGE_MLP_FEATURES 12
#define WEDGE_MLP_PARAMS 5057
#define WEDGE_MLP_CANDIDATES 6

/* FP32 forward on n rows (d_x row-major n x 12) into d_y (n); device memory. */
wedge_status wedge_mlp_forward(const float* d_params, const float* d_x, uint32_t n, float* d_y,
                               wedge_stream_t stream);
/* The same model as the decision evaluates it: BF16 copy of the weights,
 * BF16 activations, FP32 accumulation.  Synchronises the stream. */
wedge_status wedge_mlp_forward_bf16(const float* d_params, const float* d_x, uint32_t n, float* d_y,
                                    wedge_stream_t stream);
/* *d_loss = mean_i (f(x_i) - t_i)^2 and d_grad (5057) = its gradient with
 * respect to the parameters (FP32, device memory). */
wedge_status wedge_mlp_loss_grad(const float* d_params, const float* d_x, const float* d_t, uint32_t n,
                                 float* d_grad, float* d_loss, wedge_stream_t stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step t >= 1) on d_params
 * with moment buffers d_m, d_v (5057 floats each, start at zero). */
wedge_status wedge_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, uint32_t t, float lr,
                            wedge_stream_t stream);
/* Installs (params != NULL, host or device FP32) or removes the cost model
 * used by WEDGE_SWITCH_LEARNED on g; without one the threshold decides. */
wedge_status wedge_set_cost_model(wedge_graph_t g, const float* params);
/* The band of fullness / E (the share of edges the frontier's out-edges
 * make up) inside which WEDGE_SWITCH_LEARNED evaluates the cost model on g;
 * below lo it takes the Wedge Frontier at k = 0, above hi a dense pull,
 * without inference (the band is learned from the training traces: outside
 * it every traced iteration's fastest candidate was that one).  Default
 * [0, 3e38]: always evaluate.  Errors: INVALID_ARG (lo < 0, hi < lo). */
wedge_status wedge_set_learned_band(wedge_graph_t g, float lo, float hi);
/* Training traces: runs app (BFS, CC, SSSP) from root with the threshold
 * policy of opts (log2_coarsen <= 4), and before every pull t (t < cap and
 * t < max_iters, 0 = no limit) times each candidate c (transformation +
 * pull, from the same saved state) into h_ms[t*6+c], with its features in
 * h_features[(t*6+c)*12 ..], and the threshold's choice in h_chosen[t]
 * (0 dense, 1+k sparse).  Host outputs; synchronous.  *n_iters = rows. */
wedge_status wedge_trace_candidates(wedge_graph_t g, wedge_app app, uint32_t root, const wedge_opts* opts,
                                    uint32_t max_iters, float* h_features, float* h_ms, uint32_t* h_chosen,
                                    uint32_t cap, uint32_t* n_iters, wedge_stream_t stream);

/* ---- Batched BFS (not in the paper) ------------------------------------
 * Up to 64 BFS queries in one run (multi-source BFS): each vertex carries a
 * 64-bit mask of the queries that reached it and of those for which it is in
 * the current frontier.  The union of the queries' frontiers drives the
 * fullness decision and the Wedge Frontier (Sections 3.3, 3.4), so every
 * pull serves all queries.  The loop runs in one persistent cooperative
 * launch (bounded grid barriers), captured in a CUDA graph per
 * (queries, roots, output, options).
 *  roots[nroots] (host or device) with root_query[nroots] giving the query
 *  of each root (NULL: root i is query i); several roots may share a query
 *  (a query's level is then the distance to the nearest of its roots, as
 *  for graphs concatenated block-diagonally, one root per graph).
 *  d_levels (device, V * nqueries uint32): vertex-major,
 *  d_levels[v * nqueries + q] = hop distance of v from query q's roots
 *  (0xFFFFFFFF if unreached).  opts as for wedge_run_bfs (learned switch
 *  not used).  Errors: INVALID_ARG (ids, sizes, host output), TIMEOUT,
 *  MAX_ITERS (when stats != NULL), CUDA. */
wedge_status wedge_run_bfs_batch(wedge_graph_t g, const uint32_t* roots, const uint32_t* root_query,
                                 uint32_t nroots, uint32_t nqueries, uint32_t* d_levels,
                                 const wedge_opts* opts, wedge_stats* stats, wedge_stream_t stream);

/* wedge_run_bfs_batch with 8-bit levels: d_levels (device, V * nqueries
 * bytes, vertex-major) receives each hop distance as one byte, 0xFF if
 * unreached -- a quarter of the 32-bit output's memory and writes, for
 * queries whose levels stay below 255.  A pull that reaches a vertex at
 * level 255 or more writes nothing for it and stops the run; the call then
 * returns NOT_SUPPORTED (the levels below 255 are written and exact; use
 * the 32-bit call).  The call waits for the run to end (it reads that check
 * back).  Other arguments and errors as above. */
wedge_status wedge_run_bfs_batch_u8(wedge_graph_t g, const uint32_t* roots, const uint32_t* root_query,
                                    uint32_t nroots, uint32_t nqueries, uint8_t* d_levels,
                                    const wedge_opts* opts, wedge_stats* stats, wedge_stream_t stream);

/* Batched SSSP (not in the paper): up to 64 single-source shortest-path
 * queries in one run (multi-source Bellman-Ford), with the arguments,
 * layout and errors of wedge_run_bfs_batch:
 *  d_dist[v * nqueries + q] = distance of v from query q's nearest root
 *  (weights, saturation at 0xFFFFFFFE and 0xFFFFFFFF for unreached as in
 *  wedge_run_sssp).  Each vertex carries a 64-bit mask of the queries whose
 *  distance it improved in the last iteration; the union of those masks is
 *  the frontier that drives the fullness decision and the Wedge Frontier
 *  (Sections 3.3, 3.4).  Distances improve in place (atomic minima).
 *  INVALID_ARG also when g has no weights. */
wedge_status wedge_run_sssp_batch(wedge_graph_t g, const uint32_t* roots, const uint32_t* root_query,
                                  uint32_t nroots, uint32_t nqueries, uint32_t* d_dist,
                                  const wedge_opts* opts, wedge_stats* stats, wedge_stream_t stream);

/* Per-iteration records of the last run of g (needs opts.trace).  Copies up
 * to cap records into host memory, sets *n to the number available.
 * Synchronises the stream of that run. */
wedge_status wedge_get_trace(wedge_graph_t g, wedge_iter_record* out, uint32_t cap, uint32_t* n);

/* Degree-ordered relabelling (not in the paper; a locality step before
 * wedge_graph_create).  Every pull gathers one value per in-edge, indexed by
 * the edge's source; new ids that follow descending out-degree put the most
 * gathered values on shared cache lines.  New vertex i is old vertex
 * old_of_new[i], the i-th by descending out-degree, ties by ascending old
 * id; its in-edges are old_of_new[i]'s in their original order, each source
 * u renamed new_of_old[u] (weights carried along).
 *  In (device): d_offsets[V+1], d_src[E], d_w[E] or NULL, a CSC as above.
 *  Out (device, caller-owned, not overlapping the inputs): d_new_offsets[V+1],
 *  d_new_src[E], d_new_w[E] (NULL exactly when d_w is), d_new_of_old[V],
 *  d_old_of_new[V] (or NULL).
 *  Validates like wedge_graph_create (offsets, source ids) and synchronises
 *  `stream` once to read the result; the rest is stream-ordered.  Device
 *  scratch of about 28 (V+1) + E/256 bytes comes from the library's pool.
 *  Errors: INVALID_ARG (V == 0, E too large, NULL or host arrays, malformed
 *  CSC), OUT_OF_MEMORY, CUDA. */
wedge_status wedge_csc_relabel_by_degree(uint32_t V, uint64_t E, const uint32_t* d_offsets,
                                         const uint32_t* d_src, const uint32_t* d_w,
                                         uint32_t* d_new_offsets, uint32_t* d_new_src,
                                         uint32_t* d_new_w, uint32_t* d_new_of_old,
                                         uint32_t* d_old_of_new, wedge_stream_t stream);

/* Results of a relabelled graph back in the original ids:
 * d_out[v * width + c] = d_in[new_of_old[v] * width + c] for v < V, c < width
 * (width 1: levels, distances, PageRank values as 32-bit words; width Q:
 * the vertex-major rows of a batched run).  Device arrays, d_in != d_out;
 * stream-ordered.  Errors: INVALID_ARG, CUDA. */
wedge_status wedge_permute_rows(uint32_t V, uint32_t width, const uint32_t* d_new_of_old,
                                const uint32_t* d_in, uint32_t* d_out, wedge_stream_t stream);

/* Component labels of a relabelled graph back in the original ids.  A CC
 * label names the smallest vertex id of its component; after a relabelling
 * that is a new id, so this takes, per component, the smallest old id:
 * d_out[old_of_new[i]] = min { old_of_new[j] : d_labels[j] == d_labels[i] }.
 * d_scratch[V] is overwritten; all device arrays, pairwise distinct;
 * labels >= V (which no CC run produces) are copied unchanged.
 * Stream-ordered.  Errors: INVALID_ARG, CUDA. */
wedge_status wedge_cc_labels_to_original(uint32_t V, const uint32_t* d_old_of_new,
                                         const uint32_t* d_labels, uint32_t* d_scratch,
                                         uint32_t* d_out, wedge_stream_t stream);

/* Self-test of the bounded device waits (not in the paper).  Every wait in
 * the library's kernels -- mbarrier phases of the staged pull, the grid
 * barrier of the batched traversal -- gives up after 200 ms of device time
 * and records a timeout that the call returns as WEDGE_ERR_TIMEOUT, leaving
 * the device usable.  This runs one such wait that can never be satisfied
 * on the current device: kind 0 = an mbarrier that receives one of two
 * arrivals, kind 1 = a two-block grid barrier that one block never reaches.
 * Synchronous.  Returns WEDGE_ERR_TIMEOUT when the wait gave up as it must
 * (WEDGE_OK would mean it did not); INVALID_ARG for another kind; CUDA. */
wedge_status wedge_selftest_timeout(int kind);

/* Number of kernel launches the library has enqueued since load (for
 * accounting of device work). */
uint64_t wedge_kernel_launches(void);

/* Device memory of the library (graphs, their scratch) comes from one
 * memory pool per GPU that keeps what destroyed graphs release, so a new
 * graph maps no new memory.  This returns the kept memory of `device`
 * (-1: every GPU) to the driver.  Memory of live graphs is not touched.
 * Errors: INVALID_ARG (device < -1), CUDA. */
wedge_status wedge_trim_memory(int device);

const char* wedge_last_error(void);
const char* wedge_version(void);

#ifdef __cplusplus
}
#endif
#endif /* WEDGE_H */

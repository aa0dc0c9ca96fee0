/*
 * Oracle for the Wedge hot path: a plain, slow, single-threaded CPU
 * restatement of what the engine computes, written from the paper
 * (Grossman & Kozyrakis, "A New Frontier for Pull-Based Graph Processing",
 * arXiv 1903.07754).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  It shares nothing
 * with the CUDA engine (no headers, helpers or tables) and the engine never
 * calls it.
 *
 * Graph input (as the engine's boundary takes it, Section 2.2): CSC with
 * off[V+1] and src[E]; the in-edges of v are src[off[v] .. off[v+1]), and
 * w[E] (optional) holds SSSP weights in the same order.  Unreached BFS levels
 * and SSSP distances are 0xFFFFFFFF.
 *
 * Readings of the paper used here (the paper is silent on these):
 *  - SSSP additions saturate at 0xFFFFFFFE so that a finite distance never
 *    becomes the "unreached" value.
 *  - CC is HCC label propagation (Section 5, "Applications") run on an
 *    undirected (symmetrised) input, so the fixed point labels every vertex
 *    with the smallest id in its component.
 *  - PageRank (named in Section 1 and excluded from the paper's evaluation in
 *    Section 5) uses the textbook iterate: pr0 = 1/V and
 *    pr'(v) = (1-d)/V + d * (sum_{u->v} pr(u)/outdeg(u) + D/V), with D the
 *    rank held by vertices of out-degree 0, spread uniformly.
 *  - The fullness test sends the next iteration to the Wedge Frontier iff
 *    fullness * 10^4 < tau_bp * E (tau in basis points of |E|, strict "<").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define INF32 0xFFFFFFFFu
#define SAT32 0xFFFFFFFEu

enum { OR_BFS = 0, OR_CC = 1, OR_SSSP = 2 };
enum { OR_MODE_DENSE = 0, OR_MODE_SPARSE = 1 };
enum { OR_POLICY_THRESHOLD = 0, OR_POLICY_ALWAYS_DENSE = 1, OR_POLICY_ALWAYS_SPARSE = 2 };

/* ------------------------------------------------------------------ */
/* Out-edge view (CSR) of the CSC, by a counting sort over sources.     */
/* Row u lists u's out-edges in increasing CSC position (so in          */
/* increasing destination id); pos[j] is that CSC position.             */
/* Section 2.2: CSR holds out-edges, CSC in-edges.                       */
/* ------------------------------------------------------------------ */
void or_csc_to_csr(uint32_t V, uint64_t E, const uint32_t* off, const uint32_t* src,
                   uint64_t* csr_off, uint32_t* csr_dst, uint64_t* csr_pos) {
    uint64_t* fill = (uint64_t*)calloc((size_t)V + 1, sizeof(uint64_t));
    memset(csr_off, 0, sizeof(uint64_t) * ((size_t)V + 1));
    for (uint64_t p = 0; p < E; ++p) csr_off[src[p] + 1]++;
    for (uint32_t u = 0; u < V; ++u) csr_off[u + 1] += csr_off[u];
    for (uint32_t v = 0; v < V; ++v)
        for (uint64_t p = off[v]; p < off[v + 1]; ++p) {
            uint32_t u = src[p];
            uint64_t j = csr_off[u] + fill[u]++;
            csr_dst[j] = v;
            if (csr_pos) csr_pos[j] = p;
        }
    free(fill);
}

/* Out-degree of every vertex. */
void or_outdeg(uint32_t V, uint64_t E, const uint32_t* src, uint32_t* outdeg) {
    memset(outdeg, 0, sizeof(uint32_t) * V);
    for (uint64_t p = 0; p < E; ++p) outdeg[src[p]]++;
}

/* ------------------------------------------------------------------ */
/* BFS with a FIFO queue over out-edges: the push pattern of Section     */
/* 2.1 driven by a source-oriented frontier (Section 1).                */
/* ------------------------------------------------------------------ */
void or_bfs_push(uint32_t V, const uint64_t* csr_off, const uint32_t* csr_dst, uint32_t root,
                 uint32_t* level) {
    uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * (V ? V : 1));
    for (uint32_t v = 0; v < V; ++v) level[v] = INF32;
    if (root >= V) {
        free(queue);
        return;
    }
    uint64_t head = 0, tail = 0;
    level[root] = 0;
    queue[tail++] = root;
    while (head < tail) {
        uint32_t u = queue[head++];
        for (uint64_t j = csr_off[u]; j < csr_off[u + 1]; ++j) {
            uint32_t v = csr_dst[j];
            if (level[v] == INF32) {
                level[v] = level[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
}

/* ------------------------------------------------------------------ */
/* Connected components by union-find (union by rank, path halving);    */
/* label = smallest vertex id of the set.  Treats every edge as         */
/* undirected.                                                          */
/* ------------------------------------------------------------------ */
static uint32_t uf_find(uint32_t* parent, uint32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

void or_cc_union_find(uint32_t V, const uint32_t* off, const uint32_t* src, uint32_t* label) {
    uint32_t* parent = (uint32_t*)malloc(sizeof(uint32_t) * (V ? V : 1));
    uint8_t* rank = (uint8_t*)calloc(V ? V : 1, 1);
    uint32_t* minid = (uint32_t*)malloc(sizeof(uint32_t) * (V ? V : 1));
    for (uint32_t v = 0; v < V; ++v) parent[v] = v;
    for (uint32_t v = 0; v < V; ++v)
        for (uint64_t p = off[v]; p < off[v + 1]; ++p) {
            uint32_t a = uf_find(parent, v), b = uf_find(parent, src[p]);
            if (a == b) continue;
            if (rank[a] < rank[b]) {
                uint32_t t = a;
                a = b;
                b = t;
            }
            parent[b] = a;
            if (rank[a] == rank[b]) rank[a]++;
        }
    for (uint32_t v = 0; v < V; ++v) minid[v] = INF32;
    for (uint32_t v = 0; v < V; ++v) {
        uint32_t r = uf_find(parent, v);
        if (v < minid[r]) minid[r] = v;
    }
    for (uint32_t v = 0; v < V; ++v) label[v] = minid[uf_find(parent, v)];
    free(parent);
    free(rank);
    free(minid);
}

/* ------------------------------------------------------------------ */
/* SSSP by Dijkstra with a binary heap (lazy deletion) over out-edges.  */
/* ------------------------------------------------------------------ */
typedef struct {
    uint64_t d;
    uint32_t v;
} heap_item;

static void heap_push(heap_item* h, uint64_t* n, heap_item x) {
    uint64_t i = (*n)++;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h[p].d <= x.d) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = x;
}

static heap_item heap_pop(heap_item* h, uint64_t* n) {
    heap_item top = h[0], last = h[--(*n)];
    uint64_t i = 0;
    for (;;) {
        uint64_t c = 2 * i + 1;
        if (c >= *n) break;
        if (c + 1 < *n && h[c + 1].d < h[c].d) c++;
        if (last.d <= h[c].d) break;
        h[i] = h[c];
        i = c;
    }
    h[i] = last;
    return top;
}

void or_sssp_dijkstra(uint32_t V, uint64_t E, const uint64_t* csr_off, const uint32_t* csr_dst,
                      const uint64_t* csr_pos, const uint32_t* w, uint32_t root, uint32_t* dist) {
    for (uint32_t v = 0; v < V; ++v) dist[v] = INF32;
    if (root >= V) return;
    heap_item* h = (heap_item*)malloc(sizeof(heap_item) * (E + 1));
    uint8_t* done = (uint8_t*)calloc(V, 1);
    uint64_t n = 0;
    dist[root] = 0;
    heap_item s = {0, root};
    heap_push(h, &n, s);
    while (n > 0) {
        heap_item it = heap_pop(h, &n);
        uint32_t u = it.v;
        if (done[u]) continue;
        done[u] = 1;
        for (uint64_t j = csr_off[u]; j < csr_off[u + 1]; ++j) {
            uint32_t v = csr_dst[j];
            uint64_t cand = (uint64_t)dist[u] + w[csr_pos[j]];
            if (cand > SAT32) cand = SAT32;
            if (cand < dist[v]) {
                dist[v] = (uint32_t)cand;
                heap_item x = {cand, v};
                heap_push(h, &n, x);
            }
        }
    }
    free(h);
    free(done);
}

/* ------------------------------------------------------------------ */
/* Bellman-Ford, push form: relax the out-edges of the vertices whose   */
/* distance changed in the previous round (Section 2.1, push).          */
/* ------------------------------------------------------------------ */
void or_sssp_push(uint32_t V, const uint64_t* csr_off, const uint32_t* csr_dst,
                  const uint64_t* csr_pos, const uint32_t* w, uint32_t root, uint32_t* dist) {
    uint8_t* active = (uint8_t*)calloc(V ? V : 1, 1);
    uint8_t* next = (uint8_t*)calloc(V ? V : 1, 1);
    for (uint32_t v = 0; v < V; ++v) dist[v] = INF32;
    if (root >= V) goto out;
    dist[root] = 0;
    active[root] = 1;
    for (;;) {
        int any = 0;
        memset(next, 0, V);
        /* synchronous round: read a snapshot of the distances */
        uint32_t* snap = (uint32_t*)malloc(sizeof(uint32_t) * V);
        memcpy(snap, dist, sizeof(uint32_t) * V);
        for (uint32_t u = 0; u < V; ++u) {
            if (!active[u]) continue;
            for (uint64_t j = csr_off[u]; j < csr_off[u + 1]; ++j) {
                uint32_t v = csr_dst[j];
                uint64_t cand = (uint64_t)snap[u] + w[csr_pos[j]];
                if (cand > SAT32) cand = SAT32;
                if (cand < dist[v]) {
                    dist[v] = (uint32_t)cand;
                    next[v] = 1;
                    any = 1;
                }
            }
        }
        free(snap);
        uint8_t* t = active;
        active = next;
        next = t;
        if (!any) break;
    }
out:
    free(active);
    free(next);
}

/* ------------------------------------------------------------------ */
/* PageRank in FP64, pull form (Section 2.1: iterate destinations,       */
/* aggregate in-edges, one write per vertex).                            */
/* ------------------------------------------------------------------ */
void or_pr_pull(uint32_t V, const uint32_t* off, const uint32_t* src, const uint32_t* outdeg,
                double d, uint32_t iters, double* pr) {
    double* contrib = (double*)malloc(sizeof(double) * (V ? V : 1));
    for (uint32_t v = 0; v < V; ++v) pr[v] = 1.0 / V;
    for (uint32_t t = 0; t < iters; ++t) {
        double dangling = 0.0;
        for (uint32_t u = 0; u < V; ++u) {
            if (outdeg[u] == 0) {
                dangling += pr[u];
                contrib[u] = 0.0;
            } else {
                contrib[u] = pr[u] / outdeg[u];
            }
        }
        for (uint32_t v = 0; v < V; ++v) {
            double sum = 0.0;
            for (uint64_t p = off[v]; p < off[v + 1]; ++p) sum += contrib[src[p]];
            pr[v] = (1.0 - d) / V + d * (sum + dangling / V);
        }
    }
    free(contrib);
}

/* The pull's aggregation on its own (Section 2.1): out[v] = sum of x[u]
 * over the in-edges (u, v), in FP64, in CSC order.  PageRank's in-edge pass
 * is this with x[u] = pr(u)/outdeg(u). */
void or_in_sums(uint32_t V, const uint32_t* off, const uint32_t* src, const double* x, double* out) {
    for (uint32_t v = 0; v < V; ++v) {
        double sum = 0.0;
        for (uint64_t p = off[v]; p < off[v + 1]; ++p) sum += x[src[p]];
        out[v] = sum;
    }
}

/* PageRank in FP64, push form: scatter pr(u)/outdeg(u) along out-edges. */
void or_pr_push(uint32_t V, const uint64_t* csr_off, const uint32_t* csr_dst, double d,
                uint32_t iters, double* pr) {
    double* acc = (double*)malloc(sizeof(double) * (V ? V : 1));
    for (uint32_t v = 0; v < V; ++v) pr[v] = 1.0 / V;
    for (uint32_t t = 0; t < iters; ++t) {
        double dangling = 0.0;
        for (uint32_t v = 0; v < V; ++v) acc[v] = 0.0;
        for (uint32_t u = 0; u < V; ++u) {
            uint64_t deg = csr_off[u + 1] - csr_off[u];
            if (deg == 0) {
                dangling += pr[u];
                continue;
            }
            double c = pr[u] / (double)deg;
            for (uint64_t j = csr_off[u]; j < csr_off[u + 1]; ++j) acc[csr_dst[j]] += c;
        }
        for (uint32_t v = 0; v < V; ++v) pr[v] = (1.0 - d) / V + d * (acc[v] + dangling / V);
    }
    free(acc);
}

/* ------------------------------------------------------------------ */
/* Wedge Frontier (Sections 3.3, 3.4 "Frontier Precision", 4).          */
/* Edges are grouped by position in the CSC edge array, `group` edges   */
/* per group (group = 1 is the highest precision).  The Wedge Frontier  */
/* of a source-oriented vertex frontier is the set of groups holding at */
/* least one edge whose source is in that frontier.                     */
/* ------------------------------------------------------------------ */

/* By definition: scan every edge position.  frontier is one byte per vertex.
 * Writes the groups in increasing order; returns their number. */
uint64_t or_wedge_groups_scan(uint64_t E, const uint32_t* src, const uint8_t* frontier,
                              uint64_t group, uint64_t* out) {
    uint64_t n = 0;
    uint64_t last = UINT64_MAX;
    for (uint64_t p = 0; p < E; ++p) {
        if (!frontier[src[p]]) continue;
        uint64_t gidx = p / group;
        if (gidx != last) {
            out[n++] = gidx;
            last = gidx;
        }
    }
    return n;
}

/* Edge index (Sections 3.3 and 4): a CSR keyed by source whose entries are
 * the Wedge Frontier positions (groups of `group` edges) of that source's
 * out-edges, each listed once, in increasing order.  eidx_off has V+1
 * entries; eidx needs at most E entries.  Returns the entry count. */
uint64_t or_edge_index(uint32_t V, uint64_t E, const uint32_t* off, const uint32_t* src,
                       uint64_t group, uint64_t* eidx_off, uint64_t* eidx) {
    uint64_t* csr_off = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)V + 1));
    uint32_t* csr_dst = (uint32_t*)malloc(sizeof(uint32_t) * (E ? E : 1));
    uint64_t* csr_pos = (uint64_t*)malloc(sizeof(uint64_t) * (E ? E : 1));
    or_csc_to_csr(V, E, off, src, csr_off, csr_dst, csr_pos);
    uint64_t n = 0;
    for (uint32_t u = 0; u < V; ++u) {
        eidx_off[u] = n;
        uint64_t last = UINT64_MAX;
        for (uint64_t j = csr_off[u]; j < csr_off[u + 1]; ++j) {
            uint64_t gidx = csr_pos[j] / group; /* csr_pos increases along the row */
            if (gidx != last) {
                eidx[n++] = gidx;
                last = gidx;
            }
        }
    }
    eidx_off[V] = n;
    free(csr_off);
    free(csr_dst);
    free(csr_pos);
    return n;
}

/* The transformation step as the paper describes it (Section 4): for every
 * vertex set in the traditional frontier, walk its edge-index row and set the
 * listed bits of a bit-mask with one bit per group; then list the set bits in
 * order.  ngroups = ceil(E / group).  Returns the number listed. */
uint64_t or_wedge_groups_index(uint32_t V, const uint64_t* eidx_off, const uint64_t* eidx,
                               const uint8_t* frontier, uint64_t ngroups, uint64_t* out) {
    uint8_t* mask = (uint8_t*)calloc(ngroups ? ngroups : 1, 1);
    for (uint32_t u = 0; u < V; ++u) {
        if (!frontier[u]) continue;
        for (uint64_t j = eidx_off[u]; j < eidx_off[u + 1]; ++j) mask[eidx[j]] = 1;
    }
    uint64_t n = 0;
    for (uint64_t g = 0; g < ngroups; ++g)
        if (mask[g]) out[n++] = g;
    free(mask);
    return n;
}

/* Frontier fullness (Section 5.2, "Frontier Fullness Threshold"): the sum of
 * the out-degrees of the frontier's vertices. */
uint64_t or_fullness(uint32_t V, const uint32_t* outdeg, const uint8_t* frontier) {
    uint64_t f = 0;
    for (uint32_t u = 0; u < V; ++u)
        if (frontier[u]) f += outdeg[u];
    return f;
}

/* ------------------------------------------------------------------ */
/* One Wedge run of BFS, CC or SSSP (Fig. 5 control flow, Sections 3.2,  */
/* 3.4, 5): synchronous pull iterations; after each one the produced     */
/* source-oriented frontier decides, by the fullness threshold, whether  */
/* the next iteration pulls over all edges or only over the edge groups  */
/* of the Wedge Frontier.                                                */
/*                                                                      */
/* Iteration t consumes frontier F_t (vertices whose value changed in    */
/* t-1; F_0 = {root} for BFS/SSSP, all vertices for CC) and produces     */
/* F_{t+1}.  Values are read from the previous iteration's copy (BSP,     */
/* Section 2).  BFS pulls v only while v is unvisited and takes level    */
/* t+1 when an in-neighbour is in F_t (Section 5.2: visited vertices are */
/* skipped).                                                            */
/*                                                                      */
/* trace (optional, 5 u64 per iteration): |F_t|, fullness(F_t), mode     */
/* (0 dense, 1 sparse), number of groups pulled (0 when dense), edges    */
/* pulled.  Returns the number of iterations (pull steps) executed.      */
/* ------------------------------------------------------------------ */
uint64_t or_wedge_run(int app, uint32_t V, uint64_t E, const uint32_t* off, const uint32_t* src,
                      const uint32_t* w, uint32_t root, int policy, uint32_t tau_bp,
                      uint64_t group, uint64_t max_iters, uint32_t* val, uint64_t* trace,
                      uint64_t trace_cap) {
    uint32_t* outdeg = (uint32_t*)malloc(sizeof(uint32_t) * (V ? V : 1));
    uint32_t* old = (uint32_t*)malloc(sizeof(uint32_t) * (V ? V : 1));
    uint8_t* front = (uint8_t*)calloc(V ? V : 1, 1);
    uint8_t* next = (uint8_t*)calloc(V ? V : 1, 1);
    uint64_t ngroups = group ? (E + group - 1) / group : 0;
    uint8_t* gmask = (uint8_t*)calloc(ngroups ? ngroups : 1, 1);
    or_outdeg(V, E, src, outdeg);

    for (uint32_t v = 0; v < V; ++v) {
        if (app == OR_CC) {
            val[v] = v;
            front[v] = 1;
        } else {
            val[v] = INF32;
        }
    }
    if (app != OR_CC && root < V) {
        val[root] = 0;
        front[root] = 1;
    }

    uint64_t t = 0;
    for (; t < max_iters; ++t) {
        uint64_t nfront = 0;
        for (uint32_t v = 0; v < V; ++v) nfront += front[v];
        if (nfront == 0) break;
        uint64_t full = or_fullness(V, outdeg, front);
        int sparse;
        if (policy == OR_POLICY_ALWAYS_DENSE) sparse = 0;
        else if (policy == OR_POLICY_ALWAYS_SPARSE) sparse = 1;
        else sparse = full * 10000ull < (uint64_t)tau_bp * E;

        uint64_t ngsel = 0;
        if (sparse) {
            memset(gmask, 0, ngroups ? ngroups : 1);
            for (uint64_t p = 0; p < E; ++p)
                if (front[src[p]]) gmask[p / group] = 1;
            for (uint64_t g = 0; g < ngroups; ++g) ngsel += gmask[g];
        }

        memcpy(old, val, sizeof(uint32_t) * V);
        memset(next, 0, V);
        uint64_t pulled = 0;
        for (uint32_t v = 0; v < V; ++v) {
            if (app == OR_BFS && old[v] != INF32) continue; /* visited: skipped */
            for (uint64_t p = off[v]; p < off[v + 1]; ++p) {
                if (sparse && !gmask[p / group]) continue;
                ++pulled;
                uint32_t u = src[p];
                if (app == OR_BFS) {
                    if (front[u] && val[v] == INF32) val[v] = (uint32_t)(t + 1);
                } else if (app == OR_CC) {
                    if (old[u] < val[v]) val[v] = old[u];
                } else {
                    if (old[u] == INF32) continue;
                    uint64_t cand = (uint64_t)old[u] + w[p];
                    if (cand > SAT32) cand = SAT32;
                    if (cand < val[v]) val[v] = (uint32_t)cand;
                }
            }
            if (val[v] != old[v]) next[v] = 1;
        }
        if (trace && t < trace_cap) {
            trace[5 * t + 0] = nfront;
            trace[5 * t + 1] = full;
            trace[5 * t + 2] = (uint64_t)sparse;
            trace[5 * t + 3] = ngsel;
            trace[5 * t + 4] = pulled;
        }
        uint8_t* tmp = front;
        front = next;
        next = tmp;
    }
    free(outdeg);
    free(old);
    free(front);
    free(next);
    free(gmask);
    return t;
}

/* ------------------------------------------------------------------ */
/* All-cores timing variants (the CPU baseline's multi-threaded leg):   */
/* the same dense pulls, every iteration over all in-edges (Section 2.1,*/
/* pull), with the loop over destinations shared among OpenMP threads.  */
/* Each destination is computed by one thread in CSC order, from the    */
/* previous iteration's values, so the results are the single-threaded  */
/* functions' bit for bit.  Built with -fopenmp when the compiler has   */
/* it; otherwise these run on one thread.                               */
/* ------------------------------------------------------------------ */
#ifdef _OPENMP
#include <omp.h>
#endif

int or_omp_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* BFS, CC or SSSP by dense pulls until the frontier is empty; returns the
 * number of pulls.  Same values as or_wedge_run(..., ALWAYS_DENSE, ...). */
uint64_t or_dense_pull_omp(int app, uint32_t V, const uint32_t* off, const uint32_t* src, const uint32_t* w,
                           uint32_t root, uint32_t* val) {
    uint32_t* old = (uint32_t*)malloc(sizeof(uint32_t) * (V ? V : 1));
    uint8_t* front = (uint8_t*)calloc(V ? V : 1, 1);
    uint8_t* next = (uint8_t*)calloc(V ? V : 1, 1);
    for (uint32_t v = 0; v < V; ++v) {
        val[v] = (app == OR_CC) ? v : INF32;
        front[v] = (app == OR_CC);
    }
    if (app != OR_CC && root < V) {
        val[root] = 0;
        front[root] = 1;
    }
    uint64_t t = 0;
    for (;; ++t) {
        uint64_t nfront = 0;
        for (uint32_t v = 0; v < V; ++v) nfront += front[v];
        if (nfront == 0) break;
        memcpy(old, val, sizeof(uint32_t) * V);
        int64_t n = (int64_t)V;
#pragma omp parallel for schedule(dynamic, 4096)
        for (int64_t vi = 0; vi < n; ++vi) {
            const uint32_t v = (uint32_t)vi;
            next[v] = 0;
            if (app == OR_BFS && old[v] != INF32) continue;
            uint32_t best = old[v];
            for (uint64_t p = off[v]; p < off[v + 1]; ++p) {
                const uint32_t u = src[p];
                if (app == OR_BFS) {
                    if (front[u] && best == INF32) best = (uint32_t)(t + 1);
                } else if (app == OR_CC) {
                    if (old[u] < best) best = old[u];
                } else if (old[u] != INF32) {
                    uint64_t cand = (uint64_t)old[u] + w[p];
                    if (cand > SAT32) cand = SAT32;
                    if (cand < best) best = (uint32_t)cand;
                }
            }
            val[v] = best;
            if (best != old[v]) next[v] = 1;
        }
        uint8_t* tmp = front;
        front = next;
        next = tmp;
    }
    free(old);
    free(front);
    free(next);
    return t;
}

/* PageRank as or_pr_pull, the destination loop shared among threads. */
void or_pr_pull_omp(uint32_t V, const uint32_t* off, const uint32_t* src, const uint32_t* outdeg, double d,
                    uint32_t iters, double* pr) {
    double* contrib = (double*)malloc(sizeof(double) * (V ? V : 1));
    for (uint32_t v = 0; v < V; ++v) pr[v] = 1.0 / V;
    for (uint32_t t = 0; t < iters; ++t) {
        double dangling = 0.0;
        for (uint32_t u = 0; u < V; ++u) {
            if (outdeg[u] == 0) {
                dangling += pr[u];
                contrib[u] = 0.0;
            } else {
                contrib[u] = pr[u] / outdeg[u];
            }
        }
        int64_t n = (int64_t)V;
#pragma omp parallel for schedule(dynamic, 4096)
        for (int64_t vi = 0; vi < n; ++vi) {
            const uint32_t v = (uint32_t)vi;
            double sum = 0.0;
            for (uint64_t p = off[v]; p < off[v + 1]; ++p) sum += contrib[src[p]];
            pr[v] = (1.0 - d) / V + d * (sum + dangling / V);
        }
    }
    free(contrib);
}

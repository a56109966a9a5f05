/*
 * gc.h -- C ABI of the GB300 batch-dynamic 4-node graphlet counter.
 *
 * The library maintains, for one simple undirected graph resident in GPU
 * memory, the counts of the six connected induced 4-vertex graphlets, in the
 * order of Fig. 1 of "Efficient Batch Dynamic Graphlet Counting"
 * (arXiv 2308.14493):
 *
 *     out[0] g1 3-path        out[3] g4 tailed triangle
 *     out[1] g2 3-star        out[4] g5 diamond
 *     out[2] g3 4-cycle       out[5] g6 4-clique
 *
 * Problem 1 (Sec. 3) defines the maintained quantity; Algorithm 2 (FDGC,
 * Sec. 4.3) is the update: for a batch B = A u D, take the region H induced
 * by the k-hop neighbourhood of the batch endpoints, count graphlets in
 * G_a = (H \ D) u A and G_b = (H \ A) u D, add C_a - C_b to the counts, then
 * commit G <- G \ D u A.  Insert-only batches are IGC (Algorithm 1, Sec. 4.2).
 *
 * Conventions for every entry point:
 *  - Return GC_OK (0) or a negative GC_E* code; gc_last_error() then holds
 *    a one-line reason.  A failed call leaves the graph and its counts
 *    exactly as they were.
 *  - Vertex ids are int32 in [0, n); n is fixed by gc_open.  n < 2^30.
 *  - Edge pairs are int32 [k][2] arrays, row-major: pair i is (p[2i], p[2i+1]).
 *  - All entry points are synchronous: when they return, every input buffer
 *    may be reused and every output is written.  A handle is not thread-safe;
 *    separate handles are independent.
 *  - The caller owns every buffer it passes; the library copies what it
 *    needs and owns all device memory it allocates.
 */
#ifndef GC_H
#define GC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GC_OK = 0,
    GC_EINVAL = -1,   /* bad argument: null pointer, id out of range, self-loop, malformed CSR */
    GC_ENOMEM = -2,   /* device or host allocation failed */
    GC_ECUDA = -3,    /* a CUDA runtime call failed; see gc_last_error() */
    GC_ETIMEOUT = -4  /* reserved: a bounded device-side wait ran out */
};

typedef struct gc_graph gc_graph;

/* Options for gc_open.  Zero-initialised fields take the defaults. */
typedef struct {
    /* Device allocator callbacks (both or neither).  alloc returns device
       memory of at least `bytes` bytes usable on `stream` (the handle's
       stream), or NULL, which makes the call that needed it return
       GC_ENOMEM with the graph and its counts unchanged; free releases a
       pointer alloc returned, in the order of `stream`.  NULL for both: the
       library uses cudaMallocAsync / cudaFreeAsync on its stream.  The
       Python binding's TorchAllocator passes PyTorch's caching allocator. */
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, void *stream, void *ctx);
    void *ctx;
    void *stream;        /* cudaStream_t to run on; NULL: the library makes one */
    int32_t region_hops; /* k of the k-hop region; 0 -> 3 as in Sec. 4.2; must be >= 2 */
    float slack;         /* spare capacity per adjacency row; 0 -> 0.25 */
    int32_t device;      /* CUDA device ordinal; 0 -> current device */
    int32_t dense_cluster; /* CTAs per cluster of the heavy 4-cycle kernel: 0 auto, 8 or 16 */
    int32_t chunk_threshold; /* wedge bound above which a 4-cycle pivot is counted in shared memory
                                over id-range chunks; <= 0: never (the cluster kernel takes them) */
    int32_t local_max_pairs; /* batches of at most this many pairs (as passed) to gc_apply_batch,
                                gc_count_batch and their _device forms, and such batches within
                                gc_apply_batches* runs (taken one at a time, in order), take the
                                edge-local delta: the same counts from only the terms a batch can
                                change (edges at its endpoints, 4-cliques and 4-cycles through its
                                pairs) instead of a region recount.  0: never; gc_autotune sets
                                it by measurement */
    int32_t serial_count;    /* 1: the counting kernels of a pass run one after another on the
                                handle's stream instead of side by side on three side streams
                                (slower; each kernel's own time, e.g. gc_stats.ms_stage[7], is
                                then that of the kernel alone); 0: side by side */
    int32_t reserved[3];
} gc_options;

/* Per-batch record of the last gc_apply_batch* call. */
typedef struct {
    int64_t n_ins_raw, n_del_raw;   /* pairs passed in */
    int64_t n_ins, n_del;           /* pairs applied after normalisation (|A|, |D|) */
    int64_t repeats;                /* pairs dropped as repeats within A or within D */
    int64_t cancelled;              /* pairs present in both A and D, dropped from both (Sec. 5) */
    int64_t noop_ins, noop_del;     /* insertions of present edges, deletions of absent ones */
    int64_t region_vertices;        /* |W|, the k-hop region */
    int64_t region_entries;         /* directed adjacency entries of the region union graph */
    int64_t edges_a, edges_b;       /* undirected edges of G_a and G_b */
    int64_t Ca[6], Cb[6];           /* induced counts of G_a and G_b */
    int64_t sums_a[6], sums_b[6];   /* [P, S, TT, D, K, Q]: non-induced 3-paths, 3-stars,
                                       tailed triangles, diamonds, 4-cliques, 4-cycles */
    int64_t num_edges;              /* edges of the graph after the batch */
    float ms_device;                /* device time of the batch (CUDA events) */
    float ms_wall;                  /* host wall time of the call */
    int32_t relayouts;              /* adjacency re-layouts the batch needed */
    int32_t path;                   /* 0: region recount (Algorithm 2); 2: a batched run whose
                                       later batches went in pairs (gc_tuning.pair_min_share);
                                       1: edge-local delta, for
                                       which region_vertices is |V_X| (the endpoints),
                                       region_entries their union-row entries, Ca / sums_a the
                                       six induced / non-induced deltas and Cb / sums_b zero,
                                       C3a the 3-vertex deltas, work_triangles the probes */
    int32_t reserved[4];
    /* device time per stage (CUDA events):
       [0] normalise  [1] region walk  [2] union graph  [3] triangles + 4-cliques
       [4] 4-cycles   [5] edge terms + closed forms     [6] commit
       [7] the heavy-pivot 4-cycle kernels alone (k_c4_dense_t and, when a
           tuning enables it, k_c4_chunk), timed on the stream they run on
       Stages 3 and 4 run side by side: each is timed from the start of the
       counting pass to its own end. */
    float ms_stage[8];
    /* work of the counting pass, for roofline accounting */
    int64_t work_triangles;         /* sum over union-graph out-edges u->v of |N+(u)| + |N+(v)| */
    int64_t work_wedges;            /* wedges u-v-w (v, w below u) walked for the 4-cycles */
    int32_t launches;               /* kernels the call launched */
    int32_t reserved2[3];
    int64_t C3a[2], C3b[2];         /* 3-vertex counts of G_a and G_b: [0] induced 2-paths
                                       (open wedges), [1] triangles */
    /* work of the heavy-pivot 4-cycle kernels of ms_stage[7], for their own
       roofline: the wedges they walked, and the counter updates they sent to
       L2 (reductions that return nothing; atomics that return the old value;
       the shared-memory counters of k_c4_chunk send none) */
    int64_t work_wedges_heavy;
    int64_t l2_red_heavy, l2_atom_heavy;
} gc_stats;

/* Fill *opt with the defaults. */
void gc_default_options(gc_options *opt);

/*
 * Open a graph from a host CSR and count it.
 *   n        vertices, 0 <= n < 2^30
 *   row_ptr  host int32[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = 2m
 *   col      host int32[row_ptr[n]]: neighbours; rows in any order
 *   opt      NULL for defaults
 *   out      receives the handle
 * The CSR must be symmetric, without self-loops or repeated entries
 * (GC_EINVAL otherwise).  The initial counts are a full static count, which
 * equals streaming every edge into an empty graph (Algorithm 2 starts from
 * F = 0 on an empty graph).  Input is copied; the caller keeps ownership.
 */
int gc_open(int32_t n, const int32_t *row_ptr, const int32_t *col,
            const gc_options *opt, gc_graph **out);

/* Full static recount of the current graph into out[6] (the recount
   baseline of Sec. 4.1).  Does not change the maintained counts. */
int gc_count_static(gc_graph *g, uint64_t out[6]);

/* The maintained counts. */
int gc_counts(const gc_graph *g, uint64_t out[6]);

/* The maintained 3-vertex graphlet counts, a by-product of the same per-edge
   triangle counts and degrees (Sec. 3 notes PGD yields them too):
   out[0] induced 2-paths (open wedges) = sum_v C(d_v, 2) - 3 triangles,
   out[1] triangles.  They follow every batch exactly as the 4-vertex
   counts do (F3 += C3_a - C3_b). */
int gc_counts3(const gc_graph *g, uint64_t out[2]);

/* Induced counts of all eleven 4-vertex graphs, from the maintained counts,
   the 3-vertex counts, n and m (no device work): [0..5] the six connected
   graphlets of gc_counts, [6] triangle + isolated vertex, [7] 2-path +
   isolated vertex, [8] two vertex-disjoint edges, [9] one edge + two
   isolated vertices, [10] empty; they sum to C(n, 4).  Each count is
   128-bit (C(n, 4) passes 2^64 near n = 100,000): out[2i] holds its low
   64 bits, out[2i + 1] its high 64 bits.  The disconnected counts follow
   from counting, two ways, the triangles with a fourth vertex, the 2-paths
   with a fourth vertex, the pairs of vertex-disjoint edges and the edges
   with two more vertices (each lies in exactly one 4-set, and each induced
   type holds a fixed number of them). */
int gc_counts_all(const gc_graph *g, uint64_t out[22]);

/* Per-vertex (local) graphlet counts of the current graph: out[6 x + k] =
   the induced connected 4-vertex graphlets of type k (order of gc_counts)
   that contain vertex x (external ids, out holds 6 n words, host memory).
   The containment identity of the global counts holds per vertex, so the
   non-induced copies through each vertex, counted by its role in them,
   invert the same way; the sum over vertices is 4 x gc_counts.  Runs a
   static pass plus the per-vertex kernels (device scratch of about 4 bytes
   per adjacency entry, 64 bytes per vertex, and one 4-byte counter array
   per 4-cycle block, 2 GB at most, all freed on return); the maintained
   counts are not changed.  gc_batch_stats().ms_device gives the device
   time of the per-vertex kernels. */
int gc_vertex_counts(gc_graph *g, uint64_t *out);

/* The same per vertex and orbit: out[11 x + j] = the induced connected
   4-vertex graphlets holding vertex x in orbit 4 + j (orbits 4..14: 3-path
   end, middle; 3-star leaf, centre; 4-cycle; tailed triangle tail end,
   other triangle corner, attachment; diamond degree-2 corner, degree-3
   corner; 4-clique).  out holds 11 n words.  The role counts invert with
   the triangular containment of roles in orbits; the orbits of a graphlet
   sum to its per-vertex count. */
int gc_vertex_orbits(gc_graph *g, uint64_t *out);

/* Per-edge (local) graphlet counts of the current graph.  Row r describes
   the edge edges[2 r] < edges[2 r + 1] (external ids; the rows run over the
   m = gc_num_edges(g) edges in increasing (lo, hi) order), and out[6 r + k]
   is the number of induced connected 4-vertex graphlets of type k (order of
   gc_counts) that contain that edge.  edges (int32[2 m], host) may be NULL;
   out (uint64[6 m], host) may be NULL only when m = 0.  The containment
   identity of the global counts holds per edge: the non-induced copies of
   each connected 4-vertex subgraph through the edge, counted by the edge's
   role in them, invert with a triangular matrix.  Summed over the edges,
   type k gives (3, 3, 4, 4, 5, 6)[k] x gc_counts.  Runs a static pass plus
   the per-edge kernels (device scratch of 52 bytes per adjacency entry,
   two per edge; 8 bytes per vertex; the device copy of the output; and one
   4-byte counter array per 4-cycle block, 2 GB at most; all freed on
   return); the maintained counts are not changed.  gc_batch_stats().ms_device gives the device time of the
   per-edge kernels. */
int gc_edge_counts(gc_graph *g, int32_t *edges, uint64_t *out);

/* The same per edge orbit: out[10 r + j] = the induced connected 4-vertex
   graphlets holding the edge of row r in edge orbit j: 0 3-path end edge,
   1 3-path middle edge, 2 3-star edge, 3 4-cycle edge, 4 tailed-triangle
   tail, 5 tailed-triangle edge opposite the attachment, 6 tailed-triangle
   edge at the attachment, 7 diamond outer edge, 8 diamond chord, 9
   4-clique edge.  out holds 10 m words; the orbits of a graphlet sum to
   its per-edge count. */
int gc_edge_orbits(gc_graph *g, int32_t *edges, uint64_t *out);

/*
 * Apply one batch (Algorithm 2) and return the updated counts.
 *   ins   host int32[n_ins][2]: pairs to insert (may be NULL when n_ins = 0)
 *   del   host int32[n_del][2]: pairs to delete (may be NULL when n_del = 0)
 *   out   host uint64[6]: counts after the batch (may be NULL)
 * Pairs are unordered; repeats collapse; a pair in both lists is dropped from
 * both; inserting a present edge or deleting an absent one does nothing.
 * Self-loops or ids outside [0, n) give GC_EINVAL and change nothing.
 */
int gc_apply_batch(gc_graph *g, const int32_t *ins, int64_t n_ins,
                   const int32_t *del, int64_t n_del, uint64_t out[6]);

/*
 * Delete vertices (Sec. 3 models a vertex deletion as the deletion of its
 * edges): every edge incident to ids[0..k) is deleted in one batch, applied
 * as gc_apply_batch would; the vertices stay, isolated (a vertex is
 * inserted by gc_add_vertices and gains its edges by gc_apply_batch).  Ids
 * outside [0, n) give GC_EINVAL and change
 * nothing; repeated ids are allowed.  out: counts after the deletion.
 */
int gc_delete_vertices(gc_graph *g, const int32_t *ids, int64_t k, uint64_t out[6]);

/*
 * Add k isolated vertices; their ids are [n, n + k) with n the count before
 * the call (*first_id receives n; first_id may be NULL).  The counts do not
 * change (an isolated vertex is in no connected graphlet); later batches may
 * use the new ids.  GC_EINVAL if n + k would reach 2^30.
 */
int gc_add_vertices(gc_graph *g, int64_t k, int32_t *first_id);

/* Vertices of the graph (n). */
int32_t gc_num_vertices(const gc_graph *g);

/* As gc_apply_batch, with the pair arrays in device memory (int32, same
   layout).  The library does not read the pairs on the host: the
   normalisation kernel checks every pair on the device, and a pair with an
   id outside [0, n) or a self-loop makes the call return GC_EINVAL with the
   graph and the counts unchanged. */
int gc_apply_batch_device(gc_graph *g, const int32_t *d_ins, int64_t n_ins,
                          const int32_t *d_del, int64_t n_del, uint64_t out[6]);

/*
 * Count one batch against the current graph without applying it: out
 * receives the counts of G (+) B, the graph and the maintained counts stay as
 * they were.  The same Algorithm 2 step as gc_apply_batch, minus the commit
 * (a what-if query; k of these on one graph give the independent mode of
 * gc_apply_batches).  Arguments, batch semantics and errors as for
 * gc_apply_batch / gc_apply_batch_device.
 */
int gc_count_batch(gc_graph *g, const int32_t *ins, int64_t n_ins,
                   const int32_t *del, int64_t n_del, uint64_t out[6]);
int gc_count_batch_device(gc_graph *g, const int32_t *d_ins, int64_t n_ins,
                          const int32_t *d_del, int64_t n_del, uint64_t out[6]);

/*
 * Apply k batches in one device launch sequence (a CUDA graph replayed per
 * batch, with batch sizes read on the device).
 *   ins[i], n_ins[i], del[i], n_del[i]   host pair arrays of batch i
 *   independent  0: batches apply in order, each on the graph the previous
 *                   one left (sequential stream);
 *                1: every batch is counted against the current graph and
 *                   nothing is committed (what-if batches on one snapshot)
 *   out          host uint64[k][6]: counts after each batch
 * Results equal k calls of gc_apply_batch (independent = 0), or k calls each
 * made on a fresh copy of the graph (independent = 1).
 */
int gc_apply_batches(gc_graph *g, const int32_t *const *ins, const int64_t *n_ins,
                     const int32_t *const *del, const int64_t *n_del, int32_t k,
                     int32_t independent, uint64_t *out);

/*
 * As gc_apply_batches, with every pair already in device memory.
 *   d_pairs   device int32 pairs [.][2]
 *   batches   host int64[k][4]: for batch i, {ins_off, n_ins, del_off, n_del}
 *             -- its insertions are pairs d_pairs[ins_off .. ins_off+n_ins),
 *             its deletions d_pairs[del_off .. del_off+n_del)
 *   out       host uint64[k][6]
 * Every pair is checked on the device: a batch with an id outside [0, n) or
 * a self-loop is not applied and the call returns GC_EINVAL.
 */
int gc_apply_batches_device(gc_graph *g, const int32_t *d_pairs, const int64_t *batches, int32_t k,
                            int32_t independent, uint64_t *out);

/* Record of the last batch (of a batched call: its last batch, with the
   run's device time in ms_device and its total launches). */
int gc_batch_stats(const gc_graph *g, gc_stats *s);

/* Edges currently in the graph. */
int64_t gc_num_edges(const gc_graph *g);

/* Copy the current graph out as a host CSR with sorted rows.
   row_ptr: int32[n+1]; col: int32[2 * gc_num_edges(g)]. */
int gc_export_csr(gc_graph *g, int32_t *row_ptr, int32_t *col);

/*
 * Static count that allocates nothing.  The paper has no counterpart; this
 * entry point exists for callers that must not allocate device memory when
 * they ask for a count: a service whose device memory is all reserved up
 * front by another allocator, a latency-critical loop that cannot afford the
 * device-wide synchronisation and delay of cudaMalloc, or a plug-in inside a
 * host process that forbids device allocations after start-up.
 *
 * It computes the same six counts as gc_count_static, for a graph the caller
 * already holds in device memory, using only a fixed scratch array compiled
 * into this library (about 9 MB, held on every GPU that loads the library
 * until the process exits).  It calls no cudaMalloc, cudaFree or any other
 * allocating routine.  It orients edges by the caller's vertex ids as given
 * (renumbering by degree, as gc_open does, would need scratch of its own), so
 * its 4-cycle work is bounded by m * d_max rather than by the degree-ordered
 * bound; the counts do not depend on the order.
 *   n          vertices, 1 <= n <= GC_NOALLOC_MAX_VERTICES (n = 0 gives zeros)
 *   d_row_ptr  device int32[n+1], d_row_ptr[0] = 0, d_row_ptr[n] = nnz
 *   d_col      device int32[nnz]: a symmetric simple graph, every row sorted
 *              ascending, nnz <= GC_NOALLOC_MAX_ENTRIES
 *   stream     cudaStream_t to run on (NULL: the default stream)
 *   out        host uint64[6]: the counts, in the order of gc_count_static
 * Returns GC_EINVAL for sizes beyond the limits (before any device work) or
 * for a CSR that fails the checks, GC_ECUDA if a CUDA call fails.  The call
 * is synchronous.  The first call on each device, made with that device
 * current, looks up the scratch array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  Every call shares the one
 * scratch array and leaves its contents behind (each call clears what must
 * start at zero); calls that overlap on the GPU, from different streams or
 * host threads, race and must be serialised by the caller.
 */
#define GC_NOALLOC_MAX_VERTICES 16384
#define GC_NOALLOC_MAX_ENTRIES 524288
int gc_count_static_noalloc(int32_t n, const int32_t *d_row_ptr, const int32_t *d_col, int64_t nnz,
                            void *stream, uint64_t out[6]);

/*
 * Bin boundaries of the counting pass.  Triangle roots are binned by their
 * out-degree k, 4-cycle pivots by the wedge bound w~ (sum of the degrees of
 * their lower neighbours); each field is the upper bound of one kernel's bin,
 * clamped to the capacity that kernel was compiled for (in brackets).  The
 * bins change only the speed, never the counts.
 */
typedef struct {
    int32_t tri_warp_max;   /* warp per root                    [32]    */
    int32_t tri_small_max;  /* block per root, short out-lists  [128]   */
    int32_t tri_block_max;  /* block per root, merge beyond     [512]   */
    int32_t c4_reg_max;     /* registers                        [32]    */
    int32_t c4_warp_max;    /* warp hash in shared memory       [512]   */
    int32_t c4_block_max;   /* block hash in shared memory      [8192]  */
    int64_t c4_cta_max;     /* per-CTA hash table in L2         [32768] */
    int64_t c4_chunk_min;   /* above this and up to c4_chunk_max: shared-memory counters over
                               id-range chunks; other pivots above c4_cta_max: a CTA cluster on a
                               dense array in L2; 0 = never */
    int64_t c4_chunk_max;   /* 0 = no upper bound */
    int64_t local_max_pairs; /* batches of at most this many pairs take the edge-local delta
                                (gc_options.local_max_pairs); 0 = never */
    int64_t local_c4_heavy_min; /* gc_vertex_* and gc_edge_*: 4-cycle pivots with w~ at least this
                                   are walked 8 at a time by the whole GPU, each with its own
                                   counter array in L2; the others by one CTA each on per-CTA
                                   arrays; 0 = never (default 65536) */
    int64_t pair_min_share; /* gc_apply_batches*, sequential runs: when the region pass of a run's
                               first batch holds at least this many per mille of the graph's 2m
                               adjacency entries, the later batches go in pairs: the first of a
                               pair is committed without a count, the second counted over every
                               vertex, which gives the whole graph's counts after both (the
                               counts are the same; one pass instead of two).  The handle keeps
                               the size of that first batch: a later run whose first batch is at
                               least as large goes in pairs from its first batch.  Setting the
                               tuning forgets it.  0 = never (default 700) */
} gc_tuning;

int gc_get_tuning(const gc_graph *g, gc_tuning *t);
int gc_set_tuning(gc_graph *g, const gc_tuning *t);

/*
 * Pick the bin boundaries for this graph by measurement: static counts of
 * the current graph under a set of candidate boundaries (coordinate descent
 * from the current ones, each candidate timed `reps` times with CUDA events,
 * the minimum kept).  The fastest set is installed and returned in *best
 * (may be NULL); *best_ms (may be NULL) receives its time.  Counts are
 * checked equal across all candidates (GC_ECUDA if not).
 * Then the edge-local threshold: what-if batches of k pairs (k = 8, 16,
 * 32, ... up to m / 4 and 2^17; half deletions of edges sampled uniformly,
 * half insertions between vertices drawn in proportion to degree) are
 * timed through the edge-local delta and through the region recount;
 * local_max_pairs becomes the largest k at which the local form was faster
 * (0 if never), and the two results must be equal.
 */
int gc_autotune(gc_graph *g, int32_t reps, gc_tuning *best, float *best_ms);

/* Device memory.  gc_device_bytes: bytes the handle holds now (graph,
   counting state and scratch).  gc_batch_bytes: bytes a batch of n_ins
   insertions and n_del deletions may add to that (scratch growth, plus a
   re-layout of the adjacency if the pool may not take the insertions); an
   upper estimate made on the host, without device work.  gc_trim: release
   the scratch that the next batch re-creates on demand (synchronous).
   -1 / GC_EINVAL for a NULL handle or negative sizes. */
int64_t gc_device_bytes(const gc_graph *g);
int64_t gc_batch_bytes(const gc_graph *g, int64_t n_ins, int64_t n_del);
int gc_trim(gc_graph *g);

/*
 * Serving: a request loop over several resident graphs.  The paper has no
 * serving layer; this is the deployment form of Algorithm 2 for streams of
 * update batches that arrive for many graphs at once.
 *
 * The server takes graphs opened with gc_open (it does not own them; the
 * caller closes them after gc_server_close and does not use them while they
 * are served).  Requests are batches for one graph; they apply in submission
 * order per graph, each with the semantics of gc_apply_batch.  `slots`
 * worker threads run requests of different graphs at the same time, each on
 * its graph's stream, so their device work overlaps (continuous batching: a
 * request is admitted when a slot is free and its graph idle).  Admission by
 * memory: a request starts only if the device bytes held by all served graphs
 * plus the predicted growth (gc_batch_bytes) of every running request and of
 * this one stay within the budget; when they do not, the scratch of idle
 * graphs is released (gc_trim) first, and if that is not enough the request
 * waits for running ones.  A request that cannot fit even alone runs alone.
 * Requests are admitted oldest first among graphs that are idle.
 */
typedef struct gc_server gc_server;

typedef struct {
    int32_t slots;            /* requests in flight at once; 0 -> 4 */
    int32_t reserved0;
    int64_t hbm_budget_bytes; /* 0 -> bytes held by the graphs at open + 90% of the free device memory */
    int64_t reserved[6];
} gc_server_options;

typedef struct {
    int64_t ticket;
    int32_t graph;          /* index into the graphs passed to gc_server_open */
    int32_t status;         /* GC_OK or the GC_E* code of the batch */
    uint64_t counts[6];     /* counts of the graph after the batch */
    int64_t n_ins, n_del;   /* pairs applied after normalisation */
    int64_t region_vertices;
    float ms_device;        /* device time of the batch */
    int32_t relayouts;
    double t_submit_ms;     /* host clock, ms since gc_server_open */
    double t_admit_ms;
    double t_done_ms;
    int64_t bytes_predicted; /* admission estimate of the batch */
} gc_result;

int gc_server_open(gc_graph *const *graphs, int32_t n_graphs, const gc_server_options *opt, gc_server **out);

/* Queue a batch for graph `graph`; the pairs are copied, the call returns at
   once with a ticket.  GC_EINVAL for a bad graph index, NULL arrays with
   non-zero sizes, or a closed server. */
int gc_server_submit(gc_server *s, int32_t graph, const int32_t *ins, int64_t n_ins,
                     const int32_t *del, int64_t n_del, int64_t *ticket);

/* Block until the request is done and return its record (once per ticket;
   GC_EINVAL for an unknown ticket).  The batch's own error, if any, is in
   r->status; the call itself returns GC_OK. */
int gc_server_wait(gc_server *s, int64_t ticket, gc_result *r);

/* Block until every submitted request is done. */
int gc_server_drain(gc_server *s);

/* Peak number of requests that were running at once, and trims made. */
int gc_server_counters(const gc_server *s, int64_t *peak_inflight, int64_t *trims);

/* Finish every queued request, stop the workers, free the server (not the graphs). */
void gc_server_close(gc_server *s);

/* One-line reason for the last failure on this handle ("" if none).
   With g == NULL: the reason for the last failed gc_open. */
const char *gc_last_error(const gc_graph *g);

/* Release the handle and all its device memory.  NULL is allowed. */
void gc_close(gc_graph *g);

#ifdef __cplusplus
}
#endif

#endif /* GC_H */

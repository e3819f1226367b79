/*
 * ldd.h -- C ABI of the GB300 (sm_103a) exponential-shift low-diameter
 * decomposition library (libldd.so).
 *
 * Method: Miller, Peng, Xu, "Parallel Graph Decompositions Using Random
 * Shifts" (2013).  Every vertex u carries a shift delta_u ~ Exp(beta)
 * (Algorithm 2 step 1); every vertex v joins the center u minimising the
 * shifted distance dist(u, v) - delta_u (Eq. (1), Algorithm 2 step 2), ties
 * broken towards the smaller vertex id.  The library computes that
 * assignment exactly, as the delayed-start breadth-first search of Section 4
 * (Algorithm 1 step 3): u enters the search at round floor(delta_max) -
 * floor(delta_u), and same-round competitors are ordered by the rank of the
 * fractional part of their shift, which Section 4 shows is only a tie-breaker.
 *
 * Conventions shared by every call:
 *  - A pointer argument may be host memory (pageable or pinned) or device
 *    memory of the current CUDA device; the library detects which with
 *    cudaPointerGetAttributes and copies as needed.
 *  - The caller owns every buffer it passes.  The library owns the graph
 *    object, its device copy of the CSR and all scratch; ldd_destroy_graph
 *    frees them.
 *  - Calls are synchronous: they return after the work queued on the graph's
 *    stream (ldd_set_stream) has finished and outputs are in place.
 *  - Every call returns an ldd_status; no C++ exception crosses this ABI.
 *    ldd_last_error() gives a one-line description of the latest failure on
 *    the calling thread.
 *  - A graph object is not thread-safe: one call at a time per graph.
 */
#ifndef LDD_H
#define LDD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ldd_graph ldd_graph; /* opaque, library-owned device CSR + scratch */

typedef enum {
  LDD_OK = 0,
  LDD_ERR_ARG = -1,     /* NULL pointer, bad size, beta not finite and > 0,
                           a shift that is NaN or negative */
  LDD_ERR_GRAPH = -2,   /* CSR fails validation (see ldd_create_graph) */
  LDD_ERR_RANGE = -3,   /* a size or value beyond the supported range */
  LDD_ERR_OOM = -4,     /* device or host allocation failed */
  LDD_ERR_CUDA = -5,    /* a CUDA runtime call failed */
  LDD_ERR_TIMEOUT = -6  /* a bounded device-side wait ran out; outputs invalid */
} ldd_status;

/*
 * ldd_create_graph -- copy an undirected, unweighted graph (Definition 1.1)
 * into library-owned device memory.
 *   n        number of vertices, 0 <= n < 2^30.
 *   nnz      number of arcs (each undirected edge appears as two arcs),
 *            0 <= nnz < 2^31.
 *   row_ptr  int32[n + 1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 *   col_idx  int32[nnz], neighbours of v in col_idx[row_ptr[v] .. row_ptr[v+1]).
 *   validate nonzero: check the CSR on the host (bounds, monotone rows,
 *            symmetry: every arc (v, w) has a reverse arc (w, v)) and return
 *            LDD_ERR_GRAPH if it fails.  Self-loops and repeated arcs are
 *            accepted; they change neither the assignment nor the cut count's
 *            meaning (a repeated edge is counted with its multiplicity).
 *            With validate = 0 an asymmetric CSR gives undefined results.
 *   out      receives the graph handle.
 * Row order inside a row is free.  The input buffers may be freed after the
 * call returns.
 */
int ldd_create_graph(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                     int validate, ldd_graph** out);

/*
 * ldd_decompose -- one exponential-shift decomposition (Algorithm 2, computed
 * as Algorithm 1 / Section 4).
 *   g          graph from ldd_create_graph.
 *   beta       the Exp(beta) parameter the shifts were drawn with; must be
 *              finite and > 0.  It is checked and recorded, not used: the
 *              assignment depends on the shifts alone.
 *   shifts     double[n]: delta_u for every vertex, each finite, >= 0 and
 *              < 2^31 (a NaN or negative value gives LDD_ERR_ARG, a value
 *              >= 2^31 or infinite gives LDD_ERR_RANGE).
 *   out_center int32[n]: out_center[v] = the u minimising dist(u,v) - delta_u,
 *              smallest u on exact ties.  Every center is its own center.
 *   out_dist   int32[n]: out_dist[v] = dist(out_center[v], v) in hops.
 * Both outputs are exact (bit-identical to any correct evaluation of the
 * definition on the same FP64 shifts).
 */
int ldd_decompose(ldd_graph* g, double beta, const double* shifts, int32_t* out_center,
                  int32_t* out_dist);

/*
 * ldd_cut_edges -- number of edges between pieces (Definition 1.1, second
 * condition; Section 4 notes the check takes O(m) work).
 *   center   int32[n] piece labels (normally ldd_decompose's out_center; any
 *            labelling with values in [0, n) is accepted).
 *   out_cut  receives #{arcs (v, w) : v < w, center[v] != center[w]}, i.e.
 *            each undirected edge of a symmetric CSR counted once.
 */
int ldd_cut_edges(ldd_graph* g, const int32_t* center, int64_t* out_cut);

/*
 * ldd_decompose_ranked -- the permutation variant of Section 4: the
 * fractional parts of the shifts only break ties inside an integer level, and
 * a random permutation of the vertices can stand in for them.  Every vertex u
 * brings an integer shift levels[u] (e.g. floor(delta_u), delta_u ~ Exp(beta))
 * and a tie-break position perm[u]; every vertex v joins the u minimising
 * (dist(u, v) - levels[u], perm[u]) lexicographically, so a smaller position
 * wins among equal integer shifted distances.  No sort is needed: the
 * permutation is the rank.
 *   levels      int32[n] (host or device), each >= 0.
 *   perm        int32[n] (host or device), a permutation of 0 .. n-1.
 *   out_center, out_dist  as in ldd_decompose.
 * A negative level or a perm that is not a permutation gives LDD_ERR_ARG.
 */
int ldd_decompose_ranked(ldd_graph* g, const int32_t* levels, const int32_t* perm,
                         int32_t* out_center, int32_t* out_dist);

/*
 * ldd_decompose_retry -- the Las Vegas loop of Theorem 1.2's proof: decompose
 * with shifts[0], shifts[1], ... until one decomposition meets both bounds of
 * the wanted (beta, d) decomposition (Definition 1.1): at most max_cut edges
 * between pieces and every vertex within max_radius hops of its center (so
 * every piece has strong diameter <= 2 max_radius, Lemma 3.1).  The paper
 * shows a constant expected number of tries for max_cut ~ beta m and
 * max_radius = O(log n / beta) (Lemma 3.2, Corollary 3.5).
 *   k, shifts    k shift vectors (each n doubles, host or device), tried in
 *                order; the caller draws them (independent Exp(beta) draws).
 *   out_center, out_dist  the accepted decomposition (the last one tried if
 *                none is accepted); host or device.
 *   out_cut, out_radius   NULL or host: its cut count and max distance.
 *   out_accepted host: the index of the accepted vector, or -1 if none of the
 *                k met the bounds (the call still returns LDD_OK).
 * Cut count and radius are computed on the device for every try.
 */
int ldd_decompose_retry(ldd_graph* g, double beta, int k, const double* const* shifts,
                        int64_t max_cut, int32_t max_radius, int32_t* out_center,
                        int32_t* out_dist, int64_t* out_cut, int32_t* out_radius,
                        int32_t* out_accepted);

/*
 * ldd_decompose_batch -- k independent decompositions of g, one per shift
 * vector (as ldd_decompose, Algorithm 2 via Algorithm 1 / Section 4), and
 * optionally the cut count of each (Definition 1.1), pipelined: the k
 * decompositions are queued back to back with one host synchronisation at the
 * end, and while decomposition i runs, shift vector i + 1 is copied to the
 * device and the results of decomposition i - 1 are copied back, on two copy
 * streams of the library's own.  A decomposition whose shifts need the exact
 * fraction rank (crafted ties) is redone alone after the others.  Tree-embedding callers draw many shift vectors per graph
 * (Section 1); a sweep over beta is the same call.
 *   k           number of decompositions (0 is a no-op).
 *   betas       double[k]: as ldd_decompose's beta, each finite and > 0.
 *   shifts      k pointers, each to n doubles (host or device) as in
 *               ldd_decompose.
 *   out_center  k pointers, each to n int32 (host or device).
 *   out_dist    k pointers, each to n int32 (host or device).
 *   out_cut     NULL, or int64[k] on the host: out_cut[i] = the cut count of
 *               decomposition i, computed on the device before its labels
 *               are copied back (no upload of the labels).  When every
 *               out_center is device memory, up to four decompositions'
 *               counts come from one pass over the edges, with their labels
 *               packed 16 bytes per vertex and per cut-list group (at most
 *               32 n bytes more, kept with g after the first such call).
 * Host buffers overlap with the device work only if they are page-locked
 * (cudaHostAlloc / cudaHostRegister); otherwise the copies still happen, in
 * order.  The library keeps two shift slots and two output slots (32 n bytes)
 * after the first call.  On failure the call returns the status of the first
 * decomposition that failed; outputs of the ones before it are complete,
 * later ones are unspecified.  Results are identical to k ldd_decompose calls.
 */
int ldd_decompose_batch(ldd_graph* g, int k, const double* betas, const double* const* shifts,
                        int32_t* const* out_center, int32_t* const* out_dist, int64_t* out_cut);

/*
 * ldd_create_union -- one graph object for a batch: the disjoint union of k
 * graphs (the members), so that one call decomposes all of them.  Algorithm 2
 * never assigns a vertex to a center at infinite distance, so on a disjoint
 * union it decomposes every member independently with that member's own
 * shifts; ldd_union_decompose returns exactly what k ldd_decompose calls
 * would.  A member may appear several times (k shift vectors of one graph, as
 * tree-embedding callers draw them, Section 1).
 *   k        number of members, >= 1.
 *   members  k graphs from ldd_create_graph, on one device (unions are not
 *            accepted as members).  Their tables are copied on the device;
 *            the members may be destroyed after the call returns.
 *   out      receives the union handle.
 * Limits: the sum of the members' vertex counts, each rounded up to a
 * multiple of 32, must be < 2^30, and the sum of their arc counts < 2^31
 * (else LDD_ERR_RANGE).  ldd_decompose, ldd_decompose_batch and
 * ldd_cut_edges reject a union (LDD_ERR_ARG); ldd_set_stream, ldd_set_timing,
 * ldd_get_stats and ldd_destroy_graph work as for any graph.
 */
int ldd_create_union(int k, ldd_graph* const* members, ldd_graph** out);

/* ldd_union_size -- number of members and total = n_0 + ... + n_{k-1} (the
 * length of a union's shift and output arrays); either pointer may be NULL. */
int ldd_union_size(const ldd_graph* u, int32_t* out_k, int64_t* out_total);

/*
 * ldd_union_decompose -- decompose every member of a union in one pass
 * (Algorithm 2 via Algorithm 1 / Section 4 on the union: one rank of all
 * shifts, one persistent round loop over every member's frontier, one
 * finalize), and optionally count each member's cut edges (Definition 1.1).
 * Arrays use the caller layout: member s's n_s entries at offset
 * n_0 + ... + n_{s-1}, in member order.
 *   betas       double[k] on the host: each member's beta (finite, > 0;
 *               checked, not used, as in ldd_decompose).
 *   shifts      double[total] (host or device): member s's shifts, each as
 *               in ldd_decompose.
 *   out_center  int32[total] (host or device): member-local center ids.
 *   out_dist    int32[total] (host or device): hop distances.
 *   out_cut     NULL, or int64[k] on the host: member s's cut count.
 * Results are identical to k separate ldd_decompose / ldd_cut_edges calls.
 * Errors as in ldd_decompose; a bad shift in any member fails the whole call.
 */
int ldd_union_decompose(ldd_graph* u, const double* betas, const double* shifts,
                        int32_t* out_center, int32_t* out_dist, int64_t* out_cut);

/*
 * ldd_block_decompose -- blocks by repeated decomposition.  Section 1
 * (related work) notes that the block decomposition of Linial and Saks --
 * O(log n) blocks whose connected pieces have diameter O(log n) -- follows
 * from running a (1/2, O(log n)) decomposition again and again on the edges
 * not yet in a block, since each run leaves at most half of them in
 * expectation (Corollary 3.5: a fraction 1 - e^{-beta} < beta).  Iteration i
 * decomposes G_i = (V, E_i) (G_0 = g) with shifts[i] exactly as
 * ldd_decompose would; the edges of E_i whose two ends share a piece form
 * block i, and the edges it cuts are E_{i+1}.  The loop stops after the first
 * iteration that leaves no edge, or after k iterations.
 *   k            number of shift vectors available (iterations at most).
 *   betas        double[k] on the host: each finite and > 0 (checked, not used;
 *                the paper's choice is beta = 1/2).
 *   shifts       k pointers to n doubles (host or device), as in
 *                ldd_decompose; shift vector i is read only if iteration i runs.
 *   out_center, out_dist  NULL, or k pointers to n int32 (host or device):
 *                iteration i's decomposition of G_i (entries of iterations
 *                that do not run are left untouched).
 *   out_arc_block NULL, or int32[nnz] (host or device): the block of every arc
 *                of g's CSR, in g's arc order (both arcs of an edge get the same
 *                block; self-loops are in block 0), -1 for arcs still cut when
 *                the shift vectors run out.
 *   out_remaining NULL, or int64[k + 1] on the host: out_remaining[i] = the
 *                undirected edges of G_i (arcs (v, w) with v < w), for i = 0 ..
 *                *out_blocks; later entries are left untouched.
 *   out_blocks   host: the number of iterations run (0 for a graph without arcs
 *                or k = 0).
 * Errors as in ldd_decompose; a failure in iteration i leaves the outputs of
 * earlier iterations complete and *out_blocks = the iterations that finished.
 * The first call allocates the residual graphs' buffers (about 36 bytes per
 * arc and 220 per vertex), which stay with g until ldd_destroy_graph.
 * LDD_ERR_ARG for a union.
 */
int ldd_block_decompose(ldd_graph* g, int k, const double* betas, const double* const* shifts,
                        int32_t* const* out_center, int32_t* const* out_dist,
                        int32_t* out_arc_block, int64_t* out_remaining, int32_t* out_blocks);

/*
 * Request server: continuous batching of decomposition requests.
 *
 * A server owns `slots` workspaces (union graphs of fixed capacity, bought
 * with the HBM budget) and one worker thread per workspace.  Requests --
 * (graph, beta, shifts, output buffers), any mix of graphs -- queue in arrival
 * order.  A free worker takes every waiting request that still fits its
 * workspace (the admission test: the requests' device footprint -- vertices,
 * arcs, cut-list entries, small components -- against the workspace's
 * capacities) and decomposes them as one disjoint union (see
 * ldd_create_union): exactly the per-request results, computed together.
 * The workers' batches run side by side on the device on the workers' own
 * streams, except that their round loops (cooperative kernels that occupy
 * every SM) run one after another, ordered by events: one batch's rank,
 * finalize, cut counts and copies overlap another's, and requests that arrive
 * while a batch runs join the next one as soon as a workspace frees up.  A request whose input fails (a bad shift) fails alone: its batch
 * is rerun request by request.  A batch that holds a single request skips the
 * union and runs on that request's own graph object (at low arrival rates the
 * union would only add latency).  Graphs passed to a server must stay alive,
 * must not be destroyed until their requests are collected, and must not be
 * used on another thread while they have requests in flight.
 */
typedef struct ldd_server ldd_server;

typedef struct {
  int64_t hbm_budget_bytes; /* device memory for all workspaces together (> 0) */
  int32_t max_batch;        /* most requests per batch (>= 1) */
  int32_t slots;            /* workspaces and worker threads (>= 1) */
  int32_t one_at_a_time;    /* 1: no batching -- one worker runs each request as
                               ldd_decompose_batch(g, 1, ...) in arrival order
                               (the comparison mode); budget and caps unused */
  int32_t reserved;         /* 0 */
  int64_t max_vertices;     /* per batch, members padded to multiples of 32;
                               0: as many as the per-slot budget allows (< 2^30) */
  int64_t max_arcs;         /* per batch; 0: derived from the budget (< 2^31) */
} ldd_server_config;

typedef struct {
  int32_t status;     /* LDD_OK or the request's error */
  int32_t batch_size; /* requests decomposed together with this one */
  int64_t batch_id;   /* batches in the order workers took them */
  double submit_us;   /* server clock: microseconds since ldd_server_create */
  double start_us;    /* taken by a worker */
  double end_us;      /* results in the caller's buffers */
  double batch_fill_us; /* its batch: union built and shifts copied in (host clock) */
  double batch_run_us;  /* its batch: decomposition, cut counts and result copies, from
                           their enqueueing to their end (host clock) */
} ldd_request_info;

/* ldd_server_create -- a server on the current device.  LDD_ERR_RANGE if the
 * caps do not fit the budget; LDD_ERR_OOM if the workspaces cannot be had. */
int ldd_server_create(const ldd_server_config* cfg, ldd_server** out);

/*
 * ldd_server_submit -- queue one decomposition of g (Algorithm 2, as
 * ldd_decompose) and, if out_cut is not NULL, its cut count (Definition 1.1).
 *   shifts      double[n] host memory (page-locked for copies that overlap).
 *   out_center, out_dist  int32[n] host memory; out_cut: host int64 or NULL.
 * The buffers must stay valid until ldd_server_wait returns for the ticket.
 * LDD_ERR_RANGE: g alone exceeds a workspace.  out_ticket receives the
 * request's ticket.
 */
int ldd_server_submit(ldd_server* s, ldd_graph* g, double beta, const double* shifts,
                      int32_t* out_center, int32_t* out_dist, int64_t* out_cut,
                      int64_t* out_ticket);

/* ldd_server_wait -- block until the request is done, fill *info (may be
 * NULL), release the ticket, and return the request's status. */
int ldd_server_wait(ldd_server* s, int64_t ticket, ldd_request_info* info);

/* ldd_server_footprint -- device bytes one request on g takes of a workspace
 * (the admission measure). */
int ldd_server_footprint(const ldd_server* s, const ldd_graph* g, int64_t* out_bytes);

/* ldd_server_destroy -- finish every queued request, stop the workers and free
 * the workspaces.  Uncollected tickets are dropped.  NULL is a no-op. */
int ldd_server_destroy(ldd_server* s);

/*
 * ldd_cut_edges_noalloc -- the same count as ldd_cut_edges, for callers that
 * must not allocate device memory when they ask for it: for example a process
 * whose framework allocator owns the whole device memory pool, where a foreign
 * cudaMalloc can fail or upset the pool's accounting, or a latency-critical
 * loop that cannot afford the device-wide synchronisation of cudaMalloc and
 * cudaFree.  It needs no graph object (ldd_create_graph allocates) and makes
 * no allocation of its own; the paper has no counterpart to this entry point.
 *   n, nnz      sizes as in ldd_create_graph; nnz must be <= 2^27 (134,217,728
 *               arcs), the limit of the scratch below, else LDD_ERR_RANGE.
 *   row_ptr, col_idx, center
 *               device memory of the current CUDA device (host pointers and
 *               memory of another GPU give LDD_ERR_ARG); layouts as in
 *               ldd_create_graph / ldd_cut_edges.  The CSR is trusted: it is
 *               not validated.
 *   out_cut     host memory or device memory of the current device: receives
 *               the count.
 *   cuda_stream the stream to run on (NULL: the legacy default stream); the
 *               call returns after that stream has finished the work.
 * Scratch: a fixed array of about 256 KiB in the library's device image,
 * present on every GPU that loads the library until the process exits.  The
 * first call on each device (and again after a cudaDeviceReset, which gives
 * the device a new CUDA context) looks up that array's device address; make
 * that first call before any stream capture begins.  Every call reuses the same
 * array and clears the part that must start at zero, so two calls whose work
 * overlaps on the GPU (different streams or threads) race and must be
 * serialised by the caller.
 */
int ldd_cut_edges_noalloc(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                          const int32_t* center, int64_t* out_cut, void* cuda_stream);

/* ldd_set_stream -- queue all later work of g on this cudaStream_t (NULL:
 * the legacy default stream).  A torch.cuda.Stream's .cuda_stream works. */
int ldd_set_stream(ldd_graph* g, void* cuda_stream);

/* ldd_destroy_graph -- free the graph and its device memory (NULL is a no-op). */
void ldd_destroy_graph(ldd_graph* g);

/* ldd_status_string -- static text for a status code. */
const char* ldd_status_string(int status);

/* ldd_last_error -- description of the most recent failure on this thread
 * ("" if none).  The pointer stays valid until the next call on the thread. */
const char* ldd_last_error(void);

/*
 * Statistics of the most recent ldd_decompose / ldd_cut_edges on g.
 * Timings are CUDA-event durations on the graph's stream, recorded only
 * after ldd_set_timing(g, 1); otherwise they read -1.
 */
typedef struct {
  int64_t n, nnz;
  int64_t n_active;       /* vertices settled by the round loop: those in
                             connected components of more than 32 vertices */
  int64_t small_components;/* components of 2..32 vertices, solved one warp each */
  int64_t max_floor_shift;/* A = floor(delta_max) (Algorithm 1 step 2) */
  int64_t rounds;         /* synchronous BFS rounds executed */
  int64_t last_level;     /* level of the last round */
  int64_t items;          /* vertices expanded by the BFS */
  int64_t edges;          /* arcs out of the expanded vertices */
  int64_t pull_rounds;    /* rounds run bottom-up (direction-optimising BFS) */
  int64_t push_arcs;      /* arcs expanded in top-down rounds */
  int64_t pull_arcs;      /* arcs scanned in bottom-up rounds */
  int64_t pull_vertices;  /* vertices examined in bottom-up rounds */
  int64_t launches;       /* kernels launched by the last ldd_decompose */
  int64_t cut_launches;   /* kernels launched by the last ldd_cut_edges */
  int64_t exact_rank;     /* 1 if the fraction rank needed the exact radix-sort
                             path (a fraction bucket overflowed), else 0 */
  int32_t bfs_grid;       /* CTAs of the persistent BFS kernel */
  int32_t bfs_block;      /* threads per CTA */
  float ms_h2d;           /* shifts host -> device (0 if already on device) */
  float ms_rank;          /* split, fraction rank sort, keys, start buckets */
  float ms_bfs;           /* the persistent round loop */
  float ms_finalize;      /* keys -> (center, dist) */
  float ms_d2h;           /* outputs device -> host (0 if device outputs) */
  float ms_total;         /* whole ldd_decompose on the stream */
  float ms_cut;           /* whole ldd_cut_edges on the stream */
  float ms_replay;        /* the replayed CUDA graph (rank .. finalize), when replayed */
  int32_t replayed;       /* 1: the last decomposition ran as a graph replay */
  float ms_create_upload; /* ldd_create_graph: CSR upload to the device (events, once per graph) */
  float ms_create_components; /* ldd_create_graph: component labelling and the small-component
                             tables (device span, once per graph) */
  float ms_create_total;  /* ldd_create_graph: the whole call (host clock), including the host-side
                             cut-list build */
  float ms_block_total;   /* last ldd_block_decompose: the whole call on the stream (events) */
  float ms_block_residual;/* ... of which the residual-graph passes (filter, scan, components) */
  int64_t block_arcs_scanned; /* arcs of G_0, G_1, ... read by the residual passes */
  int64_t block_arcs_kept;    /* arcs written as G_1, G_2, ... */
  int64_t bfs_windows;    /* windows of levels the last round loop ran (ldd_tuning) */
  int64_t bfs_overflow;   /* vertices that windows carried into the next round because a
                             CTA's local queue was full */
} ldd_stats;

int ldd_get_stats(const ldd_graph* g, ldd_stats* out);
int ldd_set_timing(ldd_graph* g, int enable);

/*
 * Launch parameters of the round loop, per graph (or union).  None changes a
 * result; each changes only speed.
 */
typedef struct {
  int32_t bfs_blocks_per_sm; /* CTAs of the persistent round loop per SM (1 or 2) */
  int32_t pull_alpha;        /* go bottom-up when frontier arcs x alpha > unsettled arcs */
  int32_t pull_beta;         /* back to top-down when frontier vertices x beta < BFS vertices */
  int32_t pull_gamma;        /* ... and bottom-up only when frontier arcs x gamma > BFS vertices */
  int32_t probe_min_arcs;    /* top-down rounds with at least this many arcs read a key
                                before its atomicMin */
  int32_t low_degree_rounds; /* 1: when every vertex has at most 32 arcs, run the
                                low-degree rounds (the frontier a plain vertex list, one
                                thread per vertex, the next start bucket checked in the
                                same pass); 0: the edge-balanced rounds always */
  int32_t window_levels;     /* low-degree rounds: levels relaxed between two grid barriers
                                (each CTA going on with the vertices it reaches; exact, but a
                                vertex may be expanded twice); 0 or 1: one level per barrier;
                                8 by default */
  int32_t window_max_frontier; /* ... a window only while the frontier has at most this many
                                vertices (>= 0; 2^18 by default) */
  int32_t window_queue;      /* ... entries of a CTA's local queue per level: 0 for as many
                                as fit in shared memory, else at most that many (>= 0); the
                                rest waits for the next round */
  int32_t bfs_span;          /* edge-balanced rounds: the most arcs a CTA takes per step, a
                                multiple of 256 from 256 to 4096 (4096 by default) */
  float ms;                  /* ldd_autotune: the best decomposition time seen, ms */
} ldd_tuning;

int ldd_get_tuning(const ldd_graph* g, ldd_tuning* out);
/* LDD_ERR_ARG when a field is out of range. */
int ldd_set_tuning(ldd_graph* g, const ldd_tuning* t);

/*
 * ldd_autotune -- pick g's launch parameters for this workload by timing
 * decompositions (CUDA events on g's stream, best of reps after one warm-up)
 * while trying a few values of one parameter at a time (push/pull thresholds,
 * key-probe threshold, CTAs per SM, windows of levels, low-degree rounds,
 * arcs per CTA step), keeping a value only for a gain of 2 % or more.
 * shifts: a representative shift vector (n doubles; a union's caller-layout
 * total), host or device.  The chosen parameters stay on g and are returned
 * in *out.  Results of later decompositions are unaffected.
 */
int ldd_autotune(ldd_graph* g, const double* shifts, int reps, ldd_tuning* out);

/*
 * ldd_set_graph_replay -- enable (1) or disable (0) CUDA-graph replay of the
 * decomposition on g (a plain graph or a union).  Once enabled, the first
 * call runs as usual and the next one captures the fast path -- every kernel
 * from the control-block reset (a union's shift spread included) through
 * finalize, a union's cut counts when asked for, and the status copy to the
 * host -- into a CUDA graph on an internal stream; later calls copy their
 * shifts into the library's input buffer, replay that graph on g's stream
 * (one launch instead of about a dozen), and copy the outputs out of the
 * library's buffers.  Results are identical.  Calls that need the exact rank
 * path or a larger start-bucket table run the regular path instead, and a
 * capture the driver refuses leaves g on the regular path for good (until
 * replay is enabled again); ldd_get_stats' replayed field tells which ran.
 * Disabling frees the captured graphs.
 */
int ldd_set_graph_replay(ldd_graph* g, int enable);

/*
 * Bounded device-side waits.  The round loop ends every round at a grid-wide
 * barrier, and the fraction rank's scans wait on their predecessor tiles
 * (decoupled look-back).  Neither wait can last for ever: after the given
 * number of polls the kernel records the failure, every later kernel of the
 * call writes nothing, and the call returns LDD_ERR_TIMEOUT with outputs
 * invalid; the graph stays usable for the next call.  The defaults (2^22
 * barrier polls of >= 20 ns, 2^24 look-back polls of >= 64 ns: about 0.1 s
 * and 1 s) are far beyond any legitimate wait.  The paper has no counterpart:
 * its PRAM rounds are synchronous by definition.
 *   barrier_polls   polls of the round loop's grid barrier (0: the default;
 *                   the environment variable LDD_SPIN_LIMIT, read when the
 *                   graph is created, sets the initial value).
 *   lookback_polls  polls of a look-back wait (0: the default).
 *   stall_barrier   1: every grid barrier also waits for one CTA that does not
 *                   exist, so the round loop can only end by running out of
 *                   polls -- for tests of the timeout path; 0 normally.
 *   stall_lookback  1: the first tile of each scan waits on a predecessor that
 *                   does not exist, so every look-back runs out of polls (when
 *                   the call takes the fraction-bucket rank) -- for tests; 0
 *                   normally.
 * ldd_set_wait_limits drops a captured replay (ldd_set_graph_replay), since it
 * holds the old values.  LDD_ERR_ARG if a stall field is not 0 or 1.
 */
typedef struct {
  uint32_t barrier_polls;
  uint32_t lookback_polls;
  uint32_t stall_barrier;
  uint32_t stall_lookback;
} ldd_wait_limits;

int ldd_set_wait_limits(ldd_graph* g, const ldd_wait_limits* w);
int ldd_get_wait_limits(const ldd_graph* g, ldd_wait_limits* out);

/*
 * ldd_get_round_profile -- diagnostic: per-round timestamps of the last BFS.
 *   clocks[3i .. 3i+2]  SM clock (cycles) of the first CTA in round i: after
 *              its expansion, after its start-bucket scan, and when its closing
 *              barrier released the CTA.  Entry 0 is the level-0 starts, so
 *              round i took clocks[3i+2] - clocks[3i-1] cycles.
 *   kinds[i]   1 = top-down (push), 2 = bottom-up (pull), 3 = no frontier (jump
 *              to the next start bucket).
 * At most cap rounds (and at most 256) are written; *out_count gets the number.
 * Host buffers of 3 * cap and cap entries.
 */
int ldd_get_round_profile(const ldd_graph* g, int64_t* clocks, int32_t* kinds, int cap,
                          int* out_count);

#ifdef __cplusplus
}
#endif

#endif /* LDD_H */

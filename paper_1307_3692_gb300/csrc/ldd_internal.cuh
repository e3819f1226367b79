// Internal declarations shared by the CUDA translation units of libldd.so.
//
// Key layout (Section 4 of Miller, Peng, Xu 2013): the shifted distance
// dist(u, v) - delta_u is compared as the pair
//     level = (floor(delta_max) - floor(delta_u)) + dist(u, v)   (integer part)
//     rank  = position of u in the order (frac(delta_u) descending, u ascending)
// packed into one 64-bit word key = (level << 32) | rank, so that the
// unsigned minimum of two keys is the lexicographic minimum the paper asks
// for: smaller integer part first, larger fraction on a tie (Section 4: the
// fractional parts are tie-breakers within an integer level and can be
// replaced by a permutation), smaller id on an exact tie (Algorithm 2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ldd {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr u64 kLevelOne = 1ull << 32;

// Bits of Control::err.
enum : u32 {
  kErrShiftArg = 1u << 0,    // a shift is NaN or negative
  kErrShiftRange = 1u << 1,  // a shift is >= 2^31 or infinite
  kErrTimeout = 1u << 2,     // a bounded device-side wait ran out
  kErrBucketCap = 1u << 3,   // start-bucket table smaller than A + 2 (host grows it, reruns)
  kErrInternal = 1u << 4,    // a capacity invariant failed
  kErrRankRetry = 1u << 5,   // a long run of equal 32-bit fraction codes: redo the rank exactly
  kErrPermArg = 1u << 6,     // ranked variant: a negative level or perm not a permutation
};

// Radix sort: 8-bit digits, 256-thread CTAs, 16 keys per thread.
constexpr int kSortThreads = 256;
constexpr int kSortIpt = 16;
constexpr int kSortTile = kSortThreads * kSortIpt;  // 4096 keys per tile
constexpr int kFracDigits = 8;                       // 64-bit fraction key
constexpr int kRoundDigits = 4;                      // 32-bit start round

// BFS: base chunk of the edge-balanced frontier, and the largest span of
// edges one CTA takes per step (window held in shared memory).
constexpr int kBfsThreads = 512;
constexpr int kBfsBase = 256;
constexpr int kBfsMaxSpan = 4096;
// Graphs whose vertices all have at most this many arcs may run the round
// loop's low-degree rounds (k_bfs.cu).
constexpr int kLdMaxDegree = 32;

// Components with at most this many vertices are solved by one warp each.
constexpr u32 kSmallComp = 32;

constexpr int kRoundProfile = 256;
enum : int { kRoundPush = 1, kRoundPull = 2, kRoundSkip = 3 };

// Device control block; cudaMemsetAsync(0) at the start of every decomposition.
// The header (err .. cut) is copied back to the host after every call.
struct Control {
  // header
  u32 err;
  int A;  // floor(delta_max)
  u32 rounds;
  int last_level;
  u64 items;
  u64 edges;
  u64 cut;  // cut-edge accumulator
  // BFS runtime state
  u64 bar;         // grid-barrier arrivals (monotonic within one launch)
  u64 qctr[3];     // frontier counters: (items << 32) | edges
  u32 minrank[3];  // smallest rank among the keys of each frontier level (reset to ~0)
  u32 pull_rounds; // rounds run bottom-up
  u64 push_arcs;   // arcs expanded top-down
  u64 pull_arcs;   // arcs scanned bottom-up
  u64 pull_verts;  // vertices examined bottom-up
  u32 ucnt[3];     // lengths of the still-unsettled lists of bottom-up rounds
  u32 windows;     // windows of levels run by the last round loop
  u32 overflowed;  // ... vertices they carried into the next round (full local queues)
  u32 pad_w;
  // sort state
  u32 mask_f;     // bit d: fraction digit pass d is needed (exact path)
  u32 mask_r;     // unused (start buckets are a counting sort)
  u32 maxbucket;  // largest fraction bucket (fast path)
  u32 tile_ctr[kFracDigits + kRoundDigits];
  u32 hist_f[kFracDigits][256];
  u32 off_f[kFracDigits][256];
  u32 hist_r[kRoundDigits][256];
  u32 off_r[kRoundDigits][256];
  // round profile of the last BFS, SM clock of CTA 0: for round i, [i][0] after
  // its expansion, [i][1] after its start-bucket scan, [i][2] when its
  // barrier let CTA 0 go (entry 0: the level-0 starts); and the round's kind
  long long round_clk[kRoundProfile][3];
  int round_kind[kRoundProfile];
  u32 radius;  // max dist of the last labelling (ldd_decompose_retry)
  // windows of levels (low-degree rounds, k_bfs.cu): overflow-list lengths,
  // rotating like qctr, and the result of a scan for the next start level
  // (~level, by atomicMax; 0: none)
  u32 ovf[3];
  u32 nstart[3];
  // bottom-up rounds: the next unit of candidates a warp takes once the
  // units dealt out in advance are done (rotating like qctr)
  u32 pull_ctr[3];
};
constexpr size_t kCtlHeaderBytes = 40;       // err .. cut
constexpr size_t kCtlBfsStateOffset = 40;    // bar_count .. pull_rounds
constexpr size_t kCtlBfsStateBytes = 96;
constexpr size_t kCtlMinrankOffset = 72;

struct BfsArgs {
  const int* row_ptr;
  const int* col;
  u64* key;
  const int* bptr;   // [A + 2] start-bucket offsets into the round-sorted list
  const u32* rk[2];  // round-sorted keys (start rounds), ping-pong pair
  const u32* rv[2];  // round-sorted vertices, ping-pong pair
  u32* qv[2];        // frontier queues: vertex
  int* qrow[2];      //                  row_ptr[vertex]
  u32* qoff[2];      //                  exclusive edge offset in the frontier
                     // (low-degree rounds use qv alone)
  u32* cf[2];        // first queue slot of every base chunk of edges
  u32* ulist[2];     // vertices still unsettled after a bottom-up round (ping-pong)
  const u32* excl;   // bit v: v is not handled by the BFS
  const u32* active; // the vertices the BFS handles, ascending (n_active), or null
  const u32* first;  // first neighbour of every vertex (~0 without arcs), or null
  Control* ctl;
  u32 n;
  u32 n_active;      // vertices the BFS settles (components of more than 32 vertices)
  u64 nnz_active;    // their arcs
  u32 spin_limit;
  u32 bar_phantom;   // CTAs the grid barrier waits for beyond the launch's own: 0, or 1 to make
                     // every barrier end by running out of polls (tests of the timeout path)
  u32 pull_alpha;    // go bottom-up when frontier arcs * alpha > unsettled arcs
  u32 pull_gamma;    //   and frontier arcs * gamma > n_active (a bottom-up round reads every key)
  u32 pull_beta;     // go back top-down when frontier vertices * beta < n_active
  u32 probe_min_arcs;  // top-down rounds with at least this many arcs read a key before its atomicMin
  u32 low_degree;    // 1: every vertex has at most kLdMaxDegree arcs and the low-degree rounds
                     // run (the frontier a plain vertex list, a thread per vertex)
  u32 window_levels; // low-degree rounds: levels per window (0 or 1: one level per grid barrier)
  u32 window_max_q;  // ... a window only while the frontier has at most this many vertices
  u32 window_queue;  // ... local-queue entries per CTA and level at most (0: as many as fit)
  u32 span;          // edge-balanced rounds: arcs per CTA step at most (kBfsBase .. kBfsMaxSpan)
  const u32* wmem;   // unions: member of every 32-vertex word; else null
  u32* mrank;        // unions: [3][kmem] smallest rank per level slot and member (~0 on entry)
  u32 kmem;          // unions: members
};

// Components of 2..kSmallComp vertices (k_graph.cu): comp c has comp_len[c]
// members comp_v[comp_off[c] ..], with adjacency masks over member lanes in adj.
struct SmallComps {
  u32 ncomp = 0;
  u32 total = 0;
  u32* comp_off = nullptr;
  u32* comp_len = nullptr;
  u32* comp_v = nullptr;
  u32* adj = nullptr;
};

// Temporary device memory for labelling components at graph creation.
struct CompScratch {
  u32* parent;    // [n]
  u32* csize;     // [n]
  u32* root_off;  // [n]
  u32* fill;      // [n]
  u32* lane_of;   // [n]
  u32* comp_off;  // [n / 2 + 1]
  u32* comp_len;  // [n / 2 + 1]
  u32* comp_v;    // [n]
  u32* counters;  // [4]: components, members, vertices left to the BFS, their arcs
};

// ---------------------------------------------------------------- launchers
// Fraction rank and start buckets (k_rank.cu).  Returns kernels launched.
// Buffers of the fraction rank and the start buckets (k_rank.cu).
struct RankBufs {
  const double* shift;  // [n] shifts on the device
  u32 n;
  int num_sms;
  int* a;               // [n] floor(shift)
  u64* k0;              // [max(n, 64)] 64-bit words each: keys / scratch
  u64* k1;
  u32* v0;              // [n] values / scratch; ends as the start-bucket vertices
  u32* v1;
  void* slots;          // fraction_slot_bytes(n): bucket record slots (fast path)
  u64* status;          // look-back status words (epoch-tagged)
  u32* epoch;
  u32* order;           // [n] rank -> vertex
  u64* key;             // [n] start keys
  int* bptr;            // [bptr_cap] start-bucket offsets (rounds 0 .. A + 1)
  u32* rcur;            // [bptr_cap] scatter cursors
  u32* acnt;            // [bptr_cap] start-round counts by floor (fast path; all zero between calls)
  bool acnt_dirty;      // acnt may hold counts of an unfinished call: clear it first
  u32 bptr_cap;
  const u32* excl;      // bit v: v is not handled by the BFS (no start bucket)
  const u32* solo;      // bit v: v is alone in its component (no rank needed)
  const u32* wmem;      // unions: member of every 32-vertex word; else null
  const int* lift;      // unions: floor lift of every member (a_u += lift); else null
  Control* ctl;
  u32 lookback_limit = 1u << 24;  // polls of a look-back wait before kErrTimeout
  u32 stall_lookback = 0;         // 1: the scans' first tile waits on a status word that nothing
                                  // writes, so every look-back runs out (timeout-path tests)
};
// exact64 = false: fraction buckets + in-bucket exact ranks of the vertices
// not alone in their component (may set kErrRankRetry); true: exact 64-bit
// LSD radix sort of all vertices.  The start buckets end in v0 (vertices) and
// k0 viewed as 32-bit words (their rounds).
// chunks (optional): the shifts are still arriving; chunk c is complete once
// ev[c] has fired and covers the vertices up to end[c] (ascending).
struct ShiftChunks {
  int n = 0;
  const u32* end = nullptr;
  const cudaEvent_t* ev = nullptr;
};
int launch_rank_and_buckets(const RankBufs& r, bool exact64, cudaStream_t s,
                            const ShiftChunks* chunks = nullptr);
// Ranked variant (Section 4's permutation in place of the fractional parts):
// integer levels and a tie-break permutation given; no sort.  The same start
// buckets and keys as the exact path.
int launch_ranked_and_buckets(const RankBufs& r, const int* levels, const int* perm,
                              cudaStream_t s);
u32 fraction_bucket_bits(u32 n);
// Look-back status words the fast path's two scans use (status[0 ..)); a
// captured replay clears them and runs with the fixed epochs 1 and 2.
size_t rank_status_words(u32 n, u32 bptr_cap);
size_t fraction_slot_bytes(u32 n);
// Persistent BFS (k_bfs.cu).  Returns kernels launched, or -1 with the CUDA
// error left in *err.
// The most CTAs per SM (1 or 2) the round loop can use; returns that times num_sms.
int bfs_grid_size(int num_sms, int* blocks_per_sm);
// per_sm (1 or 2) picks the kernel instance built for that many CTAs per SM.
int launch_bfs(const BfsArgs& a, int grid, int per_sm, cudaStream_t s, cudaError_t* err);
size_t bfs_smem_bytes();
// Finalize, cut and per-graph component tables (k_graph.cu).
int launch_finalize(const u64* key, const u32* order, const u32* solo, u32 n, int* center,
                    int* dist, const u32* err, int num_sms, cudaStream_t s);
// Cut list of Definition 1.1's count.  Every undirected edge {v, w} (repeated
// edges repeated) is stored once, oriented from its cold endpoint (smaller
// degree; ties: larger id) to its hot one, and grouped by the cold endpoint:
// group g (one per cold vertex that has edges, ascending) is hot[grp_off[g] ..
// grp_off[g + 1]) with cold vertex grp_v[g].  hot[e] < 0 stands for slot
// hot[e] & 0x7fffffff of the hot table (the at most kHotSlots highest-degree
// vertices, whose labels the cut kernel keeps in shared memory).  The edges
// come in blocks of 32: blk_g[b] is the group of edge 32 b, and bit j of
// blk_mask[b] is set when edge 32 b + j (j > 0) starts a group, so edge
// 32 b + j is in group blk_g[b] + popc(blk_mask[b] & bits 0 .. j).  About 4.3
// bytes per edge, plus 12 per group (cold vertex, offset, its label per call).
// In a union (k_union.cu) hot[] and grp_v[] hold caller-layout indices
// (member-local id + the member's output offset) and grp_m[g] the member.
constexpr u32 kHotSlots = 49152;  // 192 KiB of labels per CTA
struct CutList {
  int* hot = nullptr;
  u32* grp_off = nullptr;   // [ngrp + 1]
  u32* grp_v = nullptr;     // [ngrp]
  u32* grp_m = nullptr;     // [ngrp] unions only
  int* grp_lab = nullptr;   // [ngrp] labels of the cold vertices, per cut count
                            //   (unions: [2 ngrp] words, (member << 32) | label)
  u32* blk_g = nullptr;     // [nblk]
  u32* blk_mask = nullptr;  // [nblk]
  u32 m = 0;
  u32 ngrp = 0;
  u32 nblk = 0;             // (m + 31) / 32
};
int launch_cut(const CutList& cl, const int* center, const u32* hot, u32 n_hot, int* hot_center,
               u64* out, int num_sms, cudaStream_t s);
int launch_small_comp(const SmallComps& sc, u64* key, const u32* err, int num_sms, cudaStream_t s);
// The radius of a decomposition: max over v of dist[v], into *out.
int launch_max_dist(const int* dist, u32 n, u32* out, int num_sms, cudaStream_t s);
// Labels components and fills t.comp_* and excl (bit v: kept out of the BFS);
// counts = {small components, their members, vertices left to the BFS, their arcs}.
// excl and solo: bitmasks of (n + 31) / 32 words each.
cudaError_t components_phase1(const int* row_ptr, const int2* up, u32 m_up, u32 n, int num_sms,
                              const CompScratch& t, u32* excl, u32* solo, u32 counts[4],
                              cudaStream_t s);
// components_phase1 in parts, for a caller that hooks the forest itself:
// components_init clears the tables and makes every vertex its own root
// (t.parent); components_label then labels the hooked forest as phase 1 does.
cudaError_t components_init(u32 n, int num_sms, const CompScratch& t, u32* excl, u32* solo,
                            cudaStream_t s);
cudaError_t components_label(const int* row_ptr, u32 n, int num_sms, const CompScratch& t,
                             u32* excl, u32* solo, u32 counts[4], cudaStream_t s,
                             u32 common = 0xffffffffu);
// components_phase1 from the CSR itself (no edge list): Afforest-style
// linking (first neighbours, the most common root, then the remaining arcs of
// the vertices outside it).
cudaError_t components_from_csr(const int* row_ptr, const int* col, u32 n, int num_sms,
                                const CompScratch& t, u32* excl, u32* solo, u32 counts[4],
                                cudaStream_t s);
// Residual graphs of the block decomposition (k_graph.cu), over the m arcs of
// G_i given as (src, col) on its n vertices.  Count pass (write = false):
// kept[v] += arcs of v whose ends have different centers (kept zero on entry),
// those arcs' indices onto klist (*n_kept zero on entry; room for m),
// *up_kept += those with v < w, and arc_block[orig ? orig[e] : e] = block for
// the other arcs (arc_block may be null).  Write pass: every listed arc (v, w)
// at cursor[v]++ (G_{i+1}'s row offsets over G_i's ids on entry) as
// (cid[v], cid[w]) -- G_{i+1}'s own ids -- with its input arc id; each kept
// (v, w), v < w, hooked into parent (union-find on G_{i+1}'s ids).  The order
// inside a row is free.
int launch_residual(bool write, const int* src, const int* col, const int* orig,
                    const int* center, u32 n, u32 m, int block, int* arc_block, u32* kept,
                    unsigned long long* up_kept, u32* klist, u32* n_kept, u32* cursor,
                    const u32* cid, int* new_col, int* new_orig, int* new_src, u32* parent,
                    int num_sms, cudaStream_t s);
// G_{i+1} keeps only the vertices with a kept arc.  flag[v] = 1 for them
// (flag[n] = 0), over G_i's n vertices and the kept-arc offsets off[0 .. n].
int launch_kept_flags(const int* off, u32 n, u32* flag, int num_sms, cudaStream_t s);
// With cid the exclusive scan of the flags: G_{i+1}'s row offsets new_row and
// its vertices' input ids new_map (map: G_i's, null for the input graph).
int launch_compact_rows(const int* off, const u32* cid, u32 n, int* new_row, const u32* map,
                        u32* new_map, int num_sms, cudaStream_t s);
// out[c] = full[map[c]] for G_{i+1}'s nc vertices.
int launch_gather_shifts(const double* full, const u32* map, u32 nc, double* out, int num_sms,
                         cudaStream_t s);
// An iteration's results over all n input vertices: every vertex alone, then
// G_{i+1}'s nc vertices from (cc, dc) in its own ids.
int launch_blocks_output(const int* cc, const int* dc, const u32* map, u32 nc, u32 n, int* center,
                         int* dist, int num_sms, cudaStream_t s);
// first[v] = col[row_ptr[v]], or ~0 for a vertex without arcs.
int launch_first_neighbours(const int* row_ptr, const int* col, u32 n, u32* first, int num_sms,
                            cudaStream_t s);
// src[e] = v for every arc e of row v of the CSR (row_ptr, n).
int launch_fill_src(const int* row, u32 n, int* src, int num_sms, cudaStream_t s);
// Exclusive scan of data[0 .. len) in place (k_rank.cu; decoupled look-back
// on status words tagged with ++*epoch; tile_ctr zero on entry).
int launch_exclusive_scan(u32* data, u32 len, u64* status, u32* epoch, u32* tile_ctr,
                          Control* ctl, u32 spin_limit, cudaStream_t s, u32* copy = nullptr);
// Adjacency masks of the small-component members (sc.comp_v already filled).
cudaError_t components_phase2(const int* row_ptr, const int* col, const CompScratch& t,
                              const SmallComps& sc, int num_sms, cudaStream_t s);

// ---------------------------------------------------------------- batches (k_union.cu)
// A batch of graphs runs as their disjoint union (member s at union vertices
// [voff_s, voff_s + n_s), padded to a multiple of 32).  Device view of one
// member's tables, read once while the union is built.
struct UnionMember {
  const int* row;
  const int* col;
  const int* cut_hot;   // cut list (see CutList): hot endpoints, < 0: slot of the hot table
  const u32* grp_off;
  const u32* grp_v;
  const u32* hot;       // hot table
  const u32* excl;
  const u32* solo;
  const u32* comp_off;
  const u32* comp_len;
  const u32* comp_v;
  const u32* adj;
  const u32* active;    // null unless every member has one
  u32 n;
  u32 nnz;
};
// Member offsets, k + 1 device words each: union vertices (v), arcs (e),
// cut-list entries (u), small components (c) and their members (m), active
// list entries (a), caller-layout outputs (o: n_0 + ... + n_{s-1}), and
// cut-list groups (g).
struct UnionOffsets {
  const u32* v;
  const u32* e;
  const u32* u;
  const u32* c;
  const u32* m;
  const u32* a;
  const u32* o;
  const u32* g;
};
struct UnionTables {
  int* row;
  int* col;
  CutList cut;
  u32* excl;
  u32* solo;
  u32* comp_off;
  u32* comp_len;
  u32* comp_v;
  u32* adj;
  u32* active;
  u32* wmem;  // member of every 32-vertex word
};
// largest = the longest table (elements), for the grid size.
int launch_union_concat(const UnionMember* mem, const UnionOffsets& off, u32 k,
                        const UnionTables& t, u64 largest, int num_sms, cudaStream_t s);
// Shifts to the union layout, and every member's floor lift (amax, lift: k ints).
int launch_union_spread(const double* in, const UnionOffsets& off, u32 k, u32 N,
                        const u32* excl, double* out, int* amax, int* lift, int num_sms,
                        cudaStream_t s);
int launch_union_finalize(const u64* key, const u32* order, const u32* solo,
                          const UnionOffsets& off, u32 k, u32 total, int* center, int* dist,
                          const u32* err, int num_sms, cudaStream_t s);
// Every member's cut count (cut[s], zero on entry) over the union's cut list
// (hot ids resolved, no hot table); labels in the caller layout.
int launch_union_cut(const CutList& cl, const UnionOffsets& off, const u32* wmem,
                     const int* center, u64* cut, int num_sms, cudaStream_t s);
// The union's block tables (cl.blk_g, cl.blk_mask) from its concatenated groups.
int launch_cut_blocks(const CutList& cl, int num_sms, cudaStream_t s);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ u32 lanemask_lt() {
  u32 m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ u64 ld_cg_u64(const u64* p) { return __ldcg(p); }
__device__ __forceinline__ u32 ld_cg_u32(const u32* p) { return __ldcg(p); }
__device__ __forceinline__ int ld_cg_i32(const int* p) { return __ldcg(p); }

__device__ __forceinline__ u32 ld_acquire_u32(const u32* p) {
  u32 v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Inclusive max-scan of a[0 .. len) in shared memory (len <= kLen) by a CTA of
// kThreads threads.  Warp w owns the contiguous block [w * kLen / kWarps, ...)
// and scans it 32 elements at a time with shuffles, so shared-memory accesses
// are one word per lane (no bank conflicts); warp maxima are combined through
// wtot[kThreads / 32].  The caller synchronises before and after.
template <int kThreads, int kLen>
__device__ __forceinline__ void block_max_scan(int* a, int len, int* wtot) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kPerWarp = kLen / kWarps;
  static_assert(kPerWarp % 32 == 0, "scan block must be whole warps");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int base = w * kPerWarp;
  int carry = -1;
  for (int c = 0; c < kPerWarp && base + c < len; c += 32) {
    const int i = base + c + lane;
    int x = (i < len) ? a[i] : -1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x = max(x, y);
    }
    x = max(x, carry);
    if (i < len) a[i] = x;
    carry = __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) wtot[w] = carry;
  __syncthreads();
  int pre = -1;
  for (int i = 0; i < w; ++i) pre = max(pre, wtot[i]);
  if (pre >= 0)
    for (int c = 0; c < kPerWarp && base + c < len; c += 32) {
      const int i = base + c + lane;
      if (i < len) a[i] = max(a[i], pre);
    }
}

__device__ __forceinline__ u64 ld_volatile_u64(const u64* p) {
  return *reinterpret_cast<const volatile u64*>(p);
}
__device__ __forceinline__ void st_volatile_u64(u64* p, u64 v) {
  *reinterpret_cast<volatile u64*>(p) = v;
}

}  // namespace ldd

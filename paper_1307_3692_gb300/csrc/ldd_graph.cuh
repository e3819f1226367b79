// The graph object behind the C ABI's opaque ldd_graph, and the library's
// host-side helpers that more than one translation unit uses (ldd_api.cu:
// graphs, unions, decompositions; ldd_server.cu: the request server).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/ldd.h"
#include "ldd_internal.cuh"

namespace ldd {

// Sets the text ldd_last_error() returns on this thread.
void record_error(const char* msg);
// Sets the thread's ldd_last_error() text and returns status.
int fail(int status, const char* fmt, ...) __attribute__((format(printf, 2, 3)));

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(LDD_ERR_CUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                             \
  } while (0)

// Restores the caller's current device when a call returns.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && (prev == dev || cudaSetDevice(dev) == cudaSuccess))
      ok = true;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// True for device or managed memory; false for pageable or pinned host memory.
bool is_device_ptr(const void* p);
size_t align_up(size_t x, size_t a);

// Capacities of a union workspace (elements of each table).
struct UnionCaps {
  u64 N = 0;      // union vertices, members padded to multiples of 32
  u64 E = 0;      // arcs
  u64 M = 0;      // cut-list entries (undirected edges)
  u64 G = 0;      // cut-list groups (cold vertices with edges)
  u64 C = 0;      // small components
  u64 T = 0;      // their members
  u64 total = 0;  // caller-layout entries (sum of member sizes)
  u32 k = 0;      // members
};
struct Blocks;  // state of ldd_block_decompose (ldd_blocks.cu)
}  // namespace ldd

using namespace ldd;

// Round loops that share a device through a gate run one after another: each
// one's stream waits on the event recorded after the previous one was
// enqueued, and only the enqueueing is serialised (under mu).  The round loop
// is a cooperative kernel that occupies every SM, so two of them never run
// side by side; what overlaps on the device is everything around them (rank,
// finalize, cut counts, copies).
struct BfsGate {
  std::mutex mu;
  cudaEvent_t last = nullptr;  // recorded after the last round loop enqueued, or none
};

struct ldd_graph {
  int32_t n = 0;
  int64_t nnz = 0;
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  u32 n_active = 0;
  u64 nnz_active = 0;
  u32 m_up = 0;                // arcs (v, w) with v < w
  // device CSR and graph tables
  int* d_row = nullptr;
  int* d_col = nullptr;
  CutList cut;                 // grouped cut list (cut count of Definition 1.1)
  u32* d_active = nullptr;     // vertices the BFS handles, ascending (when few enough)
  u32* d_first = nullptr;      // first neighbour of every vertex (single graphs)
  u32* d_hot = nullptr;        // hot table: the n_hot highest-degree vertices
  int* d_hot_center = nullptr; // their labels, gathered per cut count
  int4* d_lab4 = nullptr;      // batches: up to four labelings packed per vertex (fused cut counts)
  int4* d_hot4 = nullptr;      // ... the hot table's packed labels
  int4* d_grp4 = nullptr;      // ... every cut-list group's packed cold label
  u32 n_hot = 0;
  u32* d_excl = nullptr;      // bit v: v is not handled by the BFS (no arcs or a small component)
  u32* d_solo = nullptr;      // bit v: v is alone in its component (inside the d_excl allocation)
  SmallComps sc;              // components of 2..32 vertices, solved one warp each
  // scratch arena
  void* arena = nullptr;
  double* d_shift = nullptr;
  int* d_a = nullptr;
  u64* d_k[2] = {nullptr, nullptr};
  u32* d_v[2] = {nullptr, nullptr};
  u64* d_status = nullptr;
  u32* d_order = nullptr;
  u64* d_key = nullptr;
  u32* d_qv[2] = {nullptr, nullptr};
  int* d_qrow[2] = {nullptr, nullptr};
  u32* d_qoff[2] = {nullptr, nullptr};
  u32* d_cf[2] = {nullptr, nullptr};
  u32* d_ulist[2] = {nullptr, nullptr};
  void* d_slots = nullptr;
  int* d_center = nullptr;
  int* d_dist = nullptr;
  Control* d_ctl = nullptr;
  int* d_bptr = nullptr;
  u32* d_rcur = nullptr;
  u32* d_acnt = nullptr;       // start-round counts by floor value (all zero between calls)
  bool acnt_dirty = true;      // d_acnt may hold counts: clear before the next fast path
  u32 bptr_cap = 0;
  size_t status_bytes = 0;
  u32 epoch = 0;
  // host side
  unsigned char* h_hdr = nullptr;  // pinned copy of the control header
  unsigned char* h_bhdr = nullptr;  // pinned headers of a pipelined batch, one per decomposition
  int h_bhdr_cap = 0;
  int bfs_grid = 0;
  int bfs_per_sm = 0;
  u32 spin_limit = 0;
  u32 lookback_limit = 1u << 24;  // polls of a look-back wait (fraction rank scans)
  u32 stall_barrier = 0;          // ldd_set_wait_limits: timeout-path tests
  u32 stall_lookback = 0;
  u32 pull_alpha = 0;
  u32 pull_beta = 0;
  u32 pull_gamma = 0;
  u32 probe_min_arcs = 1u << 16;
  u32 max_degree = 0;          // largest row of the CSR (unions: of any member)
  bool low_degree_rounds = true;  // tuning: low-degree rounds when max_degree allows
  u32 window_levels = 0;          // tuning: levels per window in low-degree rounds (0: none)
  u32 window_max_q = 1u << 18;    // tuning: windows only for frontiers up to this size
  u32 window_queue = 0;           // tuning: local-queue entries per CTA and level (0: all that fit)
  u32 bfs_span = kBfsMaxSpan;     // tuning: arcs per CTA step of an edge-balanced round
  bool timing = false;
  cudaEvent_t ev[8] = {};
  BfsGate* gate = nullptr;       // set by the request server on its workspaces
  cudaEvent_t ev_gate = nullptr;  // ... recorded after this graph's round loop
  // pipelined batches (ldd_decompose_batch), set up on first use
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaStream_t cut_stream = nullptr;  // cut counts, overlapping the next decomposition's rank
  cudaEvent_t ev_in[2] = {}, ev_used[2] = {}, ev_out[2] = {}, ev_cut[2] = {};
  static constexpr int kUploadChunks = 4;  // the first shift vector of a batch, uploaded in pieces
  cudaEvent_t ev_chunk[kUploadChunks] = {};
  u64* d_bcut = nullptr;              // [h_bhdr_cap] cut counts of a batch (device)
  u64* h_bcut = nullptr;              // [h_bhdr_cap] their pinned copy
  void* batch_arena = nullptr;  // two shift slots (8n each) and two output slots (8n each)
  // disjoint unions (ldd_create_union): member offsets and caller-layout staging
  struct Union {
    UnionCaps cap;                 // capacities the tables were allocated for
    u32 k = 0;
    u32 total = 0;                 // n_0 + ... + n_{k-1}: caller-layout length
    std::vector<u32> h_ooff;       // caller-layout offsets, k + 1
    std::vector<u32> h_voff;       // union-vertex offsets, k + 1
    UnionMember* d_mem = nullptr;  // k member views (valid only while building)
    u32* d_offs = nullptr;         // 8 arrays of cap.k + 1: v, e, u, c, m, a, o, g
    u32* d_active_buf = nullptr;   // [cap.N] active list (g->d_active when every member has one)
    UnionOffsets off{};
    double* d_shift_in = nullptr;  // [total] caller-layout shifts from the host
    int* d_out_c = nullptr;        // [total] caller-layout labels (host outputs, cut count)
    int* d_out_d = nullptr;        // [total]
    u64* d_cut = nullptr;          // [k]
    u32* d_wmem = nullptr;         // [N / 32] member of every 32-vertex word
    int* d_amax = nullptr;         // [k] largest floor of each member, then [k] its lift
    u32* d_mrank = nullptr;        // [3][k] the round loop's per-member bottom-up floors
  };
  Union* uni = nullptr;
  // block decomposition (ldd_block_decompose, ldd_blocks.cu): residual graphs,
  // created on the first call
  ldd::Blocks* blk = nullptr;
  // captured CUDA graph of one fast-path decomposition (ldd_set_graph_replay)
  bool replay = false;
  bool replay_broken = false;        // capture failed once: regular path only
  int regular_runs = 0;              // regular decompositions so far (capture waits for one)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec[2] = {};     // [with union cut counts]
  int replay_launches[2] = {};
  u64* h_cut = nullptr;              // pinned copy of a union's cut counts
  ldd_stats stats;
};

namespace ldd {

// Frees every device and host resource of g (not g itself).
int free_graph_memory(ldd_graph* g);
// Scratch arena, pinned header, events and launch parameters of a graph whose
// sizes (n, nnz, device, num_sms) are set (ldd_api.cu).
int finish_setup(ldd_graph* g);
// The block decomposition's state of g (ldd_blocks.cu); null is a no-op.
void free_blocks(ldd_graph* g);
void record(ldd_graph* g, int i);
float elapsed(ldd_graph* g, int a, int b);
// One decomposition on g's stream from device shifts into device outputs
// (union: caller layout), with the fast rank path's retries; synchronises.
// d_levels, d_perm: the ranked variant (integer levels and a tie-break
// permutation in place of FP64 shifts); else null.
int decompose_on_device(ldd_graph* g, const double* d_shift, int* center, int* dist,
                        int* launches_out, const int* d_levels = nullptr,
                        const int* d_perm = nullptr);

// Sizes a union would need for these members.
UnionCaps union_needs(int k, ldd_graph* const* members);
// Device bytes union_alloc takes for caps (tables, scratch, staging).
u64 union_bytes(const UnionCaps& c);
// A fresh union graph object with room for caps on device dev.
int union_alloc(ldd_graph** out, int dev, const UnionCaps& caps);
// Fills u from members on stream s (members' tables are read by kernels on
// s: keep them alive until s has finished); sync: wait for s.
int union_fill(ldd_graph* u, int k, ldd_graph* const* members, cudaStream_t s, bool sync);
// Shifts (caller layout, device) spread, decomposition, and optionally the
// members' cut counts into u's d_cut; outputs in the caller layout (device).
int union_run(ldd_graph* u, const double* d_in, int* center, int* dist, bool want_cut,
              int* launches_out, int* cut_launches_out);

// Cut counts (Definition 1.1) of K = 1 .. 4 labelings centers[0 .. K) of one
// graph in one pass over its cut list (k_graph.cu): the labelings are packed
// into lab4 [n], the hot table's and the groups' packed labels gathered into
// hot4 [n_hot] and grp4 [cl.ngrp], and out[i] += the count of labeling i.
// Returns the kernels queued on s.
int launch_cut4(const CutList& cl, const int* const* centers, int K, u32 n, const u32* hot,
                u32 n_hot, int4* lab4, int4* hot4, int4* grp4, u64* out, int num_sms,
                cudaStream_t s);

}  // namespace ldd

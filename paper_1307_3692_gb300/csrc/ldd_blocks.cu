// ldd_block_decompose: blocks by repeated low-diameter decomposition.
//
// Section 1 (related work) of Miller, Peng, Xu 2013 notes that the block
// decomposition of Linial and Saks -- O(log n) blocks whose connected pieces
// have diameter O(log n) -- follows from running a (1/2, O(log n))
// decomposition again and again on the edges not yet in a block: each run
// cuts at most half of what is left in expectation (Corollary 3.5 bounds the
// fraction by 1 - e^{-beta}).  Iteration i decomposes G_i = (V, E_i) with the
// caller's shift vector i; the edges of E_i whose two ends share a piece form
// block i, and the cut ones are E_{i+1}.
//
// Everything stays on the device.  G_0 is the graph itself.  After
// decomposition i, one pass over G_i's arcs (k_residual_count in k_graph.cu,
// arc-parallel with the arcs' source vertices) stamps block i on the arcs
// inside pieces and lists the others; a pass over that list writes them, with
// their input arc ids and sources, as G_{i+1}'s CSR and hooks G_{i+1}'s
// union-find forest, so its component tables (the small-component solver and
// the round loop's exclusion bits) follow without another pass over the
// arcs.  G_1, G_2, ... share one graph object with ping-pong CSR buffers, all
// sized by the input, allocated on the first call (with G_0's arc sources)
// and kept on the input graph until it is destroyed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "../../include/ldd.h"
#include "ldd_graph.cuh"

namespace ldd {

struct Blocks {
  ldd_graph* r = nullptr;      // graph object of G_i, i >= 1
  int* row[2] = {};            // [n + 1]: kept-arc counts, then G_{i+1}'s row offsets
  int* col[2] = {};            // [nnz]
  int* orig[2] = {};           // [nnz] input arc id of every arc of G_i
  int* src[2] = {};            // [nnz] source vertex of every arc of G_i, i >= 1
  u32* map[2] = {};            // [n] input id of every vertex of G_i, i >= 1
  int* off = nullptr;          // [n + 1] kept arcs per vertex of G_i, then their offsets
  u32* cid = nullptr;          // [n + 1] vertices with kept arcs, then their ids in G_{i+1}
  int* src0 = nullptr;         // [nnz] source vertex of every arc of G_0
  u32* klist = nullptr;        // [nnz] the count pass's kept arcs
  u32* cursor = nullptr;       // [n + 1] the write pass's next place per row
  int* arc_block = nullptr;    // [nnz] block of every input arc (when the caller's is not on the device)
  u32* tmp = nullptr;          // union-find and component scratch
  CompScratch t{};
  unsigned long long* up = nullptr;  // undirected edges left (device counter)
  u32* n_kept = nullptr;
  unsigned long long* h_up = nullptr;  // pinned: [0] edges left, [1] arcs left
  cudaEvent_t ev[4] = {};      // call start / end, residual passes start / end
};

void free_blocks(ldd_graph* g) {
  Blocks* b = g->blk;
  if (!b) return;
  if (b->r) {
    // the CSR and the small-component lists belong to b, not to r
    b->r->d_row = nullptr;
    b->r->d_col = nullptr;
    b->r->sc.comp_off = b->r->sc.comp_len = b->r->sc.comp_v = nullptr;
    free_graph_memory(b->r);
    delete b->r;
  }
  for (int j = 0; j < 2; ++j) {
    cudaFree(b->row[j]);
    cudaFree(b->col[j]);
    cudaFree(b->orig[j]);
    cudaFree(b->src[j]);
    cudaFree(b->map[j]);
  }
  cudaFree(b->off);
  cudaFree(b->cid);
  cudaFree(b->src0);
  cudaFree(b->klist);
  cudaFree(b->cursor);
  cudaFree(b->arc_block);
  cudaFree(b->tmp);
  cudaFree(b->up);
  cudaFree(b->n_kept);
  if (b->h_up) cudaFreeHost(b->h_up);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  delete b;
  g->blk = nullptr;
}

namespace {

int setup_blocks(ldd_graph* g) {
  if (g->blk) return LDD_OK;
  Blocks* b = new (std::nothrow) Blocks();
  if (!b) return fail(LDD_ERR_OOM, "host allocation failed");
  g->blk = b;
  const size_t n = (size_t)g->n, nnz = std::max<size_t>((size_t)g->nnz, 1);
  const size_t words = std::max<size_t>((n + 31) / 32, 1);
  bool ok = true;
  for (int j = 0; j < 2; ++j)
    ok = ok && cudaMalloc(&b->row[j], (n + 1) * 4) == cudaSuccess &&
         cudaMalloc(&b->col[j], nnz * 4) == cudaSuccess &&
         cudaMalloc(&b->orig[j], nnz * 4) == cudaSuccess &&
         cudaMalloc(&b->src[j], nnz * 4) == cudaSuccess &&
         cudaMalloc(&b->map[j], std::max<size_t>(n, 1) * 4) == cudaSuccess;
  ok = ok && cudaMalloc(&b->off, (n + 1) * 4) == cudaSuccess &&
       cudaMalloc(&b->cid, (n + 1) * 4) == cudaSuccess;
  ok = ok && cudaMalloc(&b->src0, nnz * 4) == cudaSuccess &&
       cudaMalloc(&b->klist, nnz * 4) == cudaSuccess &&
       cudaMalloc(&b->cursor, (n + 1) * 4) == cudaSuccess &&
       cudaMalloc(&b->arc_block, nnz * 4) == cudaSuccess &&
       cudaMalloc(&b->tmp, (7 * n + 2 * (n / 2 + 1) + 4) * 4) == cudaSuccess &&
       cudaMalloc(&b->up, sizeof(unsigned long long)) == cudaSuccess &&
       cudaMalloc(&b->n_kept, 4) == cudaSuccess &&
       cudaMallocHost(&b->h_up, 2 * sizeof(unsigned long long)) == cudaSuccess;
  for (auto& e : b->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_blocks(g);
    return fail(LDD_ERR_OOM, "device allocation for the block decomposition failed");
  }
  CompScratch& t = b->t;
  t.parent = b->tmp;
  t.csize = b->tmp + n;
  t.root_off = b->tmp + 2 * n;
  t.fill = b->tmp + 3 * n;
  t.lane_of = b->tmp + 4 * n;
  t.comp_v = b->tmp + 5 * n;
  t.comp_off = b->tmp + 6 * n;
  t.comp_len = t.comp_off + (n / 2 + 1);
  t.counters = t.comp_len + (n / 2 + 1);
  // the residual graph object: sizes of the input (upper bounds), own scratch
  ldd_graph* r = new (std::nothrow) ldd_graph();
  if (!r) {
    free_blocks(g);
    return fail(LDD_ERR_OOM, "host allocation failed");
  }
  b->r = r;
  memset(&r->stats, 0, sizeof(r->stats));
  r->n = g->n;
  r->nnz = g->nnz;
  r->device = g->device;
  r->num_sms = g->num_sms;
  if (cudaMalloc(&r->d_excl, 2 * words * 4) != cudaSuccess ||
      cudaMalloc(&r->sc.adj, std::max<size_t>(n, 1) * 4) != cudaSuccess) {
    cudaGetLastError();
    free_blocks(g);
    return fail(LDD_ERR_OOM, "device allocation for the block decomposition failed");
  }
  r->d_solo = r->d_excl + words;
  int rc = finish_setup(r);
  if (rc != LDD_OK) {
    free_blocks(g);
    return rc;
  }
  launch_fill_src(g->d_row, (u32)n, b->src0, g->num_sms, g->stream);
  if (cudaGetLastError() != cudaSuccess) {
    free_blocks(g);
    return fail(LDD_ERR_CUDA, "arc sources of the graph");
  }
  return LDD_OK;
}

// The residual graph object takes the input graph's stream and launch
// parameters (tuning and wait limits) for the coming iterations.
void sync_params(ldd_graph* g, ldd_graph* r) {
  r->stream = g->stream;
  r->timing = false;
  r->spin_limit = g->spin_limit;
  r->lookback_limit = g->lookback_limit;
  r->stall_barrier = g->stall_barrier;
  r->stall_lookback = g->stall_lookback;
  r->pull_alpha = g->pull_alpha;
  r->pull_beta = g->pull_beta;
  r->pull_gamma = g->pull_gamma;
  r->probe_min_arcs = g->probe_min_arcs;
  r->low_degree_rounds = g->low_degree_rounds;
  r->max_degree = g->max_degree;  // residual rows are never longer
}

}  // namespace
}  // namespace ldd

extern "C" int ldd_block_decompose(ldd_graph* g, int k, const double* betas,
                                   const double* const* shifts, int32_t* const* out_center,
                                   int32_t* const* out_dist, int32_t* out_arc_block,
                                   int64_t* out_remaining, int32_t* out_blocks) {
  using namespace ldd;
  record_error("");  // this call's failures only
  if (out_blocks) *out_blocks = 0;
  if (!g || !out_blocks) return fail(LDD_ERR_ARG, "NULL graph or out_blocks");
  if (g->uni) return fail(LDD_ERR_ARG, "a union graph has no block decomposition");
  if (k < 0) return fail(LDD_ERR_ARG, "k = %d is negative", k);
  if (k > 0 && (!betas || !shifts)) return fail(LDD_ERR_ARG, "NULL betas or shifts");
  for (int i = 0; i < k; ++i) {
    if (!(betas[i] > 0.0) || isinf(betas[i]))
      return fail(LDD_ERR_ARG, "betas[%d] must be finite and > 0", i);
    if (g->n > 0 && !shifts[i]) return fail(LDD_ERR_ARG, "shifts[%d] is NULL", i);
    if (g->n > 0 && out_center && !out_center[i])
      return fail(LDD_ERR_ARG, "out_center[%d] is NULL", i);
    if (g->n > 0 && out_dist && !out_dist[i]) return fail(LDD_ERR_ARG, "out_dist[%d] is NULL", i);
  }
  if (out_remaining) out_remaining[0] = (int64_t)g->m_up;
  if (g->n == 0 || g->nnz == 0 || k == 0) return LDD_OK;
  DeviceGuard dg(g->device);
  if (!dg.ok) return fail(LDD_ERR_CUDA, "cannot select device %d", g->device);
  int rc = setup_blocks(g);
  if (rc != LDD_OK) return rc;
  Blocks& B = *g->blk;
  ldd_graph* r = B.r;
  sync_params(g, r);
  cudaStream_t s = g->stream;
  const size_t n = (size_t)g->n;
  const bool dev_blk = out_arc_block && is_device_ptr(out_arc_block);
  int* arc_block = dev_blk ? out_arc_block : B.arc_block;
  CUDA_TRY(cudaEventRecord(B.ev[0], s));
  CUDA_TRY(cudaMemsetAsync(arc_block, 0xff, (size_t)g->nnz * 4, s));
  float ms_residual = 0.f;
  u64 arcs_scanned = 0, arcs_kept = 0;
  auto residual_ms = [&]() {
    float ms = 0.f;
    if (cudaEventSynchronize(B.ev[3]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, B.ev[2], B.ev[3]) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.f;
    }
    return ms;
  };
  ldd_graph* cur = g;  // G_i
  const int* cur_src = B.src0;
  const int* cur_col = g->d_col;
  const int* cur_orig = nullptr;  // G_0's arcs are the input arcs
  const u32* cur_map = nullptr;   // G_0's vertices are the input vertices
  u32 cur_m = (u32)g->nnz, cur_n = (u32)n;
  int blocks = 0;
  for (int i = 0; i < k; ++i) {
    // decomposition i of G_i, then its results over all n input vertices
    const double* d_shift = shifts[i];
    if (!is_device_ptr(shifts[i])) {
      CUDA_TRY(cudaMemcpyAsync(g->d_shift, shifts[i], n * 8, cudaMemcpyHostToDevice, s));
      d_shift = g->d_shift;
    }
    if (cur != g) {  // G_i's own vertices only
      launch_gather_shifts(d_shift, cur_map, cur_n, r->d_shift, g->num_sms, s);
      d_shift = r->d_shift;
    }
    const bool dev_c = out_center && is_device_ptr(out_center[i]);
    const bool dev_d = out_dist && is_device_ptr(out_dist[i]);
    int* center = dev_c ? out_center[i] : g->d_center;
    int* dist = dev_d ? out_dist[i] : g->d_dist;
    int* cur_center = cur == g ? center : r->d_center;  // in G_i's ids
    int launches = 0;
    if ((rc = decompose_on_device(cur, d_shift, cur_center, cur == g ? dist : r->d_dist,
                                  &launches)) != LDD_OK) {
      cudaStreamSynchronize(s);
      *out_blocks = blocks;
      return rc;
    }
    if (cur != g)
      launch_blocks_output(r->d_center, r->d_dist, cur_map, cur_n, (u32)n, center, dist,
                           g->num_sms, s);
    if (out_center && !dev_c)
      CUDA_TRY(cudaMemcpyAsync(out_center[i], center, n * 4, cudaMemcpyDeviceToHost, s));
    if (out_dist && !dev_d)
      CUDA_TRY(cudaMemcpyAsync(out_dist[i], dist, n * 4, cudaMemcpyDeviceToHost, s));
    blocks = i + 1;
    // block i and G_{i+1}; r's control block and look-back words serve the scans
    const int j = i & 1;
    CUDA_TRY(cudaEventRecord(B.ev[2], s));
    CUDA_TRY(cudaMemsetAsync(r->d_ctl, 0, sizeof(Control), s));
    CUDA_TRY(cudaMemsetAsync(B.off, 0, ((size_t)cur_n + 1) * 4, s));
    CUDA_TRY(cudaMemsetAsync(B.up, 0, sizeof(unsigned long long), s));
    CUDA_TRY(cudaMemsetAsync(B.n_kept, 0, 4, s));
    if (r->epoch > 0xfffff000u) {
      CUDA_TRY(cudaMemsetAsync(r->d_status, 0, r->status_bytes, s));
      r->epoch = 0;
    }
    launch_residual(false, cur_src, cur_col, cur_orig, cur_center, cur_n, cur_m, i, arc_block,
                    reinterpret_cast<u32*>(B.off), B.up, B.klist, B.n_kept, nullptr, nullptr,
                    nullptr, nullptr, nullptr, nullptr, g->num_sms, s);
    launch_exclusive_scan(reinterpret_cast<u32*>(B.off), cur_n + 1, r->d_status, &r->epoch,
                          &r->d_ctl->tile_ctr[0], r->d_ctl, r->lookback_limit, s, B.cursor);
    // G_{i+1} keeps the vertices with kept arcs, numbered in their order
    launch_kept_flags(B.off, cur_n, B.cid, g->num_sms, s);
    launch_exclusive_scan(B.cid, cur_n + 1, r->d_status, &r->epoch, &r->d_ctl->tile_ctr[1],
                          r->d_ctl, r->lookback_limit, s);
    CUDA_TRY(cudaMemcpyAsync(B.h_up, B.up, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(B.h_up + 1, B.off + cur_n, 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<u32*>(B.h_up + 1) + 1, B.cid + cur_n, 4,
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(r->h_hdr, r->d_ctl, 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaEventRecord(B.ev[3], s));
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s));
    ms_residual += residual_ms();
    arcs_scanned += cur_m;
    u32 err;
    memcpy(&err, r->h_hdr, 4);
    if (err) {
      *out_blocks = blocks;
      return (err & kErrTimeout) ? fail(LDD_ERR_TIMEOUT, "a device-side wait ran out")
                                 : fail(LDD_ERR_CUDA, "device error bits 0x%x", err);
    }
    const u64 edges_left = B.h_up[0];
    const u32 arcs_left = (u32)B.h_up[1];
    const u32 n_next = (u32)(B.h_up[1] >> 32);
    if (out_remaining) out_remaining[i + 1] = (int64_t)edges_left;
    if (arcs_left == 0 || i + 1 == k) break;
    // G_{i+1}: rows and vertex ids, arcs, component forest, component tables
    arcs_kept += arcs_left;
    CUDA_TRY(cudaEventRecord(B.ev[2], s));
    launch_compact_rows(B.off, B.cid, cur_n, B.row[j], cur_map, B.map[j], g->num_sms, s);
    cudaError_t e = components_init(n_next, g->num_sms, B.t, r->d_excl, r->d_solo, s);
    if (e != cudaSuccess) return fail(LDD_ERR_CUDA, "component set-up: %s", cudaGetErrorString(e));
    launch_residual(true, cur_src, cur_col, cur_orig, cur_center, cur_n, cur_m, i, nullptr,
                    nullptr, nullptr, B.klist, B.n_kept, B.cursor, B.cid, B.col[j], B.orig[j],
                    B.src[j], B.t.parent, g->num_sms, s);
    u32 counts[4] = {0, 0, 0, 0};
    e = components_label(B.row[j], n_next, g->num_sms, B.t, r->d_excl, r->d_solo, counts, s);
    if (e != cudaSuccess) return fail(LDD_ERR_CUDA, "component labelling: %s", cudaGetErrorString(e));
    r->n = (int32_t)n_next;
    r->sc.ncomp = counts[0];
    r->sc.total = counts[1];
    r->sc.comp_off = B.t.comp_off;
    r->sc.comp_len = B.t.comp_len;
    r->sc.comp_v = B.t.comp_v;
    r->n_active = counts[2];
    r->nnz_active = counts[3];
    r->m_up = (u32)edges_left;
    r->d_row = B.row[j];
    r->d_col = B.col[j];
    if ((e = components_phase2(r->d_row, r->d_col, B.t, r->sc, g->num_sms, s)) != cudaSuccess)
      return fail(LDD_ERR_CUDA, "component adjacency: %s", cudaGetErrorString(e));
    CUDA_TRY(cudaEventRecord(B.ev[3], s));
    ms_residual += residual_ms();
    r->nnz = (int64_t)arcs_left;
    cur = r;
    cur_src = B.src[j];
    cur_col = B.col[j];
    cur_orig = B.orig[j];
    cur_map = B.map[j];
    cur_m = arcs_left;
    cur_n = n_next;
  }
  if (out_arc_block && !dev_blk)
    CUDA_TRY(cudaMemcpyAsync(out_arc_block, arc_block, (size_t)g->nnz * 4, cudaMemcpyDeviceToHost,
                             s));
  CUDA_TRY(cudaEventRecord(B.ev[1], s));
  CUDA_TRY(cudaStreamSynchronize(s));
  float ms_total = -1.f;
  if (cudaEventElapsedTime(&ms_total, B.ev[0], B.ev[1]) != cudaSuccess) {
    cudaGetLastError();
    ms_total = -1.f;
  }
  g->stats.ms_block_total = ms_total;
  g->stats.ms_block_residual = ms_residual;
  g->stats.block_arcs_scanned = (int64_t)arcs_scanned;
  g->stats.block_arcs_kept = (int64_t)arcs_kept;
  *out_blocks = blocks;
  return LDD_OK;
}

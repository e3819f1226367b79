// C ABI of libldd.so (declared in include/ldd.h): the graph object, argument
// checks, host/device pointer handling, scratch memory and the order of the
// kernels of one decomposition (Miller, Peng, Xu 2013, Algorithm 1):
//   step 1 (shifts)      : given by the caller, copied to the device if needed
//   step 2 (delta_max)   : the split of k_bplace / k_split64   (k_rank.cu)
//   Section 4 tie-break  : fraction rank, keys, start buckets  (k_rank.cu)
//   step 3 (BFS)         : persistent cooperative k_bfs        (k_bfs.cu)
//                          and k_small_comp for components of <= 32 vertices
//   step 4 (assignment)  : k_finalize                          (k_graph.cu)
// and of the entry points built on it: cut counts (Definition 1.1), the
// permutation variant and the retry loop (Section 4, Theorem 1.2's proof),
// pipelined batches, disjoint unions (k_union.cu), CUDA-graph replay of the
// fast path, and launch-parameter tuning.  The request server is in
// ldd_server.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <vector>

#include "../../include/ldd.h"
#include "ldd_graph.cuh"

using namespace ldd;

static_assert(offsetof(Control, bar) == kCtlBfsStateOffset, "control layout");
static_assert(offsetof(Control, mask_f) == kCtlBfsStateOffset + kCtlBfsStateBytes,
              "control layout");
static_assert(offsetof(Control, cut) + sizeof(u64) == kCtlHeaderBytes, "control layout");
static_assert(offsetof(Control, minrank) == kCtlMinrankOffset, "control layout");

namespace ldd {

thread_local char g_last_error[512] = "";

int fail(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return status;
}

// True for device or managed memory; false for pageable or pinned host memory.
bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

u32 env_u32(const char* name, u32 dflt) {
  const char* v = getenv(name);
  if (!v || !*v) return dflt;
  char* end = nullptr;
  unsigned long x = strtoul(v, &end, 10);
  return (end && *end == 0 && x > 0 && x <= 0xffffffffUL) ? (u32)x : dflt;
}

// Sets the text ldd_last_error() returns on this thread (used by entry points
// defined in other translation units).
void record_error(const char* msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }
}  // namespace ldd


namespace ldd {

int free_graph_memory(ldd_graph* g) {
  free_blocks(g);
  cudaFree(g->d_row);
  cudaFree(g->d_col);
  cudaFree(g->cut.hot);
  cudaFree(g->cut.grp_off);
  cudaFree(g->cut.grp_v);
  cudaFree(g->cut.blk_g);
  cudaFree(g->cut.blk_mask);
  cudaFree(g->cut.grp_m);
  cudaFree(g->cut.grp_lab);
  cudaFree(g->d_hot);
  if (!g->uni) cudaFree(g->d_active);  // a union's list lives in d_active_buf
  cudaFree(g->d_first);
  cudaFree(g->d_hot_center);
  cudaFree(g->d_lab4);
  cudaFree(g->d_hot4);
  cudaFree(g->d_grp4);
  cudaFree(g->d_excl);
  cudaFree(g->sc.comp_off);
  cudaFree(g->sc.comp_len);
  cudaFree(g->sc.comp_v);
  cudaFree(g->sc.adj);
  cudaFree(g->arena);
  cudaFree(g->d_bptr);
  cudaFree(g->d_rcur);
  cudaFree(g->d_acnt);
  cudaFree(g->batch_arena);
  if (g->h_hdr) cudaFreeHost(g->h_hdr);
  if (g->h_bhdr) cudaFreeHost(g->h_bhdr);
  if (g->h_bcut) cudaFreeHost(g->h_bcut);
  cudaFree(g->d_bcut);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  if (g->ev_gate) cudaEventDestroy(g->ev_gate);
  for (int i = 0; i < 2; ++i) {
    if (g->ev_in[i]) cudaEventDestroy(g->ev_in[i]);
    if (g->ev_used[i]) cudaEventDestroy(g->ev_used[i]);
    if (g->ev_out[i]) cudaEventDestroy(g->ev_out[i]);
  }
  if (g->copy_in) cudaStreamDestroy(g->copy_in);
  if (g->copy_out) cudaStreamDestroy(g->copy_out);
  if (g->cut_stream) cudaStreamDestroy(g->cut_stream);
  for (int i = 0; i < 2; ++i)
    if (g->ev_cut[i]) cudaEventDestroy(g->ev_cut[i]);
  for (auto& e : g->ev_chunk)
    if (e) cudaEventDestroy(e);
  for (auto& x : g->gexec)
    if (x) cudaGraphExecDestroy(x);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  if (g->h_cut) cudaFreeHost(g->h_cut);
  if (g->uni) {
    cudaFree(g->uni->d_active_buf);
    cudaFree(g->uni->d_mem);
    cudaFree(g->uni->d_offs);
    cudaFree(g->uni->d_shift_in);
    cudaFree(g->uni->d_out_c);
    cudaFree(g->uni->d_cut);
    cudaFree(g->uni->d_wmem);
    cudaFree(g->uni->d_amax);
    cudaFree(g->uni->d_mrank);
    delete g->uni;
    g->uni = nullptr;
  }
  return 0;
}

// Host-side CSR check: bounds, monotone rows, every arc has its reverse.
int validate_csr(int32_t n, int64_t nnz, const int32_t* rp, const int32_t* col) {
  if (rp[0] != 0) return fail(LDD_ERR_GRAPH, "row_ptr[0] = %d, expected 0", rp[0]);
  if ((int64_t)rp[n] != nnz)
    return fail(LDD_ERR_GRAPH, "row_ptr[n] = %d, expected nnz = %lld", rp[n], (long long)nnz);
  for (int32_t v = 0; v < n; ++v)
    if (rp[v + 1] < rp[v]) return fail(LDD_ERR_GRAPH, "row_ptr decreases at vertex %d", v);
  for (int64_t e = 0; e < nnz; ++e)
    if (col[e] < 0 || col[e] >= n)
      return fail(LDD_ERR_GRAPH, "col_idx[%lld] = %d out of [0, %d)", (long long)e, col[e], n);
  std::vector<int32_t> sorted(col, col + nnz);
  for (int32_t v = 0; v < n; ++v) std::sort(sorted.begin() + rp[v], sorted.begin() + rp[v + 1]);
  for (int32_t v = 0; v < n; ++v)
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
      const int32_t w = col[e];
      if (!std::binary_search(sorted.begin() + rp[w], sorted.begin() + rp[w + 1], v))
        return fail(LDD_ERR_GRAPH, "arc (%d, %d) has no reverse arc: the graph must be undirected",
                    v, w);
    }
  return LDD_OK;
}

int alloc_scratch(ldd_graph* g) {
  const size_t n = (size_t)g->n;
  const size_t nk = std::max<size_t>(n, 64);  // 64-bit words per key buffer
  const size_t ntiles = (n + kSortTile - 1) / kSortTile + 1;
  const size_t ncf = (size_t)g->nnz / kBfsBase + 2;
  g->status_bytes = ntiles * 256 * sizeof(u64);
  struct Part {
    void** p;
    size_t bytes;
  } parts[] = {
      {(void**)&g->d_shift, 8 * n},       {(void**)&g->d_a, 4 * n},
      {(void**)&g->d_k[0], 8 * nk},       {(void**)&g->d_k[1], 8 * nk},
      {(void**)&g->d_v[0], 4 * n},        {(void**)&g->d_v[1], 4 * n},
      {(void**)&g->d_status, g->status_bytes},
      {(void**)&g->d_order, 4 * n},       {(void**)&g->d_key, 8 * n},
      {(void**)&g->d_qv[0], 4 * n},       {(void**)&g->d_qv[1], 4 * n},
      {(void**)&g->d_qrow[0], 4 * n},     {(void**)&g->d_qrow[1], 4 * n},
      {(void**)&g->d_qoff[0], 4 * n},     {(void**)&g->d_qoff[1], 4 * n},
      {(void**)&g->d_cf[0], 4 * ncf},     {(void**)&g->d_cf[1], 4 * ncf},
      {(void**)&g->d_ulist[0], 4 * n},    {(void**)&g->d_ulist[1], 4 * n},
      {(void**)&g->d_slots, n ? fraction_slot_bytes((u32)n) : 0},
      {(void**)&g->d_center, 4 * n},      {(void**)&g->d_dist, 4 * n},
      {(void**)&g->d_ctl, sizeof(Control)},
  };
  size_t total = 0;
  for (auto& p : parts) total += align_up(p.bytes ? p.bytes : 1, 256);
  if (cudaMalloc(&g->arena, total) != cudaSuccess) {
    cudaGetLastError();
    return fail(LDD_ERR_OOM, "cudaMalloc of %zu bytes of scratch failed", total);
  }
  size_t off = 0;
  for (auto& p : parts) {
    *p.p = (char*)g->arena + off;
    off += align_up(p.bytes ? p.bytes : 1, 256);
  }
  CUDA_TRY(cudaMemset(g->d_status, 0, g->status_bytes));
  g->bptr_cap = (u32)std::min<size_t>(n + 2, 0xffffffffu);
  g->acnt_dirty = true;  // cleared by the first fast-path attempt
  if (cudaMalloc(&g->d_bptr, (size_t)g->bptr_cap * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&g->d_rcur, (size_t)g->bptr_cap * sizeof(u32)) != cudaSuccess ||
      cudaMalloc(&g->d_acnt, (size_t)g->bptr_cap * sizeof(u32)) != cudaSuccess) {
    cudaGetLastError();
    return fail(LDD_ERR_OOM, "cudaMalloc of the start-bucket table failed");
  }
  return LDD_OK;
}

// Component labels and the small-component tables (two device phases, the
// table sizes read back in between).
int build_component_tables(ldd_graph* g) {
  const size_t n = (size_t)g->n;
  const size_t words = std::max<size_t>((n + 31) / 32, 1);
  if (cudaMalloc(&g->d_excl, 2 * words * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(LDD_ERR_OOM, "device allocation of the exclusion bitmasks failed");
  }
  g->d_solo = g->d_excl + words;
  if (n == 0) return LDD_OK;
  u32* tmp = nullptr;
  if (cudaMalloc(&tmp, (7 * n + 2 * (n / 2 + 1) + 4) * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(LDD_ERR_OOM, "device allocation for component labelling failed");
  }
  CompScratch t;
  t.parent = tmp;
  t.csize = tmp + n;
  t.root_off = tmp + 2 * n;
  t.fill = tmp + 3 * n;
  t.lane_of = tmp + 4 * n;
  t.comp_v = tmp + 5 * n;
  t.comp_off = tmp + 6 * n;
  t.comp_len = t.comp_off + (n / 2 + 1);
  t.counters = t.comp_len + (n / 2 + 1);
  u32 counts[4] = {0, 0, 0, 0};
  cudaError_t e = components_from_csr(g->d_row, g->d_col, (u32)n, g->num_sms, t, g->d_excl,
                                      g->d_solo, counts, nullptr);
  int rc = LDD_OK;
  SmallComps& sc = g->sc;
  if (e != cudaSuccess) {
    rc = fail(LDD_ERR_CUDA, "component labelling failed: %s", cudaGetErrorString(e));
  } else {
    sc.ncomp = counts[0];
    sc.total = counts[1];
    g->n_active = counts[2];
    g->nnz_active = counts[3];
    if (sc.ncomp > 0 &&
        (cudaMalloc(&sc.comp_off, sc.ncomp * 4) != cudaSuccess ||
         cudaMalloc(&sc.comp_len, sc.ncomp * 4) != cudaSuccess ||
         cudaMalloc(&sc.comp_v, sc.total * 4) != cudaSuccess ||
         cudaMalloc(&sc.adj, sc.total * 4) != cudaSuccess)) {
      cudaGetLastError();
      rc = fail(LDD_ERR_OOM, "device allocation of the component tables failed");
    } else if (sc.ncomp > 0) {
      if (cudaMemcpy(sc.comp_off, t.comp_off, sc.ncomp * 4, cudaMemcpyDeviceToDevice) != cudaSuccess ||
          cudaMemcpy(sc.comp_len, t.comp_len, sc.ncomp * 4, cudaMemcpyDeviceToDevice) != cudaSuccess ||
          cudaMemcpy(sc.comp_v, t.comp_v, sc.total * 4, cudaMemcpyDeviceToDevice) != cudaSuccess)
        rc = fail(LDD_ERR_CUDA, "copy of the component tables failed");
      else if ((e = components_phase2(g->d_row, g->d_col, t, sc, g->num_sms, nullptr)) !=
               cudaSuccess)
        rc = fail(LDD_ERR_CUDA, "component adjacency failed: %s", cudaGetErrorString(e));
    }
  }
  cudaFree(tmp);
  return rc;
}

// The grouped cut list of launch_cut (CutList): each edge oriented from its
// cold endpoint to its hot one (larger degree, ties to the smaller id),
// grouped by the cold endpoint with a counting sort, and hot endpoints in the
// hot table encoded as (slot | 2^31).  With degree skew most label reads of
// the cut then hit the shared-memory copy of the hot table, the cold side is
// read once per group, and the edge stream is 4 bytes per edge.
int build_cut_list(ldd_graph* g, const std::vector<int32_t>& rp, const std::vector<int2>& up) {
  const size_t n = (size_t)g->n, m = up.size();
  CutList& cl = g->cut;
  cl.m = (u32)m;
  cl.nblk = (u32)((m + 31) / 32);
  auto deg = [&](int32_t v) { return rp[v + 1] - rp[v]; };
  auto hotter = [&](int32_t a, int32_t b) {
    const int32_t da = deg(a), db = deg(b);
    return da > db || (da == db && a < b);
  };
  const size_t K = m ? std::min<size_t>(kHotSlots, n) : 0;
  std::vector<int32_t> ids(n);
  for (size_t v = 0; v < n; ++v) ids[v] = (int32_t)v;
  if (K > 0 && K < n) std::nth_element(ids.begin(), ids.begin() + K, ids.end(), hotter);
  std::sort(ids.begin(), ids.begin() + K, hotter);
  std::vector<int32_t> slot(n, -1);
  for (size_t i = 0; i < K; ++i) slot[ids[i]] = (int32_t)i;
  std::vector<u32> start(n + 1, 0);
  for (const int2& e : up) ++start[(hotter(e.x, e.y) ? e.y : e.x) + 1];
  for (size_t v = 0; v < n; ++v) start[v + 1] += start[v];
  std::vector<u32> grp_off, grp_v;
  for (size_t v = 0; v < n; ++v)
    if (start[v + 1] > start[v]) {
      grp_v.push_back((u32)v);
      grp_off.push_back(start[v]);
    }
  cl.ngrp = (u32)grp_v.size();
  grp_off.push_back((u32)m);
  std::vector<int32_t> hot(m);
  for (const int2& e : up) {
    const bool xh = hotter(e.x, e.y);
    const int32_t h = xh ? e.x : e.y, cold = xh ? e.y : e.x;
    hot[start[cold]++] = slot[h] >= 0 ? (int32_t)(0x80000000u | (u32)slot[h]) : h;
  }
  std::vector<u32> blk_g(std::max<size_t>(cl.nblk, 1), 0), blk_mask(std::max<size_t>(cl.nblk, 1), 0);
  for (u32 gi = 0; gi < cl.ngrp; ++gi) {
    const u32 lo = grp_off[gi], hi = grp_off[gi + 1];
    if (lo & 31u) blk_mask[lo >> 5] |= 1u << (lo & 31u);
    for (u32 b = (lo + 31) / 32; b * 32 < hi; ++b) blk_g[b] = gi;
  }
  g->n_hot = (u32)K;
  if (cudaMalloc(&cl.hot, std::max<size_t>(m, 1) * 4) != cudaSuccess ||
      cudaMalloc(&cl.grp_off, grp_off.size() * 4) != cudaSuccess ||
      cudaMalloc(&cl.grp_v, std::max<size_t>(grp_v.size(), 1) * 4) != cudaSuccess ||
      cudaMalloc(&cl.grp_lab, std::max<size_t>(grp_v.size(), 1) * 4) != cudaSuccess ||
      cudaMalloc(&cl.blk_g, blk_g.size() * 4) != cudaSuccess ||
      cudaMalloc(&cl.blk_mask, blk_mask.size() * 4) != cudaSuccess ||
      cudaMalloc(&g->d_hot, std::max<size_t>(K, 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->d_hot_center, std::max<size_t>(K, 1) * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(LDD_ERR_OOM, "device allocation of the cut list failed");
  }
  if ((K && cudaMemcpy(g->d_hot, ids.data(), K * 4, cudaMemcpyHostToDevice) != cudaSuccess) ||
      (m && cudaMemcpy(cl.hot, hot.data(), m * 4, cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(cl.grp_off, grp_off.data(), grp_off.size() * 4, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      (cl.ngrp && cudaMemcpy(cl.grp_v, grp_v.data(), grp_v.size() * 4, cudaMemcpyHostToDevice) !=
                      cudaSuccess) ||
      cudaMemcpy(cl.blk_g, blk_g.data(), blk_g.size() * 4, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(cl.blk_mask, blk_mask.data(), blk_mask.size() * 4, cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return fail(LDD_ERR_CUDA, "upload of the cut list failed");
  return LDD_OK;
}

// The vertices the BFS handles, in ascending order, for the first bottom-up
// round of a decomposition -- built only when they are at most 3/4 of all
// vertices (else scanning every id and skipping the excluded ones is cheaper
// than reading the list).
int build_active_list(ldd_graph* g) {
  const size_t n = (size_t)g->n;
  if (n == 0 || (size_t)g->n_active * 4 > n * 3) return LDD_OK;
  std::vector<u32> excl((n + 31) / 32);
  if (cudaMemcpy(excl.data(), g->d_excl, excl.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(LDD_ERR_CUDA, "copy of the exclusion bitmask failed");
  std::vector<u32> act;
  act.reserve(g->n_active);
  for (size_t v = 0; v < n; ++v)
    if (!((excl[v >> 5] >> (v & 31)) & 1u)) act.push_back((u32)v);
  if (act.size() != g->n_active) return fail(LDD_ERR_CUDA, "inconsistent component tables");
  if (act.empty()) return LDD_OK;
  if (cudaMalloc(&g->d_active, act.size() * 4) != cudaSuccess) {
    cudaGetLastError();
    return fail(LDD_ERR_OOM, "device allocation of the active list failed");
  }
  if (cudaMemcpy(g->d_active, act.data(), act.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(LDD_ERR_CUDA, "upload of the active list failed");
  return LDD_OK;
}

void record(ldd_graph* g, int i) {
  if (g->timing) cudaEventRecord(g->ev[i], g->stream);
}

float elapsed(ldd_graph* g, int a, int b) {
  float ms = -1.f;
  if (!g->timing || cudaEventElapsedTime(&ms, g->ev[a], g->ev[b]) != cudaSuccess) {
    cudaGetLastError();
    return -1.f;
  }
  return ms;
}

BfsArgs bfs_args(ldd_graph* g) {
  BfsArgs a;
  a.row_ptr = g->d_row;
  a.col = g->d_col;
  a.key = g->d_key;
  a.bptr = g->d_bptr;
  a.rk[0] = a.rk[1] = reinterpret_cast<const u32*>(g->d_k[0]);  // start rounds, 32-bit
  a.rv[0] = a.rv[1] = g->d_v[0];                                 // start-bucket vertices
  for (int b = 0; b < 2; ++b) {
    a.qv[b] = g->d_qv[b];
    a.qrow[b] = g->d_qrow[b];
    a.qoff[b] = g->d_qoff[b];
    a.cf[b] = g->d_cf[b];
    a.ulist[b] = g->d_ulist[b];
  }
  a.excl = g->d_excl;
  a.active = g->d_active;
  a.first = g->d_first;
  a.ctl = g->d_ctl;
  a.n = (u32)g->n;
  a.n_active = g->n_active;
  a.nnz_active = g->nnz_active;
  a.spin_limit = g->spin_limit;
  a.bar_phantom = g->stall_barrier ? 1u : 0u;
  a.pull_alpha = g->pull_alpha;
  a.pull_beta = g->pull_beta;
  a.pull_gamma = g->pull_gamma;
  a.probe_min_arcs = g->probe_min_arcs;
  a.low_degree = (g->low_degree_rounds && g->max_degree <= (u32)kLdMaxDegree) ? 1u : 0u;
  a.window_levels = g->window_levels;
  a.window_max_q = g->window_max_q;
  a.window_queue = g->window_queue;
  a.span = g->bfs_span;
  a.wmem = g->uni ? g->uni->d_wmem : nullptr;
  a.mrank = g->uni ? g->uni->d_mrank : nullptr;
  a.kmem = g->uni ? g->uni->k : 0;
  return a;
}

// Small components, BFS and finalize into (center, dist) device buffers.
// Returns launches or < 0.
int run_bfs_finalize(ldd_graph* g, int* center, int* dist, int* status) {
  int launches = 0;
  cudaStream_t s = g->stream;
  launches += launch_small_comp(g->sc, g->d_key, &g->d_ctl->err, g->num_sms, s);
  if (g->n_active > 0) {
    cudaError_t e = cudaMemsetAsync((char*)g->d_ctl + kCtlMinrankOffset, 0xff, 3 * sizeof(u32), s);
    if (e == cudaSuccess && g->uni)
      e = cudaMemsetAsync(g->uni->d_mrank, 0xff, 3 * (size_t)g->uni->k * sizeof(u32), s);
    if (e != cudaSuccess) {
      *status = fail(LDD_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
      return -1;
    }
    std::unique_lock<std::mutex> gate_lk;
    if (g->gate) {  // after the round loop enqueued last through the same gate
      gate_lk = std::unique_lock<std::mutex>(g->gate->mu);
      if (g->gate->last) e = cudaStreamWaitEvent(s, g->gate->last, 0);
      if (e != cudaSuccess) {
        *status = fail(LDD_ERR_CUDA, "cudaStreamWaitEvent: %s", cudaGetErrorString(e));
        return -1;
      }
    }
    if (launch_bfs(bfs_args(g), g->bfs_grid, g->bfs_per_sm, s, &e) < 0) {
      *status = fail(LDD_ERR_CUDA, "cooperative launch of the BFS kernel (%d x %d) failed: %s",
                     g->bfs_grid, kBfsThreads, cudaGetErrorString(e));
      return -1;
    }
    if (g->gate) {
      if ((e = cudaEventRecord(g->ev_gate, s)) != cudaSuccess) {
        *status = fail(LDD_ERR_CUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
        return -1;
      }
      g->gate->last = g->ev_gate;
    }
    ++launches;
  }
  record(g, 3);
  if (g->uni)  // caller layout, member-local ids
    launches += launch_union_finalize(g->d_key, g->d_order, g->d_solo, g->uni->off, g->uni->k,
                                      g->uni->total, center, dist, &g->d_ctl->err, g->num_sms, s);
  else
    launches += launch_finalize(g->d_key, g->d_order, g->d_solo, (u32)g->n, center, dist,
                                &g->d_ctl->err, g->num_sms, s);
  return launches;
}

constexpr u32 kDefaultBarrierPolls = 1u << 22;   // grid barrier: each poll >= 20 ns after 64
constexpr u32 kDefaultLookbackPolls = 1u << 24;  // look-back: each poll >= 64 ns after 16
// Low-degree rounds of a single graph relax eight levels between grid
// barriers by default, those of a union one (ldd_autotune tries both).
// Measured: 256^3 grid 4.0 -> 3.4 ms, 256^2 0.49 -> 0.35 ms with windows;
// unions of random geometric graphs were as fast or faster level by level.
constexpr u32 kDefaultWindowLevels = 8;
constexpr u32 kDefaultUnionWindowLevels = 1;

// Scratch arena, pinned header, events and launch parameters: the part of
// graph creation that only depends on the sizes and the tables being built.
int finish_setup(ldd_graph* g) {
  int rc;
  if ((rc = alloc_scratch(g)) != LDD_OK) return rc;
  if (cudaMallocHost(&g->h_hdr, 256) != cudaSuccess)
    return fail(LDD_ERR_OOM, "pinned host allocation failed");
  for (auto& e : g->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(LDD_ERR_CUDA, "cudaEventCreate");
  int max_per_sm = 0;
  if (bfs_grid_size(g->num_sms, &max_per_sm) <= 0)
    return fail(LDD_ERR_CUDA, "BFS kernel occupancy query failed");
  // one CTA per SM for a single graph (thin frontiers, cheapest barrier), two
  // for a union (its wide bottom-up rounds of many members want the warps);
  // ldd_autotune and ldd_set_tuning choose per workload
  g->bfs_per_sm = std::min(max_per_sm, g->uni ? 2 : 1);
  const u32 per_sm = env_u32("LDD_BFS_BLOCKS_PER_SM", 0);
  if (per_sm > 0 && (int)per_sm <= max_per_sm) g->bfs_per_sm = (int)per_sm;
  g->bfs_grid = g->bfs_per_sm * g->num_sms;
  g->spin_limit = env_u32("LDD_SPIN_LIMIT", kDefaultBarrierPolls);
  g->lookback_limit = kDefaultLookbackPolls;
  g->pull_alpha = env_u32("LDD_PULL_ALPHA", 14);
  g->pull_beta = env_u32("LDD_PULL_BETA", 24);
  g->pull_gamma = env_u32("LDD_PULL_GAMMA", 8);
  g->probe_min_arcs = env_u32("LDD_PROBE_MIN_ARCS", 1u << 16);
  const char* ldr = getenv("LDD_LOW_DEGREE_ROUNDS");  // "0": edge-balanced rounds only
  g->low_degree_rounds = !(ldr && ldr[0] == '0' && ldr[1] == 0);
  g->window_levels =
      env_u32("LDD_WINDOW_LEVELS", g->uni ? kDefaultUnionWindowLevels : kDefaultWindowLevels);
  g->window_max_q = env_u32("LDD_WINDOW_MAX_FRONTIER", 1u << 18);
  g->stats.n = g->n;
  g->stats.nnz = g->nnz;
  g->stats.n_active = g->n_active;
  g->stats.small_components = g->sc.ncomp;
  g->stats.bfs_grid = g->bfs_grid;
  g->stats.bfs_block = kBfsThreads;
  return LDD_OK;
}

struct Header {  // the control block up to and including the BFS runtime state
  u32 err;
  int A;
  u32 rounds;
  int last_level;
  u64 items;
  u64 edges;
  u64 cut;
  u64 bar;
  u64 qctr[3];
  u32 minrank[3];
  u32 pull_rounds;
  u64 push_arcs;
  u64 pull_arcs;
  u64 pull_verts;
  u32 ucnt[3];
  u32 windows;
  u32 overflowed;
  u32 pad_w;
};
static_assert(sizeof(Header) == kCtlHeaderBytes + kCtlBfsStateBytes, "header layout");

RankBufs rank_bufs(ldd_graph* g, const double* d_shift) {
  RankBufs rb;
  rb.shift = d_shift;
  rb.n = (u32)g->n;
  rb.num_sms = g->num_sms;
  rb.a = g->d_a;
  rb.k0 = g->d_k[0];
  rb.k1 = g->d_k[1];
  rb.v0 = g->d_v[0];
  rb.v1 = g->d_v[1];
  rb.slots = g->d_slots;
  rb.status = g->d_status;
  rb.epoch = &g->epoch;
  rb.order = g->d_order;
  rb.key = g->d_key;
  rb.excl = g->d_excl;
  rb.solo = g->d_solo;
  rb.wmem = g->uni ? g->uni->d_wmem : nullptr;
  rb.lift = g->uni ? g->uni->d_amax + g->uni->k : nullptr;
  rb.ctl = g->d_ctl;
  rb.lookback_limit = g->lookback_limit;
  rb.stall_lookback = g->stall_lookback;
  rb.bptr = g->d_bptr;
  rb.rcur = g->d_rcur;
  rb.acnt = g->d_acnt;
  rb.acnt_dirty = g->acnt_dirty;
  rb.bptr_cap = g->bptr_cap;
  return rb;
}

void header_stats(ldd_graph* g, const Header& h, bool exact64) {
  ldd_stats& st = g->stats;
  st.max_floor_shift = h.A;
  st.exact_rank = exact64 ? 1 : 0;
  st.rounds = h.rounds;
  st.last_level = h.last_level;
  st.items = (int64_t)h.items;
  st.edges = (int64_t)h.edges;
  st.pull_rounds = h.pull_rounds;
  st.push_arcs = (int64_t)h.push_arcs;
  st.pull_arcs = (int64_t)h.pull_arcs;
  st.pull_vertices = (int64_t)h.pull_verts;
  st.bfs_windows = h.windows;
  st.bfs_overflow = h.overflowed;
}

int header_error(u32 err) {
  if (err & kErrShiftArg) return fail(LDD_ERR_ARG, "a shift is NaN or negative");
  if (err & kErrPermArg)
    return fail(LDD_ERR_ARG, "levels must be >= 0 and perm a permutation of 0 .. n-1");
  if (err & kErrShiftRange) return fail(LDD_ERR_RANGE, "a shift is >= 2^31 or infinite");
  if (err & kErrTimeout) return fail(LDD_ERR_TIMEOUT, "a device-side wait ran out");
  return fail(LDD_ERR_CUDA, "device error bits 0x%x", err);
}

void drop_replay(ldd_graph* g) {
  for (auto& x : g->gexec)
    if (x) {
      cudaGraphExecDestroy(x);
      x = nullptr;
    }
}

// One decomposition with the shifts already on the device and device
// outputs, on the graph's stream (events 1 .. 4 when timing): rank and start
// buckets, the round loop, finalize, with the retries of the fast rank path.
// Fills the device-side statistics of g->stats.
int decompose_on_device(ldd_graph* g, const double* d_shift, int* center, int* dist,
                        int* launches_out, const int* d_levels, const int* d_perm) {
  cudaStream_t s = g->stream;
  int launches = 0;
  RankBufs rb = rank_bufs(g, d_shift);
  Header h;
  int status = LDD_OK;
  bool exact64 = false;
  if (g->epoch > 0xfffff000u) {  // status tags would wrap: clear and restart
    CUDA_TRY(cudaMemsetAsync(g->d_status, 0, g->status_bytes, s));
    g->epoch = 0;
  }
  CUDA_TRY(cudaMemsetAsync(g->d_ctl, 0, sizeof(Control), s));
  record(g, 1);
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (attempt) CUDA_TRY(cudaMemsetAsync(g->d_ctl, 0, sizeof(Control), s));
    rb = rank_bufs(g, d_shift);
    rb.bptr = g->d_bptr;
    rb.rcur = g->d_rcur;
    rb.acnt = g->d_acnt;
    rb.acnt_dirty = g->acnt_dirty;
    rb.bptr_cap = g->bptr_cap;
    if (!exact64 && !d_levels) g->acnt_dirty = true;  // until this attempt has consumed the counts
    launches += d_levels ? launch_ranked_and_buckets(rb, d_levels, d_perm, s)
                         : launch_rank_and_buckets(rb, exact64, s);
    record(g, 2);
    const int l = run_bfs_finalize(g, center, dist, &status);
    if (l < 0) return status;
    launches += l;
    record(g, 4);
    CUDA_TRY(cudaMemcpyAsync(g->h_hdr, g->d_ctl, sizeof(Header), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(s));
    memcpy(&h, g->h_hdr, sizeof(h));
    if (!exact64 && !d_levels && h.err == 0) g->acnt_dirty = false;  // the scan cleared them
    const u32 retry = kErrRankRetry | kErrBucketCap;
    if (h.err == 0 || (h.err & ~retry) != 0) break;
    // A fraction bucket too full to rank in place (crafted shifts): every
    // kernel after the split was skipped; redo with the exact path.
    if (h.err & kErrRankRetry) exact64 = true;
    if (h.err & kErrBucketCap) {
      // floor(delta_max) + 2 exceeds the start-bucket table: grow it, redo.
      const size_t need = (size_t)h.A + 2;
      cudaFree(g->d_bptr);
      cudaFree(g->d_rcur);
      cudaFree(g->d_acnt);
      g->d_bptr = nullptr;
      g->d_rcur = nullptr;
      g->d_acnt = nullptr;
      g->bptr_cap = 0;
      if (cudaMalloc(&g->d_bptr, need * sizeof(int)) != cudaSuccess ||
          cudaMalloc(&g->d_rcur, need * sizeof(u32)) != cudaSuccess ||
          cudaMalloc(&g->d_acnt, need * sizeof(u32)) != cudaSuccess) {
        cudaGetLastError();
        return fail(LDD_ERR_OOM, "start-bucket table of %zu entries", need);
      }
      g->bptr_cap = (u32)need;
      g->acnt_dirty = true;  // cleared by the next fast-path attempt
      drop_replay(g);        // a captured replay holds the old table
    }
  }
  if (h.err) return header_error(h.err);
  header_stats(g, h, exact64);
  ldd_stats& st = g->stats;
  st.ms_rank = elapsed(g, 1, 2);
  st.ms_bfs = elapsed(g, 2, 3);
  st.ms_finalize = elapsed(g, 3, 4);
  st.replayed = 0;
  ++g->regular_runs;
  *launches_out = launches;
  return LDD_OK;
}

// The library-owned outputs a replay writes: caller layout for a union.
int* replay_center(ldd_graph* g) { return g->uni ? g->uni->d_out_c : g->d_center; }
int* replay_dist(ldd_graph* g) { return g->uni ? g->uni->d_out_d : g->d_dist; }

// Queues one fast-path decomposition on g->stream with no host synchronisation,
// as it is captured: control block and look-back status cleared, [a union's
// shifts spread from the caller layout,] rank with the fixed epochs 1 and 2,
// BFS, finalize into the library's outputs, [the union's cut counts,] and the
// header copied to the pinned host block.  Returns kernels queued, or -1.
int enqueue_fast(ldd_graph* g, bool want_cut) {
  cudaStream_t s = g->stream;
  int launches = 0;
  if (cudaMemsetAsync(g->d_ctl, 0, sizeof(Control), s) != cudaSuccess) return -1;
  const size_t words = rank_status_words((u32)g->n, g->bptr_cap);
  if (cudaMemsetAsync(g->d_status, 0, words * sizeof(u64), s) != cudaSuccess) return -1;
  if (g->uni) {
    ldd_graph::Union& U = *g->uni;
    launches += launch_union_spread(U.d_shift_in, U.off, U.k, (u32)g->n, g->d_excl, g->d_shift,
                                    U.d_amax, U.d_amax + U.k, g->num_sms, s);
  }
  u32 epoch = 0;  // the two scans run with epochs 1 and 2 on cleared status words
  RankBufs rb = rank_bufs(g, g->d_shift);
  rb.epoch = &epoch;
  rb.acnt_dirty = false;  // cleared before every launch of the replay
  launches += launch_rank_and_buckets(rb, false, s);
  int status = LDD_OK;
  const int l = run_bfs_finalize(g, replay_center(g), replay_dist(g), &status);
  if (l < 0) return -1;
  launches += l;
  if (g->uni && want_cut) {
    ldd_graph::Union& U = *g->uni;
    if (cudaMemsetAsync(U.d_cut, 0, (size_t)U.k * 8, s) != cudaSuccess) return -1;
    launches += launch_union_cut(g->cut, U.off, U.d_wmem, U.d_out_c, U.d_cut, g->num_sms, s);
    if (cudaMemcpyAsync(g->h_cut, U.d_cut, (size_t)U.k * 8, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
      return -1;
  }
  if (cudaMemcpyAsync(g->h_hdr, g->d_ctl, sizeof(Header), cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return -1;
  return cudaGetLastError() == cudaSuccess ? launches : -1;
}

// Captures enqueue_fast into an executable graph (slot: with union cut
// counts).  A capture that fails marks the graph replay_broken; the regular
// path then runs.
void capture_fast(ldd_graph* g, bool want_cut) {
  const int slot = want_cut ? 1 : 0;
  if (!g->cap_stream &&
      cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    g->replay_broken = true;
    return;
  }
  if (g->uni && want_cut && !g->h_cut &&
      cudaMallocHost(&g->h_cut, std::max<size_t>(g->uni->k, 1) * 8) != cudaSuccess) {
    cudaGetLastError();
    g->replay_broken = true;
    return;
  }
  cudaStream_t saved = g->stream;
  const bool saved_timing = g->timing;
  g->stream = g->cap_stream;
  g->timing = false;
  cudaGraph_t graph = nullptr;
  int launches = -1;
  if (cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    launches = enqueue_fast(g, want_cut);
    if (cudaStreamEndCapture(g->cap_stream, &graph) != cudaSuccess) launches = -1;
  }
  g->stream = saved;
  g->timing = saved_timing;
  cudaGraphExec_t exec = nullptr;
  if (launches < 0 || !graph || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    g->replay_broken = true;
    exec = nullptr;
  }
  if (graph) cudaGraphDestroy(graph);
  g->gexec[slot] = exec;
  g->replay_launches[slot] = launches;
}

constexpr int kRunRegular = 1;  // replay_fast: take the regular path instead

// One decomposition by graph replay, the shifts already in the library's
// input buffer (d_shift, or a union's caller-layout d_shift_in).  Returns
// LDD_OK, an error, or kRunRegular (no capture yet, capture failed, or the
// fast rank path asked for a retry).
int replay_fast(ldd_graph* g, bool want_cut, int* launches_out) {
  if (!g->replay || g->replay_broken || g->regular_runs == 0) return kRunRegular;
  const int slot = want_cut ? 1 : 0;
  cudaStream_t s = g->stream;
  if (g->acnt_dirty) {
    CUDA_TRY(cudaMemsetAsync(g->d_acnt, 0, (size_t)g->bptr_cap * 4, s));
    g->acnt_dirty = false;
  }
  if (!g->gexec[slot]) capture_fast(g, want_cut);
  if (!g->gexec[slot]) return kRunRegular;
  record(g, 1);
  CUDA_TRY(cudaGraphLaunch(g->gexec[slot], s));
  record(g, 4);
  CUDA_TRY(cudaStreamSynchronize(s));
  Header h;
  memcpy(&h, g->h_hdr, sizeof(h));
  if (h.err & (kErrRankRetry | kErrBucketCap)) {
    g->acnt_dirty = true;  // the counts may be half consumed
    return kRunRegular;
  }
  if (h.err) return header_error(h.err);
  header_stats(g, h, false);
  ldd_stats& st = g->stats;
  st.ms_rank = st.ms_bfs = st.ms_finalize = -1.f;
  st.ms_replay = elapsed(g, 1, 4);
  st.replayed = 1;
  *launches_out = g->replay_launches[slot];
  return LDD_OK;
}

// Cut count of a device labelling on the graph's stream (events 6, 7).
int cut_on_device(ldd_graph* g, const int* d_center, int64_t* out_cut) {
  cudaStream_t s = g->stream;
  record(g, 6);
  CUDA_TRY(cudaMemsetAsync(&g->d_ctl->cut, 0, sizeof(u64), s));
  const int l = launch_cut(g->cut, d_center, g->d_hot, g->n_hot, g->d_hot_center,
                           &g->d_ctl->cut, g->num_sms, s);
  CUDA_TRY(cudaMemcpyAsync(g->h_hdr + 128, &g->d_ctl->cut, sizeof(u64), cudaMemcpyDeviceToHost, s));
  record(g, 7);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
  u64 cut;
  memcpy(&cut, g->h_hdr + 128, sizeof(cut));
  *out_cut = (int64_t)cut;
  g->stats.cut_launches = l;
  g->stats.ms_cut = elapsed(g, 6, 7);
  return LDD_OK;
}

// One fast-path decomposition of a plain graph queued on g->stream with no
// host synchronisation, in two parts.  enqueue_rank: control block cleared,
// rank and start buckets.  enqueue_bfs_finalize: BFS and finalize into
// center/dist; the shifts are no longer needed and the labels are final once
// it has run.  A fast rank path that asks for the exact path leaves the floor
// counts cleared and skips the rest, so the decompositions queued behind it
// run as usual.
int enqueue_rank(ldd_graph* g, const double* d_shift, int* launches,
                 const ShiftChunks* chunks = nullptr) {
  cudaStream_t s = g->stream;
  if (g->epoch > 0xfffff000u) {  // status tags would wrap: clear and restart
    CUDA_TRY(cudaMemsetAsync(g->d_status, 0, g->status_bytes, s));
    g->epoch = 0;
  }
  CUDA_TRY(cudaMemsetAsync(g->d_ctl, 0, sizeof(Control), s));
  if (g->acnt_dirty) {
    CUDA_TRY(cudaMemsetAsync(g->d_acnt, 0, (size_t)g->bptr_cap * 4, s));
    g->acnt_dirty = false;
  }
  RankBufs rb = rank_bufs(g, d_shift);
  rb.acnt_dirty = false;
  *launches += launch_rank_and_buckets(rb, false, s, chunks);
  return LDD_OK;
}

int enqueue_bfs_finalize(ldd_graph* g, int* center, int* dist, int* launches) {
  int status = LDD_OK;
  const int lb = run_bfs_finalize(g, center, dist, &status);
  if (lb < 0) {
    g->acnt_dirty = true;
    return status;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g->acnt_dirty = true;
    return fail(LDD_ERR_CUDA, "%s", cudaGetErrorString(e));
  }
  *launches += lb;
  return LDD_OK;
}

// Packed-label buffers of the fused cut counts of a batch, allocated on first use.
int ensure_cut4(ldd_graph* g) {
  if (g->d_lab4) return LDD_OK;
  const size_t n = std::max<size_t>((size_t)g->n, 1), nh = std::max<size_t>(g->n_hot, 1),
               ng = std::max<size_t>(g->cut.ngrp, 1);
  if (cudaMalloc(&g->d_lab4, n * sizeof(int4)) != cudaSuccess ||
      cudaMalloc(&g->d_hot4, nh * sizeof(int4)) != cudaSuccess ||
      cudaMalloc(&g->d_grp4, ng * sizeof(int4)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(g->d_lab4);
    cudaFree(g->d_hot4);
    cudaFree(g->d_grp4);
    g->d_lab4 = g->d_hot4 = g->d_grp4 = nullptr;
    return fail(LDD_ERR_OOM, "packed labels for the fused cut counts: allocation failed");
  }
  return LDD_OK;
}

// Pinned headers and the device / pinned cut counts of a batch of k.
int ensure_batch_headers(ldd_graph* g, int k) {
  if (g->h_bhdr_cap >= k) return LDD_OK;
  if (g->h_bhdr) cudaFreeHost(g->h_bhdr);
  if (g->h_bcut) cudaFreeHost(g->h_bcut);
  cudaFree(g->d_bcut);
  g->h_bhdr = nullptr;
  g->h_bcut = nullptr;
  g->d_bcut = nullptr;
  g->h_bhdr_cap = 0;
  if (cudaMallocHost(&g->h_bhdr, (size_t)k * sizeof(Header)) != cudaSuccess ||
      cudaMallocHost(&g->h_bcut, (size_t)k * sizeof(u64)) != cudaSuccess ||
      cudaMalloc(&g->d_bcut, (size_t)k * sizeof(u64)) != cudaSuccess) {
    cudaGetLastError();
    return fail(LDD_ERR_OOM, "batch state for %d decompositions: allocation failed", k);
  }
  g->h_bhdr_cap = k;
  return LDD_OK;
}

// Streams and staging of ldd_decompose_batch, created on first use.
int setup_batch(ldd_graph* g) {
  if (g->batch_arena) return LDD_OK;
  const size_t n = (size_t)g->n;
  if (cudaStreamCreateWithFlags(&g->copy_in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&g->copy_out, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&g->cut_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return fail(LDD_ERR_CUDA, "cudaStreamCreate for the batch pipeline failed");
  }
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreateWithFlags(&g->ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_used[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_out[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->ev_cut[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(LDD_ERR_CUDA, "cudaEventCreate for the batch pipeline failed");
    }
  for (auto& e : g->ev_chunk)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(LDD_ERR_CUDA, "cudaEventCreate for the batch pipeline failed");
    }
  if (cudaMalloc(&g->batch_arena, 4 * align_up(8 * n, 256)) != cudaSuccess) {
    cudaGetLastError();
    g->batch_arena = nullptr;
    return fail(LDD_ERR_OOM, "cudaMalloc of the batch staging (%zu bytes) failed",
                4 * align_up(8 * n, 256));
  }
  return LDD_OK;
}

// ---------------------------------------------------------------- unions
UnionCaps union_needs(int k, ldd_graph* const* members) {
  UnionCaps c;
  c.k = (u32)k;
  for (int i = 0; i < k; ++i) {
    const ldd_graph* m = members[i];
    c.N += ((u64)m->n + 31) / 32 * 32;
    c.E += (u64)m->nnz;
    c.M += m->m_up;
    c.G += m->cut.ngrp;
    c.C += m->sc.ncomp;
    c.T += m->sc.total;
    c.total += (u64)m->n;
  }
  return c;
}

u64 union_bytes(const UnionCaps& c) {
  // tables: row, col, cut list, masks, small components, active list, word
  // members; staging: shifts in, outputs, offsets; scratch arena; start
  // buckets (three tables of N + 2)
  const u64 N = c.N, words = std::max<u64>(N / 32, 1);
  u64 b = 4 * (N + 1) + 4 * c.E + 4 * c.M + 20 * c.G + 8 * (c.M / 32 + 1) + 8 * words +
          8 * c.C + 8 * c.T + 4 * N + 4 * words;
  b += 16 * c.total + 8 * c.total + 32ull * (c.k + 1) + 8ull * c.k + sizeof(UnionMember) * c.k;
  const u64 nk = std::max<u64>(N, 64);
  b += 8 * N + 4 * N + 16 * nk + 8 * N + ((N + kSortTile - 1) / kSortTile + 1) * 2048 + 4 * N +
       8 * N + 24 * N + 8 * (c.E / kBfsBase + 2) + 8 * N + (N ? fraction_slot_bytes((u32)N) : 0) +
       8 * N + sizeof(Control);
  b += 12 * (N + 2);
  return b;
}

int union_alloc(ldd_graph** out, int dev, const UnionCaps& c) {
  *out = nullptr;
  ldd_graph* g = new (std::nothrow) ldd_graph();
  if (!g) return fail(LDD_ERR_OOM, "host allocation failed");
  auto bail = [&](int status) {
    free_graph_memory(g);
    delete g;
    return status;
  };
  g->uni = new (std::nothrow) ldd_graph::Union();
  if (!g->uni) return bail(fail(LDD_ERR_OOM, "host allocation failed"));
  ldd_graph::Union& U = *g->uni;
  U.cap = c;
  memset(&g->stats, 0, sizeof(g->stats));
  g->device = dev;
  if (cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(LDD_ERR_CUDA, "no usable CUDA device"));
  }
  const u64 N = c.N, words = std::max<u64>(N / 32, 1), K = std::max<u32>(c.k, 1);
  const u64 total = std::max<u64>(c.total, 1);
  if (cudaMalloc(&g->d_row, (N + 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->d_col, std::max<u64>(c.E, 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->cut.hot, std::max<u64>(c.M, 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->cut.grp_off, (c.G + 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->cut.grp_v, std::max<u64>(c.G, 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->cut.grp_m, std::max<u64>(c.G, 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->cut.grp_lab, std::max<u64>(c.G, 1) * 8) != cudaSuccess ||
      cudaMalloc(&g->cut.blk_g, (c.M / 32 + 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->cut.blk_mask, (c.M / 32 + 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->d_excl, 2 * words * 4) != cudaSuccess ||
      cudaMalloc(&g->sc.comp_off, std::max<u64>(c.C, 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->sc.comp_len, std::max<u64>(c.C, 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->sc.comp_v, std::max<u64>(c.T, 1) * 4) != cudaSuccess ||
      cudaMalloc(&g->sc.adj, std::max<u64>(c.T, 1) * 4) != cudaSuccess ||
      cudaMalloc(&U.d_active_buf, std::max<u64>(N, 1) * 4) != cudaSuccess ||
      cudaMalloc(&U.d_mem, K * sizeof(UnionMember)) != cudaSuccess ||
      cudaMalloc(&U.d_offs, 8 * (K + 1) * 4) != cudaSuccess ||
      cudaMalloc(&U.d_shift_in, total * 8) != cudaSuccess ||
      cudaMalloc(&U.d_out_c, total * 8) != cudaSuccess ||
      cudaMalloc(&U.d_cut, K * 8) != cudaSuccess ||
      cudaMalloc(&U.d_wmem, words * 4) != cudaSuccess ||
      cudaMalloc(&U.d_amax, 2 * K * 4) != cudaSuccess ||
      cudaMalloc(&U.d_mrank, 3 * K * 4) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(LDD_ERR_OOM, "device allocation of a union (%llu vertices, %llu arcs) "
                     "failed", (unsigned long long)N, (unsigned long long)c.E));
  }
  g->d_solo = g->d_excl + words;
  U.d_out_d = U.d_out_c + total;
  const u32* d = U.d_offs;
  const size_t K1 = K + 1;
  U.off = UnionOffsets{d,          d + K1,     d + 2 * K1, d + 3 * K1,
                       d + 4 * K1, d + 5 * K1, d + 6 * K1, d + 7 * K1};
  // the scratch arena and launch set-up are sized by the capacities
  g->n = (int32_t)N;
  g->nnz = (int64_t)c.E;
  int rc = finish_setup(g);
  if (rc != LDD_OK) return bail(rc);
  *out = g;
  return LDD_OK;
}

int union_fill(ldd_graph* g, int k, ldd_graph* const* members, cudaStream_t s, bool sync) {
  ldd_graph::Union& U = *g->uni;
  const UnionCaps need = union_needs(k, members);
  if ((u32)k > U.cap.k || need.N > U.cap.N || need.E > U.cap.E || need.M > U.cap.M ||
      need.G > U.cap.G || need.C > U.cap.C || need.T > U.cap.T || need.total > U.cap.total)
    return fail(LDD_ERR_RANGE, "members exceed the union's capacity");
  const size_t K1 = (size_t)U.cap.k + 1;
  std::vector<u32> offs(8 * K1, 0);
  bool all_active = true;
  u64 nnz_active = 0, n_active = 0;
  u32 max_deg = 0;
  auto at = [&](int t, int i) -> u32& { return offs[(size_t)t * K1 + (size_t)i]; };
  for (int i = 0; i < k; ++i) {
    const ldd_graph* m = members[i];
    at(0, i + 1) = at(0, i) + (u32)(((u64)m->n + 31) / 32 * 32);
    at(1, i + 1) = at(1, i) + (u32)m->nnz;
    at(2, i + 1) = at(2, i) + m->m_up;
    at(3, i + 1) = at(3, i) + m->sc.ncomp;
    at(4, i + 1) = at(4, i) + m->sc.total;
    at(5, i + 1) = at(5, i) + m->n_active;
    at(6, i + 1) = at(6, i) + (u32)m->n;
    at(7, i + 1) = at(7, i) + m->cut.ngrp;
    if (m->n_active > 0 && !m->d_active) all_active = false;
    max_deg = std::max(max_deg, m->max_degree);
    nnz_active += m->nnz_active;
    n_active += m->n_active;
  }
  g->n = (int32_t)need.N;
  g->nnz = (int64_t)need.E;
  g->m_up = (u32)need.M;
  g->sc.ncomp = (u32)need.C;
  g->sc.total = (u32)need.T;
  g->n_active = (u32)n_active;
  g->nnz_active = nnz_active;
  g->max_degree = max_deg;
  g->d_active = (all_active && n_active > 0) ? U.d_active_buf : nullptr;
  U.k = (u32)k;
  U.total = (u32)need.total;
  g->cut.m = (u32)need.M;
  g->cut.ngrp = (u32)need.G;
  g->cut.nblk = (u32)((need.M + 31) / 32);
  U.h_voff.assign(offs.begin(), offs.begin() + k + 1);
  U.h_ooff.assign(offs.begin() + 6 * K1, offs.begin() + 6 * K1 + k + 1);
  std::vector<UnionMember> mv((size_t)k);
  for (int i = 0; i < k; ++i) {
    const ldd_graph* m = members[i];
    UnionMember& d = mv[(size_t)i];
    d.row = m->d_row;
    d.col = m->d_col;
    d.cut_hot = m->cut.hot;
    d.grp_off = m->cut.grp_off;
    d.grp_v = m->cut.grp_v;
    d.hot = m->d_hot;
    d.excl = m->d_excl;
    d.solo = m->d_solo;
    d.comp_off = m->sc.comp_off;
    d.comp_len = m->sc.comp_len;
    d.comp_v = m->sc.comp_v;
    d.adj = m->sc.adj;
    d.active = m->d_active;
    d.n = (u32)m->n;
    d.nnz = (u32)m->nnz;
  }
  drop_replay(g);  // captured graphs hold the old sizes
  CUDA_TRY(cudaMemcpyAsync(U.d_mem, mv.data(), mv.size() * sizeof(UnionMember),
                           cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(U.d_offs, offs.data(), offs.size() * 4, cudaMemcpyHostToDevice, s));
  UnionTables t{g->d_row, g->d_col, g->cut, g->d_excl, g->d_solo, g->sc.comp_off,
                g->sc.comp_len, g->sc.comp_v, g->sc.adj, g->d_active, U.d_wmem};
  const u64 largest = std::max<u64>(std::max<u64>(need.N + 1, need.E), need.M);
  launch_union_concat(U.d_mem, U.off, U.k, t, largest, g->num_sms, s);
  CUDA_TRY(cudaGetLastError());
  if (sync) CUDA_TRY(cudaStreamSynchronize(s));
  g->stats.n = g->n;
  g->stats.nnz = g->nnz;
  g->stats.n_active = g->n_active;
  g->stats.small_components = g->sc.ncomp;
  return LDD_OK;
}

int union_run(ldd_graph* u, const double* d_in, int* center, int* dist, bool want_cut,
              int* launches_out, int* cut_launches_out) {
  ldd_graph::Union& U = *u->uni;
  cudaStream_t s = u->stream;
  int launches = launch_union_spread(d_in, U.off, U.k, (u32)u->n, u->d_excl, u->d_shift, U.d_amax,
                                     U.d_amax + U.k, u->num_sms, s);
  int l = 0, rc;
  if ((rc = decompose_on_device(u, u->d_shift, center, dist, &l)) != LDD_OK) return rc;
  launches += l;
  int cl = 0;
  if (want_cut) {
    record(u, 6);
    CUDA_TRY(cudaMemsetAsync(U.d_cut, 0, (size_t)U.k * 8, s));
    cl = launch_union_cut(u->cut, U.off, U.d_wmem, center, U.d_cut, u->num_sms, s);
    record(u, 7);
  }
  *launches_out = launches;
  *cut_launches_out = cl;
  return LDD_OK;
}

}  // namespace ldd

extern "C" {

const char* ldd_status_string(int status) {
  switch (status) {
    case LDD_OK: return "LDD_OK";
    case LDD_ERR_ARG: return "LDD_ERR_ARG: invalid argument";
    case LDD_ERR_GRAPH: return "LDD_ERR_GRAPH: CSR failed validation";
    case LDD_ERR_RANGE: return "LDD_ERR_RANGE: size or value out of the supported range";
    case LDD_ERR_OOM: return "LDD_ERR_OOM: allocation failed";
    case LDD_ERR_CUDA: return "LDD_ERR_CUDA: CUDA runtime error";
    case LDD_ERR_TIMEOUT: return "LDD_ERR_TIMEOUT: a bounded device wait ran out";
    default: return "unknown ldd status";
  }
}

const char* ldd_last_error(void) { return g_last_error; }

int ldd_create_graph(int32_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx,
                     int validate, ldd_graph** out) {
  g_last_error[0] = 0;
  const auto t_start = std::chrono::steady_clock::now();
  if (!out) return fail(LDD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 0 || nnz < 0) return fail(LDD_ERR_ARG, "negative size (n = %d, nnz = %lld)", n,
                                    (long long)nnz);
  if (n >= (1 << 30)) return fail(LDD_ERR_RANGE, "n = %d must be < 2^30", n);
  if (nnz >= (int64_t)1 << 31) return fail(LDD_ERR_RANGE, "nnz = %lld must be < 2^31",
                                           (long long)nnz);
  if (!row_ptr) return fail(LDD_ERR_ARG, "row_ptr is NULL");
  if (nnz > 0 && !col_idx) return fail(LDD_ERR_ARG, "col_idx is NULL");

  ldd_graph* g = new (std::nothrow) ldd_graph();
  if (!g) return fail(LDD_ERR_OOM, "host allocation failed");
  memset(&g->stats, 0, sizeof(g->stats));
  g->n = n;
  g->nnz = nnz;
  int rc = LDD_OK;
  auto bail = [&](int status) {
    free_graph_memory(g);
    delete g;
    return status;
  };
  if (cudaGetDevice(&g->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device) !=
          cudaSuccess) {
    cudaGetLastError();
    return bail(fail(LDD_ERR_CUDA, "no usable CUDA device"));
  }
  // Host copies of the CSR (the caller's buffers may live on either side).
  std::vector<int32_t> rp((size_t)n + 1), col((size_t)nnz);
  if (is_device_ptr(row_ptr)) {
    if (cudaMemcpy(rp.data(), row_ptr, rp.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return bail(fail(LDD_ERR_CUDA, "copy of row_ptr failed"));
  } else {
    memcpy(rp.data(), row_ptr, rp.size() * 4);
  }
  if (nnz > 0) {
    if (is_device_ptr(col_idx)) {
      if (cudaMemcpy(col.data(), col_idx, col.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return bail(fail(LDD_ERR_CUDA, "copy of col_idx failed"));
    } else {
      memcpy(col.data(), col_idx, col.size() * 4);
    }
  }
  if (validate && (rc = validate_csr(n, nnz, rp.data(), col.data())) != LDD_OK) return bail(rc);
  if (rp[0] != 0 || (int64_t)rp[n] != nnz)
    return bail(fail(LDD_ERR_GRAPH, "row_ptr[0] must be 0 and row_ptr[n] must be nnz"));

  for (int32_t v = 0; v < n; ++v)
    g->max_degree = std::max<u32>(g->max_degree, (u32)(rp[v + 1] - rp[v]));
  // The arcs (v, w) with v < w: one entry per undirected edge (cut count,
  // component labelling).
  std::vector<int2> up;
  up.reserve((size_t)nnz / 2 + 1);
  for (int32_t v = 0; v < n; ++v)
    for (int64_t e = rp[v]; e < rp[v + 1]; ++e)
      if (col[e] > v) up.push_back(make_int2(v, col[e]));
  g->m_up = (u32)up.size();
  cudaEvent_t ce[3] = {nullptr, nullptr, nullptr};  // upload, component labelling
  for (auto& e : ce)
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      e = nullptr;
    }
  auto mark = [&](int i) {
    if (ce[i]) cudaEventRecord(ce[i], nullptr);
  };
  auto span = [&](int a, int b) {
    float ms = -1.f;
    if (!ce[a] || !ce[b] || cudaEventSynchronize(ce[b]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, ce[a], ce[b]) != cudaSuccess) {
      cudaGetLastError();
      ms = -1.f;
    }
    return ms;
  };
  struct EventsFree {
    cudaEvent_t* e;
    ~EventsFree() {
      for (int i = 0; i < 3; ++i)
        if (e[i]) cudaEventDestroy(e[i]);
    }
  } events_free{ce};
  if (cudaMalloc(&g->d_row, rp.size() * 4) != cudaSuccess ||
      cudaMalloc(&g->d_col, std::max<size_t>(col.size(), 1) * 4) != cudaSuccess) {
    cudaGetLastError();
    return bail(fail(LDD_ERR_OOM, "device allocation of the graph failed"));
  }
  mark(0);
  if (cudaMemcpy(g->d_row, rp.data(), rp.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      (nnz > 0 &&
       cudaMemcpy(g->d_col, col.data(), col.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess))
    return bail(fail(LDD_ERR_CUDA, "upload of the graph failed"));
  mark(1);
  rc = build_component_tables(g);
  mark(2);
  if (rc != LDD_OK) return bail(rc);
  const float ms_upload = span(0, 1), ms_components = span(1, 2);
  if ((rc = build_cut_list(g, rp, up)) != LDD_OK) return bail(rc);
  if ((rc = build_active_list(g)) != LDD_OK) return bail(rc);
  if (nnz > 0) {  // first neighbours: a bottom-up scan's first probe without a col round trip
    if (cudaMalloc(&g->d_first, (size_t)n * 4) != cudaSuccess) {
      cudaGetLastError();
      return bail(fail(LDD_ERR_OOM, "device allocation of the first-neighbour table failed"));
    }
    launch_first_neighbours(g->d_row, g->d_col, (u32)n, g->d_first, g->num_sms, nullptr);
    if (cudaStreamSynchronize(nullptr) != cudaSuccess)
      return bail(fail(LDD_ERR_CUDA, "first-neighbour table"));
  }
  if ((rc = finish_setup(g)) != LDD_OK) return bail(rc);
  // low-degree rounds are latency-bound: a key probe before every atomicMin
  // is one more dependent round trip, worth it only in wide rounds
  if (g->max_degree <= (u32)kLdMaxDegree && !getenv("LDD_PROBE_MIN_ARCS"))
    g->probe_min_arcs = 1u << 20;
  g->stats.ms_create_upload = ms_upload;
  g->stats.ms_create_components = ms_components;
  g->stats.ms_create_total =
      std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  *out = g;
  return LDD_OK;
}

void ldd_destroy_graph(ldd_graph* g) {
  if (!g) return;
  DeviceGuard dg(g->device);
  cudaStreamSynchronize(g->stream);
  free_graph_memory(g);
  delete g;
}

int ldd_set_stream(ldd_graph* g, void* cuda_stream) {
  if (!g) return fail(LDD_ERR_ARG, "graph is NULL");
  g->stream = (cudaStream_t)cuda_stream;
  return LDD_OK;
}

int ldd_get_round_profile(const ldd_graph* g, int64_t* clocks, int32_t* kinds, int cap,
                          int* out_count) {
  if (!g || !clocks || !kinds || !out_count || cap < 0) return fail(LDD_ERR_ARG, "NULL argument");
  DeviceGuard dg(g->device);
  const int count = (int)std::min<int64_t>(std::min<int64_t>(g->stats.rounds + 1, kRoundProfile),
                                           cap);
  *out_count = count;
  if (count <= 0) return LDD_OK;
  CUDA_TRY(cudaMemcpyAsync(clocks, g->d_ctl->round_clk, (size_t)count * 3 * 8,
                           cudaMemcpyDeviceToHost, g->stream));
  CUDA_TRY(cudaMemcpyAsync(kinds, g->d_ctl->round_kind, (size_t)count * 4, cudaMemcpyDeviceToHost,
                           g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return LDD_OK;
}

int ldd_set_timing(ldd_graph* g, int enable) {
  if (!g) return fail(LDD_ERR_ARG, "graph is NULL");
  g->timing = enable != 0;
  return LDD_OK;
}

int ldd_get_stats(const ldd_graph* g, ldd_stats* out) {
  if (!g || !out) return fail(LDD_ERR_ARG, "NULL argument");
  *out = g->stats;
  return LDD_OK;
}

int ldd_decompose(ldd_graph* g, double beta, const double* shifts, int32_t* out_center,
                  int32_t* out_dist) {
  g_last_error[0] = 0;
  if (!g) return fail(LDD_ERR_ARG, "graph is NULL");
  if (g->uni) return fail(LDD_ERR_ARG, "a union graph is decomposed by ldd_union_decompose");
  if (!(beta > 0.0) || isinf(beta)) return fail(LDD_ERR_ARG, "beta must be finite and > 0");
  if (g->n == 0) return LDD_OK;
  if (!shifts || !out_center || !out_dist) return fail(LDD_ERR_ARG, "NULL shifts or output");
  DeviceGuard dg(g->device);
  if (!dg.ok) return fail(LDD_ERR_CUDA, "cannot select device %d", g->device);
  cudaStream_t s = g->stream;
  const size_t n = (size_t)g->n;
  const bool dev_in = is_device_ptr(shifts);
  const bool dev_c = is_device_ptr(out_center), dev_d = is_device_ptr(out_dist);
  int* center = dev_c ? out_center : g->d_center;
  int* dist = dev_d ? out_dist : g->d_dist;
  record(g, 0);
  const double* d_shift = shifts;
  int launches = 0;
  int rc = kRunRegular;
  if (g->replay && !g->replay_broken && g->regular_runs > 0) {
    // replay: inputs and outputs go through the library's own buffers
    CUDA_TRY(cudaMemcpyAsync(g->d_shift, shifts, n * 8,
                             dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    d_shift = g->d_shift;
    rc = replay_fast(g, false, &launches);
    if (rc != LDD_OK && rc != kRunRegular) return rc;
    if (rc == LDD_OK) {
      center = g->d_center;
      dist = g->d_dist;
      if (dev_c)
        CUDA_TRY(cudaMemcpyAsync(out_center, center, n * 4, cudaMemcpyDeviceToDevice, s));
      if (dev_d) CUDA_TRY(cudaMemcpyAsync(out_dist, dist, n * 4, cudaMemcpyDeviceToDevice, s));
    }
  } else if (!dev_in) {
    CUDA_TRY(cudaMemcpyAsync(g->d_shift, shifts, n * 8, cudaMemcpyHostToDevice, s));
    d_shift = g->d_shift;
  }
  if (rc == kRunRegular && (rc = decompose_on_device(g, d_shift, center, dist, &launches)) != LDD_OK)
    return rc;
  if (!dev_c) CUDA_TRY(cudaMemcpyAsync(out_center, center, n * 4, cudaMemcpyDeviceToHost, s));
  if (!dev_d) CUDA_TRY(cudaMemcpyAsync(out_dist, dist, n * 4, cudaMemcpyDeviceToHost, s));
  record(g, 5);
  CUDA_TRY(cudaStreamSynchronize(s));
  ldd_stats& st = g->stats;
  st.launches = launches;
  st.ms_h2d = dev_in ? 0.f : elapsed(g, 0, 1);
  st.ms_d2h = (dev_c && dev_d) ? 0.f : elapsed(g, 4, 5);
  st.ms_total = elapsed(g, 0, 5);
  return LDD_OK;
}

int ldd_decompose_ranked(ldd_graph* g, const int32_t* levels, const int32_t* perm,
                         int32_t* out_center, int32_t* out_dist) {
  g_last_error[0] = 0;
  if (!g) return fail(LDD_ERR_ARG, "graph is NULL");
  if (g->uni) return fail(LDD_ERR_ARG, "a union graph is decomposed by ldd_union_decompose");
  if (g->n == 0) return LDD_OK;
  if (!levels || !perm || !out_center || !out_dist)
    return fail(LDD_ERR_ARG, "NULL levels, perm or output");
  DeviceGuard dg(g->device);
  if (!dg.ok) return fail(LDD_ERR_CUDA, "cannot select device %d", g->device);
  cudaStream_t s = g->stream;
  const size_t n = (size_t)g->n;
  const bool dev_c = is_device_ptr(out_center), dev_d = is_device_ptr(out_dist);
  int* center = dev_c ? out_center : g->d_center;
  int* dist = dev_d ? out_dist : g->d_dist;
  record(g, 0);
  // host inputs go to scratch the ranked path leaves alone (v1, k1)
  const int* d_levels = levels;
  const int* d_perm = perm;
  if (!is_device_ptr(levels)) {
    CUDA_TRY(cudaMemcpyAsync(g->d_v[1], levels, n * 4, cudaMemcpyHostToDevice, s));
    d_levels = reinterpret_cast<const int*>(g->d_v[1]);
  }
  if (!is_device_ptr(perm)) {
    CUDA_TRY(cudaMemcpyAsync(g->d_k[1], perm, n * 4, cudaMemcpyHostToDevice, s));
    d_perm = reinterpret_cast<const int*>(g->d_k[1]);
  }
  int launches = 0;
  const int rc = decompose_on_device(g, nullptr, center, dist, &launches, d_levels, d_perm);
  if (rc != LDD_OK) return rc;
  if (!dev_c) CUDA_TRY(cudaMemcpyAsync(out_center, center, n * 4, cudaMemcpyDeviceToHost, s));
  if (!dev_d) CUDA_TRY(cudaMemcpyAsync(out_dist, dist, n * 4, cudaMemcpyDeviceToHost, s));
  record(g, 5);
  CUDA_TRY(cudaStreamSynchronize(s));
  ldd_stats& st = g->stats;
  st.launches = launches;
  st.ms_h2d = elapsed(g, 0, 1);
  st.ms_d2h = (dev_c && dev_d) ? 0.f : elapsed(g, 4, 5);
  st.ms_total = elapsed(g, 0, 5);
  return LDD_OK;
}

int ldd_decompose_retry(ldd_graph* g, double beta, int k, const double* const* shifts,
                        int64_t max_cut, int32_t max_radius, int32_t* out_center,
                        int32_t* out_dist, int64_t* out_cut, int32_t* out_radius,
                        int32_t* out_accepted) {
  g_last_error[0] = 0;
  if (out_accepted) *out_accepted = -1;
  if (!g || !out_accepted) return fail(LDD_ERR_ARG, "NULL graph or out_accepted");
  if (g->uni) return fail(LDD_ERR_ARG, "a union graph is decomposed by ldd_union_decompose");
  if (!(beta > 0.0) || isinf(beta)) return fail(LDD_ERR_ARG, "beta must be finite and > 0");
  if (k < 1 || !shifts) return fail(LDD_ERR_ARG, "need k >= 1 shift vectors (k = %d)", k);
  if (g->n == 0) {
    *out_accepted = 0;
    if (out_cut) *out_cut = 0;
    if (out_radius) *out_radius = 0;
    return LDD_OK;
  }
  if (!out_center || !out_dist) return fail(LDD_ERR_ARG, "NULL output");
  for (int i = 0; i < k; ++i)
    if (!shifts[i]) return fail(LDD_ERR_ARG, "shifts[%d] is NULL", i);
  DeviceGuard dg(g->device);
  if (!dg.ok) return fail(LDD_ERR_CUDA, "cannot select device %d", g->device);
  cudaStream_t s = g->stream;
  const size_t n = (size_t)g->n;
  const bool dev_c = is_device_ptr(out_center), dev_d = is_device_ptr(out_dist);
  int* center = dev_c ? out_center : g->d_center;
  int* dist = dev_d ? out_dist : g->d_dist;
  u32* d_radius = &g->d_ctl->radius;
  int64_t cut = 0;
  u32 radius = 0;
  int launches = 0;
  for (int i = 0; i < k; ++i) {
    const double* d_shift = shifts[i];
    if (!is_device_ptr(shifts[i])) {
      CUDA_TRY(cudaMemcpyAsync(g->d_shift, shifts[i], n * 8, cudaMemcpyHostToDevice, s));
      d_shift = g->d_shift;
    }
    int l = 0, rc;
    if ((rc = decompose_on_device(g, d_shift, center, dist, &l)) != LDD_OK) return rc;
    launches += l;
    if ((rc = cut_on_device(g, center, &cut)) != LDD_OK) return rc;
    launches += g->stats.cut_launches;
    launches += launch_max_dist(dist, (u32)n, d_radius, g->num_sms, s);
    CUDA_TRY(cudaMemcpyAsync(&radius, d_radius, sizeof(u32), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (cut <= max_cut && (int64_t)radius <= (int64_t)max_radius) {
      *out_accepted = i;
      break;
    }
  }
  if (!dev_c) CUDA_TRY(cudaMemcpyAsync(out_center, center, n * 4, cudaMemcpyDeviceToHost, s));
  if (!dev_d) CUDA_TRY(cudaMemcpyAsync(out_dist, dist, n * 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (out_cut) *out_cut = cut;
  if (out_radius) *out_radius = (int32_t)radius;
  g->stats.launches = launches;
  return LDD_OK;
}

int ldd_decompose_batch(ldd_graph* g, int k, const double* betas, const double* const* shifts,
                        int32_t* const* out_center, int32_t* const* out_dist, int64_t* out_cut) {
  g_last_error[0] = 0;
  if (!g) return fail(LDD_ERR_ARG, "graph is NULL");
  if (g->uni) return fail(LDD_ERR_ARG, "a union graph is decomposed by ldd_union_decompose");
  if (k < 0) return fail(LDD_ERR_ARG, "k = %d is negative", k);
  if (k == 0) return LDD_OK;
  if (!betas || !shifts || !out_center || !out_dist)
    return fail(LDD_ERR_ARG, "NULL betas, shifts or output array");
  for (int i = 0; i < k; ++i) {
    if (!(betas[i] > 0.0) || isinf(betas[i]))
      return fail(LDD_ERR_ARG, "betas[%d] must be finite and > 0", i);
    if (g->n > 0 && (!shifts[i] || !out_center[i] || !out_dist[i]))
      return fail(LDD_ERR_ARG, "NULL shifts[%d] or output %d", i, i);
  }
  if (out_cut)
    for (int i = 0; i < k; ++i) out_cut[i] = 0;
  if (g->n == 0) return LDD_OK;
  DeviceGuard dg(g->device);
  if (!dg.ok) return fail(LDD_ERR_CUDA, "cannot select device %d", g->device);
  int rc = setup_batch(g);
  if (rc != LDD_OK) return rc;
  if ((rc = ensure_batch_headers(g, k)) != LDD_OK) return rc;
  const size_t n = (size_t)g->n, slot_bytes = align_up(8 * n, 256);
  double* d_in[2] = {(double*)g->batch_arena,
                     (double*)((char*)g->batch_arena + slot_bytes)};
  int* d_c[2] = {(int*)((char*)g->batch_arena + 2 * slot_bytes),
                 (int*)((char*)g->batch_arena + 3 * slot_bytes)};
  int* d_d[2] = {d_c[0] + n, d_c[1] + n};
  cudaStream_t s = g->stream;
  // slot j's shift buffer is free once the decomposition that read it is done
  // (ev_used) and its output buffers once their download is done (ev_out)
  // The first host shift vector nothing can overlap goes up in pieces, and the
  // rank's first pass starts on each piece as it lands.
  constexpr int kC = ldd_graph::kUploadChunks;
  u32 chunk_end[kC];
  ShiftChunks first;
  const bool chunk_first = !is_device_ptr(shifts[0]) && n >= ((size_t)1 << 20);
  if (chunk_first) {
    for (int c = 0; c < kC; ++c)
      chunk_end[c] = c + 1 < kC ? (u32)(((n * (c + 1) / kC) + 31) & ~(size_t)31) : (u32)n;
    first.n = kC;
    first.end = chunk_end;
    first.ev = g->ev_chunk;
  }
  auto upload = [&](int i) -> int {
    if (is_device_ptr(shifts[i])) return LDD_OK;
    const int j = i & 1;
    CUDA_TRY(cudaStreamWaitEvent(g->copy_in, g->ev_used[j], 0));
    if (i == 0 && chunk_first) {
      size_t lo = 0;
      for (int c = 0; c < kC; ++c) {
        const size_t hi = std::min<size_t>(chunk_end[c], n);
        if (hi > lo)
          CUDA_TRY(cudaMemcpyAsync(d_in[j] + lo, shifts[i] + lo, (hi - lo) * 8,
                                   cudaMemcpyHostToDevice, g->copy_in));
        CUDA_TRY(cudaEventRecord(g->ev_chunk[c], g->copy_in));
        lo = std::max(lo, hi);
      }
    } else {
      CUDA_TRY(cudaMemcpyAsync(d_in[j], shifts[i], n * 8, cudaMemcpyHostToDevice, g->copy_in));
    }
    CUDA_TRY(cudaEventRecord(g->ev_in[j], g->copy_in));
    return LDD_OK;
  };
  for (int j = 0; j < 2; ++j) {  // a fresh pipeline: nothing in flight
    CUDA_TRY(cudaEventRecord(g->ev_used[j], s));
    CUDA_TRY(cudaEventRecord(g->ev_out[j], g->copy_out));
  }
  // on a failure, copies into the caller's buffers must be over before returning
  auto drain = [&](int status) {
    cudaStreamSynchronize(g->copy_in);
    cudaStreamSynchronize(g->copy_out);
    cudaStreamSynchronize(g->cut_stream);
    cudaStreamSynchronize(s);
    return status;
  };
  // cut counts run on their own stream, W labelings to a pass over the cut
  // list: a wave of W consecutive decompositions.  With every output on the
  // device, W = 4 and one pass (launch_cut4) counts a wave after its last
  // finalize.  With outputs in the two host-side slots, W = 1: each cut count
  // overlaps the next decomposition's rank instead, which took less time than
  // waves of two (the second pass of a wave waits for the next round loop).
  // A round loop waits for the last wave's pass, so that it runs alone and
  // the output slot that pass reads is free again.
  const bool cuts = out_cut != nullptr;
  bool all_dev_c = true;
  for (int i = 0; i < k; ++i) all_dev_c = all_dev_c && is_device_ptr(out_center[i]);
  const int W = cuts && k > 1 && all_dev_c ? 4 : 1;
  const int* wave_c[4] = {};
  int nwave = 0, waves = 0, last_cut = -1;
  if (W > 1 && (rc = ensure_cut4(g)) != LDD_OK) return rc;
  if (cuts) {
    CUDA_TRY(cudaMemsetAsync(g->d_bcut, 0, (size_t)k * sizeof(u64), s));
    for (int j = 0; j < 2; ++j) CUDA_TRY(cudaEventRecord(g->ev_cut[j], s));
  }
  record(g, 0);
  if ((rc = upload(0)) != LDD_OK) return drain(rc);
  int launches = 0;
  for (int i = 0; i < k; ++i) {
    const int j = i & 1;
    if (i + 1 < k && (rc = upload(i + 1)) != LDD_OK) return drain(rc);  // overlaps decomposition i
    const bool dev_in = is_device_ptr(shifts[i]);
    const bool dev_c = is_device_ptr(out_center[i]), dev_d = is_device_ptr(out_dist[i]);
    const bool pieces = i == 0 && chunk_first;  // the rank waits for each piece itself
    if (!dev_in && !pieces) CUDA_TRY(cudaStreamWaitEvent(s, g->ev_in[j], 0));
    if (!dev_c || !dev_d) CUDA_TRY(cudaStreamWaitEvent(s, g->ev_out[j], 0));
    int* center = dev_c ? out_center[i] : d_c[j];
    int* dist = dev_d ? out_dist[i] : d_d[j];
    if ((rc = enqueue_rank(g, dev_in ? shifts[i] : d_in[j], &launches,
                           pieces ? &first : nullptr)) != LDD_OK)
      return drain(rc);
    if (cuts && last_cut >= 0) CUDA_TRY(cudaStreamWaitEvent(s, g->ev_cut[last_cut], 0));
    if ((rc = enqueue_bfs_finalize(g, center, dist, &launches)) != LDD_OK) return drain(rc);
    CUDA_TRY(cudaMemcpyAsync(g->h_bhdr + (size_t)i * sizeof(Header), g->d_ctl, sizeof(Header),
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaEventRecord(g->ev_used[j], s));
    if (!dev_c || !dev_d) {  // download overlaps the cut count and decomposition i + 1
      CUDA_TRY(cudaStreamWaitEvent(g->copy_out, g->ev_used[j], 0));
      if (!dev_c)
        CUDA_TRY(cudaMemcpyAsync(out_center[i], center, n * 4, cudaMemcpyDeviceToHost, g->copy_out));
      if (!dev_d)
        CUDA_TRY(cudaMemcpyAsync(out_dist[i], dist, n * 4, cudaMemcpyDeviceToHost, g->copy_out));
      CUDA_TRY(cudaEventRecord(g->ev_out[j], g->copy_out));
    }
    if (cuts) {
      wave_c[nwave++] = center;
      if (nwave == W || i == k - 1) {  // the wave's last finalize is queued: count its cuts
        CUDA_TRY(cudaStreamWaitEvent(g->cut_stream, g->ev_used[j], 0));
        u64* out = g->d_bcut + (i + 1 - nwave);
        if (nwave == 1)
          launches += launch_cut(g->cut, wave_c[0], g->d_hot, g->n_hot, g->d_hot_center, out,
                                 g->num_sms, g->cut_stream);
        else
          launches += launch_cut4(g->cut, wave_c, nwave, (u32)n, g->d_hot, g->n_hot, g->d_lab4,
                                  g->d_hot4, g->d_grp4, out, g->num_sms, g->cut_stream);
        CUDA_TRY(cudaGetLastError());
        last_cut = waves++ & 1;
        CUDA_TRY(cudaEventRecord(g->ev_cut[last_cut], g->cut_stream));
        nwave = 0;
      }
    }
  }
  if (cuts)
    CUDA_TRY(cudaMemcpyAsync(g->h_bcut, g->d_bcut, (size_t)k * sizeof(u64), cudaMemcpyDeviceToHost,
                             g->cut_stream));
  CUDA_TRY(cudaStreamSynchronize(g->cut_stream));
  CUDA_TRY(cudaStreamSynchronize(g->copy_out));
  CUDA_TRY(cudaStreamSynchronize(s));
  // headers in order: the first hard error is the call's status; a fast rank
  // path that asked for the exact path (or a larger start-bucket table) is
  // redone alone on the regular path, which handles both
  for (int i = 0; i < k; ++i) {
    Header h;
    memcpy(&h, g->h_bhdr + (size_t)i * sizeof(Header), sizeof(h));
    const u32 retry = kErrRankRetry | kErrBucketCap;
    if (h.err & ~retry) return header_error(h.err);
    if (h.err == 0) {
      header_stats(g, h, false);
      if (out_cut) out_cut[i] = (int64_t)g->h_bcut[i];
      continue;
    }
    const bool dev_in = is_device_ptr(shifts[i]);
    const bool dev_c = is_device_ptr(out_center[i]), dev_d = is_device_ptr(out_dist[i]);
    if (!dev_in)
      CUDA_TRY(cudaMemcpyAsync(d_in[0], shifts[i], n * 8, cudaMemcpyHostToDevice, s));
    int* center = dev_c ? out_center[i] : d_c[0];
    int* dist = dev_d ? out_dist[i] : d_d[0];
    int l = 0;
    if ((rc = decompose_on_device(g, dev_in ? shifts[i] : d_in[0], center, dist, &l)) != LDD_OK)
      return drain(rc);
    launches += l;
    if (out_cut && (rc = cut_on_device(g, center, &out_cut[i])) != LDD_OK) return drain(rc);
    if (!dev_c)
      CUDA_TRY(cudaMemcpyAsync(out_center[i], center, n * 4, cudaMemcpyDeviceToHost, s));
    if (!dev_d) CUDA_TRY(cudaMemcpyAsync(out_dist[i], dist, n * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  g->stats.launches = launches;
  g->stats.ms_h2d = -1.f;  // overlapped: not attributable
  g->stats.ms_d2h = -1.f;
  g->stats.ms_total = -1.f;
  g->stats.ms_rank = g->stats.ms_bfs = g->stats.ms_finalize = g->stats.ms_cut = -1.f;
  g->stats.replayed = 0;
  return LDD_OK;
}

int ldd_cut_edges(ldd_graph* g, const int32_t* center, int64_t* out_cut) {
  g_last_error[0] = 0;
  if (!g || !out_cut) return fail(LDD_ERR_ARG, "NULL argument");
  if (g->uni) return fail(LDD_ERR_ARG, "a union graph's cut counts come from ldd_union_decompose");
  *out_cut = 0;
  if (g->n == 0 || g->nnz == 0) return LDD_OK;
  if (!center) return fail(LDD_ERR_ARG, "center is NULL");
  DeviceGuard dg(g->device);
  if (!dg.ok) return fail(LDD_ERR_CUDA, "cannot select device %d", g->device);
  const int* d_center = center;
  if (!is_device_ptr(center)) {
    CUDA_TRY(cudaMemcpyAsync(g->d_center, center, (size_t)g->n * 4, cudaMemcpyHostToDevice,
                             g->stream));
    d_center = g->d_center;
  }
  return cut_on_device(g, d_center, out_cut);
}

int ldd_create_union(int k, ldd_graph* const* members, ldd_graph** out) {
  g_last_error[0] = 0;
  if (!out) return fail(LDD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (k < 1 || !members) return fail(LDD_ERR_ARG, "need k >= 1 members (k = %d)", k);
  int dev = -1;
  for (int i = 0; i < k; ++i) {
    const ldd_graph* m = members[i];
    if (!m) return fail(LDD_ERR_ARG, "member %d is NULL", i);
    if (m->uni) return fail(LDD_ERR_ARG, "member %d is itself a union", i);
    if (i == 0) dev = m->device;
    if (m->device != dev) return fail(LDD_ERR_ARG, "members live on different devices");
  }
  DeviceGuard dg(dev);
  if (!dg.ok) return fail(LDD_ERR_CUDA, "cannot select device %d", dev);
  const UnionCaps c = union_needs(k, members);
  if (c.N >= (1u << 30))
    return fail(LDD_ERR_RANGE, "union of %llu vertices (padded) must be < 2^30",
                (unsigned long long)c.N);
  if (c.E >= (1ull << 31))
    return fail(LDD_ERR_RANGE, "union of %llu arcs must be < 2^31", (unsigned long long)c.E);
  ldd_graph* g = nullptr;
  int rc = union_alloc(&g, dev, c);
  if (rc != LDD_OK) return rc;
  if ((rc = union_fill(g, k, members, nullptr, true)) != LDD_OK) {
    free_graph_memory(g);
    delete g;
    return rc;
  }
  *out = g;
  return LDD_OK;
}

int ldd_union_size(const ldd_graph* u, int32_t* out_k, int64_t* out_total) {
  if (!u || !u->uni) return fail(LDD_ERR_ARG, "not a union graph");
  if (out_k) *out_k = (int32_t)u->uni->k;
  if (out_total) *out_total = (int64_t)u->uni->total;
  return LDD_OK;
}

int ldd_union_decompose(ldd_graph* u, const double* betas, const double* shifts,
                        int32_t* out_center, int32_t* out_dist, int64_t* out_cut) {
  g_last_error[0] = 0;
  if (!u || !u->uni) return fail(LDD_ERR_ARG, "not a union graph");
  ldd_graph::Union& U = *u->uni;
  if (!betas) return fail(LDD_ERR_ARG, "betas is NULL");
  for (u32 i = 0; i < U.k; ++i)
    if (!(betas[i] > 0.0) || isinf(betas[i]))
      return fail(LDD_ERR_ARG, "betas[%u] must be finite and > 0", i);
  if (out_cut)
    for (u32 i = 0; i < U.k; ++i) out_cut[i] = 0;
  if (U.total == 0) return LDD_OK;
  if (!shifts || !out_center || !out_dist) return fail(LDD_ERR_ARG, "NULL shifts or output");
  DeviceGuard dg(u->device);
  if (!dg.ok) return fail(LDD_ERR_CUDA, "cannot select device %d", u->device);
  cudaStream_t s = u->stream;
  const size_t total = U.total;
  const bool dev_c = is_device_ptr(out_center), dev_d = is_device_ptr(out_dist);
  int* center = dev_c ? out_center : U.d_out_c;
  int* dist = dev_d ? out_dist : U.d_out_d;
  record(u, 0);
  const bool dev_in = is_device_ptr(shifts);
  const double* in = shifts;
  int launches = 0, cut_launches = 0;
  int rc = kRunRegular;
  if (u->replay && !u->replay_broken && u->regular_runs > 0) {
    CUDA_TRY(cudaMemcpyAsync(U.d_shift_in, shifts, total * 8,
                             dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    in = U.d_shift_in;
    rc = replay_fast(u, out_cut != nullptr, &launches);
    if (rc != LDD_OK && rc != kRunRegular) return rc;
    if (rc == LDD_OK) {
      center = U.d_out_c;
      dist = U.d_out_d;
      if (out_cut)
        for (u32 i = 0; i < U.k; ++i) out_cut[i] = (int64_t)u->h_cut[i];
      if (dev_c)
        CUDA_TRY(cudaMemcpyAsync(out_center, center, total * 4, cudaMemcpyDeviceToDevice, s));
      if (dev_d) CUDA_TRY(cudaMemcpyAsync(out_dist, dist, total * 4, cudaMemcpyDeviceToDevice, s));
    }
  } else if (!dev_in) {
    CUDA_TRY(cudaMemcpyAsync(U.d_shift_in, shifts, total * 8, cudaMemcpyHostToDevice, s));
    in = U.d_shift_in;
  }
  if (rc == kRunRegular) {
    if ((rc = union_run(u, in, center, dist, out_cut != nullptr, &launches, &cut_launches)) !=
        LDD_OK)
      return rc;
    if (out_cut)
      CUDA_TRY(cudaMemcpyAsync(out_cut, U.d_cut, (size_t)U.k * 8, cudaMemcpyDeviceToHost, s));
  }
  if (!dev_c) CUDA_TRY(cudaMemcpyAsync(out_center, center, total * 4, cudaMemcpyDeviceToHost, s));
  if (!dev_d) CUDA_TRY(cudaMemcpyAsync(out_dist, dist, total * 4, cudaMemcpyDeviceToHost, s));
  record(u, 5);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s));
  ldd_stats& st = u->stats;
  st.launches = launches;
  st.cut_launches = cut_launches;
  st.ms_cut = (out_cut && !st.replayed) ? elapsed(u, 6, 7) : (out_cut ? -1.f : 0.f);
  st.ms_total = elapsed(u, 0, 5);
  return LDD_OK;
}

int ldd_get_tuning(const ldd_graph* g, ldd_tuning* out) {
  if (!g || !out) return fail(LDD_ERR_ARG, "NULL argument");
  out->bfs_blocks_per_sm = g->bfs_per_sm;
  out->pull_alpha = (int32_t)g->pull_alpha;
  out->pull_beta = (int32_t)g->pull_beta;
  out->pull_gamma = (int32_t)g->pull_gamma;
  out->probe_min_arcs = (int32_t)g->probe_min_arcs;
  out->low_degree_rounds = g->low_degree_rounds ? 1 : 0;
  out->window_levels = (int32_t)g->window_levels;
  out->window_max_frontier = (int32_t)std::min<u32>(g->window_max_q, 0x7fffffffu);
  out->window_queue = (int32_t)std::min<u32>(g->window_queue, 0x7fffffffu);
  out->bfs_span = (int32_t)g->bfs_span;
  out->ms = -1.f;
  return LDD_OK;
}

int ldd_set_tuning(ldd_graph* g, const ldd_tuning* t) {
  if (!g || !t) return fail(LDD_ERR_ARG, "NULL argument");
  int max_per_sm = 0;
  if (bfs_grid_size(g->num_sms, &max_per_sm) <= 0)
    return fail(LDD_ERR_CUDA, "BFS kernel occupancy query failed");
  if (t->bfs_blocks_per_sm < 1 || t->bfs_blocks_per_sm > max_per_sm || t->pull_alpha < 0 ||
      t->pull_beta < 1 || t->pull_gamma < 0 || t->probe_min_arcs < 0 ||
      (t->low_degree_rounds != 0 && t->low_degree_rounds != 1) || t->window_levels < 0 ||
      t->window_levels > 4096 || t->window_max_frontier < 0 || t->window_queue < 0 ||
      t->bfs_span < kBfsBase || t->bfs_span > kBfsMaxSpan || t->bfs_span % kBfsBase != 0)
    return fail(LDD_ERR_ARG, "tuning out of range (blocks per SM 1 .. %d)", max_per_sm);
  g->bfs_per_sm = t->bfs_blocks_per_sm;
  g->bfs_grid = g->bfs_per_sm * g->num_sms;
  g->pull_alpha = (u32)t->pull_alpha;
  g->pull_beta = (u32)t->pull_beta;
  g->pull_gamma = (u32)t->pull_gamma;
  g->probe_min_arcs = (u32)t->probe_min_arcs;
  g->low_degree_rounds = t->low_degree_rounds != 0;
  g->window_levels = (u32)t->window_levels;
  g->window_max_q = (u32)t->window_max_frontier;
  g->window_queue = (u32)t->window_queue;
  g->bfs_span = (u32)t->bfs_span;
  g->stats.bfs_grid = g->bfs_grid;
  drop_replay(g);  // captured kernels carry the old parameters
  return LDD_OK;
}

int ldd_autotune(ldd_graph* g, const double* shifts, int reps, ldd_tuning* out) {
  g_last_error[0] = 0;
  if (!g || !shifts || !out) return fail(LDD_ERR_ARG, "NULL argument");
  if (reps < 1) return fail(LDD_ERR_ARG, "reps must be >= 1");
  DeviceGuard dg(g->device);
  if (!dg.ok) return fail(LDD_ERR_CUDA, "cannot select device %d", g->device);
  if (g->n == 0) return ldd_get_tuning(g, out);
  cudaStream_t s = g->stream;
  const size_t n = g->uni ? (size_t)g->uni->total : (size_t)g->n;
  // shifts to the device once; outputs to the library's buffers
  double* d_in = g->uni ? g->uni->d_shift_in : g->d_shift;
  CUDA_TRY(cudaMemcpyAsync(d_in, shifts, n * 8,
                           is_device_ptr(shifts) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return fail(LDD_ERR_CUDA, "cudaEventCreate failed");
  }
  const bool saved_replay = g->replay;
  g->replay = false;
  // one decomposition with the current parameters, best of reps (ms), or < 0
  auto measure = [&](float* best) -> int {
    *best = 1e30f;
    for (int r = 0; r <= reps; ++r) {  // the first run warms up
      int l = 0, cl = 0, rc;
      CUDA_TRY(cudaEventRecord(e0, s));
      if (g->uni)
        rc = union_run(g, d_in, g->uni->d_out_c, g->uni->d_out_d, false, &l, &cl);
      else
        rc = decompose_on_device(g, d_in, g->d_center, g->d_dist, &l);
      if (rc != LDD_OK) return rc;
      CUDA_TRY(cudaEventRecord(e1, s));
      CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      if (r > 0) *best = std::min(*best, ms);
    }
    return LDD_OK;
  };
  ldd_tuning cur;
  ldd_get_tuning(g, &cur);
  float best_ms;
  int rc = measure(&best_ms);
  int max_per_sm = 1;
  bfs_grid_size(g->num_sms, &max_per_sm);
  // coordinate descent, one parameter at a time over a few candidates
  const int32_t alphas[] = {4, 8, 14, 24, 48};
  const int32_t betas[] = {8, 16, 24, 48, 96};
  const int32_t gammas[] = {2, 4, 8, 16, 64};
  const int32_t probes[] = {1 << 12, 1 << 16, 1 << 20, 1 << 30};
  const int32_t ld_vals[2] = {0, 1};
  const int32_t window_vals[3] = {1, 8, 16};
  const int32_t span_vals[3] = {1024, 2048, 4096};
  const bool ld_possible = g->max_degree <= (u32)kLdMaxDegree;
  for (int param = 0; param < 8 && rc == LDD_OK; ++param) {
    const int32_t* vals = param == 0 ? alphas : param == 1 ? betas : param == 2 ? gammas : probes;
    int nv = param == 3 ? 4 : 5;
    int32_t per_sm_vals[2] = {1, max_per_sm};
    if (param == 4) {
      vals = per_sm_vals;
      nv = max_per_sm > 1 ? 2 : 1;
    }
    if (param == 5) {  // windows of levels, where low-degree rounds run
      vals = window_vals;
      nv = (ld_possible && cur.low_degree_rounds) ? 3 : 0;
    }
    if (param == 6) {  // the low-degree rounds, where the graph allows them
      vals = ld_vals;
      nv = ld_possible ? 2 : 0;
    }
    if (param == 7) {  // arcs per CTA step, where edge-balanced rounds run
      vals = span_vals;
      nv = (ld_possible && cur.low_degree_rounds) ? 0 : 3;
    }
    for (int i = 0; i < nv && rc == LDD_OK; ++i) {
      ldd_tuning t = cur;
      int32_t* field = param == 0 ? &t.pull_alpha : param == 1 ? &t.pull_beta
                     : param == 2 ? &t.pull_gamma : param == 3 ? &t.probe_min_arcs
                     : param == 4 ? &t.bfs_blocks_per_sm : param == 5 ? &t.window_levels
                     : param == 6 ? &t.low_degree_rounds : &t.bfs_span;
      if (*field == vals[i]) continue;
      *field = vals[i];
      if ((rc = ldd_set_tuning(g, &t)) != LDD_OK) break;
      float ms;
      if ((rc = measure(&ms)) != LDD_OK) break;
      if (ms < best_ms * 0.98f) {  // keep only a clear gain
        best_ms = ms;
        cur = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  g->replay = saved_replay;
  const int rc2 = ldd_set_tuning(g, &cur);
  if (rc != LDD_OK) return rc;
  if (rc2 != LDD_OK) return rc2;
  *out = cur;
  out->ms = best_ms;
  return LDD_OK;
}

int ldd_set_graph_replay(ldd_graph* g, int enable) {
  if (!g) return fail(LDD_ERR_ARG, "graph is NULL");
  DeviceGuard dg(g->device);
  g->replay = enable != 0;
  if (!g->replay) {
    cudaStreamSynchronize(g->stream);
    drop_replay(g);
  }
  g->replay_broken = false;  // a new request gets a new capture attempt
  return LDD_OK;
}

int ldd_set_wait_limits(ldd_graph* g, const ldd_wait_limits* w) {
  if (!g || !w) return fail(LDD_ERR_ARG, "NULL graph or limits");
  if (w->stall_barrier > 1 || w->stall_lookback > 1)
    return fail(LDD_ERR_ARG, "stall_barrier and stall_lookback must be 0 or 1");
  DeviceGuard dg(g->device);
  cudaStreamSynchronize(g->stream);
  drop_replay(g);  // captured graphs hold the old kernel arguments
  g->spin_limit = w->barrier_polls ? w->barrier_polls : kDefaultBarrierPolls;
  g->lookback_limit = w->lookback_polls ? w->lookback_polls : kDefaultLookbackPolls;
  g->stall_barrier = w->stall_barrier;
  g->stall_lookback = w->stall_lookback;
  return LDD_OK;
}

int ldd_get_wait_limits(const ldd_graph* g, ldd_wait_limits* out) {
  if (!g || !out) return fail(LDD_ERR_ARG, "NULL graph or output");
  out->barrier_polls = g->spin_limit;
  out->lookback_polls = g->lookback_limit;
  out->stall_barrier = g->stall_barrier;
  out->stall_lookback = g->stall_lookback;
  return LDD_OK;
}

}  // extern "C"

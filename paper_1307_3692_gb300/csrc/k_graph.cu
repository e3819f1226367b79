// Per-graph tables, assignment and verification kernels (Miller, Peng, Xu 2013).
//
// finalize (Algorithm 1 step 4, Algorithm 2 step 2): a settled key
// (level << 32) | rank names the center order[rank]; the hop distance is the
// key's level minus the center's own start level, which is the level of the
// center's key (a center is its own center, so its key is its start key).
//
// cut (Definition 1.1, second condition; Section 4 notes the check costs
// O(m) work): arcs (v, w) with v < w whose endpoints have different centers.
//
// Components.  The assignment of Algorithm 2 never crosses a connected
// component (other components are at infinite distance), so every component
// is an independent instance of the same problem on the same keys.  At graph
// creation the components are labelled (union-find with atomicCAS hooking of
// the larger root under the smaller), and components of at most 32 vertices
// are listed with a 32-bit adjacency mask per vertex over the lanes of one
// warp.  Per decomposition, one warp per such component iterates
//     key[v] <- min(key[v], min over neighbours w of key[w] + 2^32)
// with warp shuffles until nothing changes: the same fixed point the BFS
// reaches, i.e. the exact labels of the super-source shortest path of
// Section 4.  Those vertices, and vertices without arcs, are kept out of the
// BFS start buckets, so the round loop ends when the large components are
// settled instead of visiting every start round up to floor(delta_max).
//
// Arc-parallel kernels (cut, hooking) split the arcs into equal spans, one per
// CTA; the rows covering a span (a precomputed first-row table over the
// vertices with arcs) are located with a block max-scan in shared memory, so
// high-degree rows are split across CTAs and reads of col are coalesced.
#include "ldd_internal.cuh"

namespace ldd {

namespace {

constexpr u32 kFull = 0xffffffffu;
constexpr int kCutWinBatch = 4;
constexpr u32 kNone = 0xffffffffu;

__global__ void __launch_bounds__(256) k_finalize(const u64* __restrict__ key,
                                                  const u32* __restrict__ order, u32 n,
                                                  int* __restrict__ center, int* __restrict__ dist,
                                                  const u32* err) {
  if (*(volatile const u32*)err != 0u) return;  // outputs are not written after a failure
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const u64 k = key[v];
    const u32 c = order[min((u32)k, n - 1)];
    const u64 kc = key[c];
    center[v] = (int)c;
    dist[v] = (int)((u32)(k >> 32) - (u32)(kc >> 32));
  }
}

struct SpanSmem {
  int owner[kCutSpan];
  u32 v[kCutSpan + 1];
  int aux[kCutSpan + 1];
  int wtot[kCutThreads / 32];
  unsigned long long wsum[kCutThreads / 32];
};

// Fills s.owner[k] with the window index of the row that holds arc e0 + k of
// span `c`; s.v[j] is that row's vertex and s.aux[j] = aux(vertex).  Returns
// false (and leaves the span unprocessed) if the tables are inconsistent.
template <class Aux>
__device__ __forceinline__ bool span_window(SpanSmem& s, const int* __restrict__ row_ptr,
                                            const u32* __restrict__ nzv,
                                            const u32* __restrict__ first, u32 n_items, u32 nnz,
                                            u32 c, u32& e0, int& len, Aux aux) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const u32 nch = (nnz + kCutSpan - 1) / kCutSpan;
  e0 = c * kCutSpan;
  const u32 e1 = min(e0 + kCutSpan, nnz);
  len = (int)(e1 - e0);
  const u32 i0 = first[c];
  const u32 ilast = (c + 1 < nch) ? first[c + 1] : n_items - 1;
  const int nwin = (int)(ilast - i0) + 1;
  if (nwin < 1 || nwin > kCutSpan + 1 || ilast >= n_items) return false;
  for (int j = t; j < len; j += kCutThreads) s.owner[j] = 0;
  __syncthreads();
  for (int j0 = 0; j0 < nwin; j0 += kCutThreads * kCutWinBatch) {
    u32 v[kCutWinBatch], off[kCutWinBatch];
#pragma unroll
    for (int i = 0; i < kCutWinBatch; ++i) {
      const int j = j0 + i * kCutThreads + t;
      v[i] = (j < nwin) ? nzv[i0 + j] : kNone;
    }
    int ax[kCutWinBatch];
#pragma unroll
    for (int i = 0; i < kCutWinBatch; ++i) {
      off[i] = e1;
      if (v[i] != kNone) {
        off[i] = (u32)row_ptr[v[i]];
        ax[i] = aux(v[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < kCutWinBatch; ++i)
      if (off[i] < e1) {
        const int j = j0 + i * kCutThreads + t;
        s.v[j] = v[i];
        s.aux[j] = ax[i];
        atomicMax(&s.owner[off[i] > e0 ? off[i] - e0 : 0u], j);
      }
  }
  __syncthreads();
  // inclusive max-scan of owner[0 .. len)
  constexpr int kPer = kCutSpan / kCutThreads;
  const int b = t * kPer;
  int run = -1;
#pragma unroll
  for (int i = 0; i < kPer; ++i)
    if (b + i < len) {
      run = max(run, s.owner[b + i]);
      s.owner[b + i] = run;
    }
  int x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x = max(x, y);
  }
  if (lane == 31) s.wtot[w] = x;
  __syncthreads();
  int carry = -1;
  for (int i = 0; i < w; ++i) carry = max(carry, s.wtot[i]);
  const int prev = __shfl_up_sync(kFull, x, 1);
  if (lane > 0) carry = max(carry, prev);
#pragma unroll
  for (int i = 0; i < kPer; ++i)
    if (b + i < len) s.owner[b + i] = max(s.owner[b + i], carry);
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(kCutThreads) k_cut(const int* __restrict__ row_ptr,
                                                     const int* __restrict__ col,
                                                     const u32* __restrict__ nzv,
                                                     const u32* __restrict__ first, u32 n_items,
                                                     u32 nnz, u32 n_vert,
                                                     const int* __restrict__ center, u64* out) {
  __shared__ SpanSmem s;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  u32 e0;
  int len;
  if (!span_window(s, row_ptr, nzv, first, n_items, nnz, blockIdx.x, e0, len,
                   [&](u32 v) { return center[v]; }))
    return;
  unsigned long long cnt = 0;
  constexpr int kPerEdge = kCutSpan / kCutThreads;
  u32 wv[kPerEdge];
#pragma unroll
  for (int i = 0; i < kPerEdge; ++i) {
    const int kk = i * kCutThreads + t;
    wv[i] = (kk < len) ? (u32)col[e0 + kk] : kNone;
  }
  int cw[kPerEdge];
#pragma unroll
  for (int i = 0; i < kPerEdge; ++i) {
    const int kk = i * kCutThreads + t;
    cw[i] = 0;
    if (wv[i] < n_vert && s.v[s.owner[kk]] < wv[i]) cw[i] = center[wv[i]];
  }
#pragma unroll
  for (int i = 0; i < kPerEdge; ++i) {
    const int kk = i * kCutThreads + t;
    if (wv[i] < n_vert) {
      const int j = s.owner[kk];
      if (s.v[j] < wv[i] && s.aux[j] != cw[i]) ++cnt;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kFull, cnt, o);
  if (lane == 0) s.wsum[w] = cnt;
  __syncthreads();
  if (t == 0) {
    unsigned long long tot = 0;
    for (int i = 0; i < kCutThreads / 32; ++i) tot += s.wsum[i];
    if (tot) atomicAdd(out, tot);
  }
}

// ---------------------------------------------------------------- components
// Root of v: parents only ever point to smaller ids, so the walk ends at the
// first vertex that is its own parent; path halving on the way.
__device__ __forceinline__ u32 cc_root(u32* parent, u32 v) {
  volatile u32* p = parent;
  u32 cur = p[v];
  if (cur != v) {
    u32 prev = v, next;
    while (cur > (next = p[cur])) {
      p[prev] = next;
      prev = cur;
      cur = next;
    }
  }
  return cur;
}

__device__ __forceinline__ void cc_unite(u32* parent, u32 a, u32 b) {
  u32 ra = cc_root(parent, a), rb = cc_root(parent, b);
  while (ra != rb) {
    if (ra < rb) {
      const u32 ret = atomicCAS(parent + rb, rb, ra);
      if (ret == rb) break;
      rb = cc_root(parent, ret);
    } else {
      const u32 ret = atomicCAS(parent + ra, ra, rb);
      if (ret == ra) break;
      ra = cc_root(parent, ret);
    }
  }
}

__global__ void k_iota(u32* p, u32 n) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) p[v] = v;
}

__global__ void __launch_bounds__(kCutThreads) k_cc_hook(const int* __restrict__ row_ptr,
                                                         const int* __restrict__ col,
                                                         const u32* __restrict__ nzv,
                                                         const u32* __restrict__ first,
                                                         u32 n_items, u32 nnz, u32 n_vert,
                                                         u32* parent) {
  __shared__ SpanSmem s;
  u32 e0;
  int len;
  if (!span_window(s, row_ptr, nzv, first, n_items, nnz, blockIdx.x, e0, len,
                   [](u32) { return 0; }))
    return;
  for (int kk = threadIdx.x; kk < len; kk += kCutThreads) {
    const u32 v = s.v[s.owner[kk]];
    const u32 w = (u32)col[e0 + kk];
    if (w < v) cc_unite(parent, v, w);  // each undirected edge once
  }
}

// Final labels.  The walk here only reads: a compressing walk could overwrite
// a label another thread has just set to the root with a non-root ancestor.
// Every store is a root, so concurrent walks stay valid.
__global__ void k_cc_finish(u32* parent, u32* csize, u32 n) {
  volatile u32* p = parent;
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    u32 r = v, nx;
    while ((nx = p[r]) != r) r = nx;
    p[v] = r;
    atomicAdd(csize + r, 1u);
  }
}

// A root of a component with 2..32 vertices reserves a slot and a range of
// the member list.
__global__ void k_small_roots(const u32* __restrict__ parent, const u32* __restrict__ csize,
                              u32 n, u32* root_off, u32* comp_off, u32* comp_len, u32* counters) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (parent[v] != v) continue;
    const u32 sz = csize[v];
    if (sz < 2 || sz > kSmallComp) continue;
    const u32 slot = atomicAdd(counters + 0, 1u);
    const u32 off = atomicAdd(counters + 1, sz);
    comp_off[slot] = off;
    comp_len[slot] = sz;
    root_off[v] = off;
  }
}

// Members take a lane of their component; every vertex gets its BFS-exclusion
// bit (no arcs, or a component of at most 32 vertices).
__global__ void k_small_members(const int* __restrict__ row_ptr, const u32* __restrict__ parent,
                                const u32* __restrict__ csize, const u32* __restrict__ root_off,
                                u32 n, u32* fill, u32* comp_v, u32* lane_of, u32* excl,
                                u32* counters) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const u32 r = parent[v];
    const u32 sz = csize[r];
    const bool small = sz <= kSmallComp;
    const bool no_arcs = row_ptr[v + 1] == row_ptr[v];
    if (small && sz >= 2) {
      const u32 pos = atomicAdd(fill + r, 1u);
      comp_v[root_off[r] + pos] = v;
      lane_of[v] = pos;
    }
    if (small || no_arcs) {
      atomicOr(excl + (v >> 5), 1u << (v & 31));
    } else {
      atomicAdd(counters + 2, 1u);  // vertices the BFS settles
    }
  }
}

__global__ void k_small_adj(const int* __restrict__ row_ptr, const int* __restrict__ col,
                            const u32* __restrict__ comp_v, const u32* __restrict__ lane_of,
                            u32 total, u32* adj) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const u32 v = comp_v[i];
    u32 m = 0;
    for (int e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      const u32 l = lane_of[col[e]];
      if (l < 32) m |= 1u << l;
    }
    adj[i] = m;
  }
}

// One warp per small component: exact relaxation to the fixed point.
__global__ void __launch_bounds__(256) k_small_comp(const u32* __restrict__ comp_off,
                                                    const u32* __restrict__ comp_len, u32 ncomp,
                                                    const u32* __restrict__ comp_v,
                                                    const u32* __restrict__ adj, u64* key,
                                                    const u32* err) {
  if (*(volatile const u32*)err != 0u) return;
  const u32 lane = threadIdx.x & 31;
  const u32 warps = gridDim.x * (blockDim.x / 32);
  for (u32 c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); c < ncomp; c += warps) {
    const u32 off = comp_off[c], sz = comp_len[c];
    u32 v = 0, m = 0;
    u64 k = ~0ull;
    if (lane < sz) {
      v = comp_v[off + lane];
      m = adj[off + lane];
      k = key[v];
    }
    for (u32 it = 0; it < sz; ++it) {
      u64 best = k;
      for (u32 t = 0; t < sz; ++t) {
        const u64 kt = __shfl_sync(kFull, k, t);
        if (m >> t & 1u) best = min(best, kt + kLevelOne);
      }
      const bool changed = best != k;
      k = best;
      if (!__any_sync(kFull, changed)) break;
    }
    if (lane < sz) key[v] = k;
  }
}

u32 grid_for(u32 n, int num_sms) {
  return (u32)max(1ll, min((long long)(n + 255) / 256, (long long)num_sms * 8));
}

}  // namespace

int launch_finalize(const u64* key, const u32* order, u32 n, int* center, int* dist,
                    const u32* err, int num_sms, cudaStream_t s) {
  k_finalize<<<grid_for(n, num_sms), 256, 0, s>>>(key, order, n, center, dist, err);
  return 1;
}

int launch_cut(const int* row_ptr, const int* col, const u32* nzv, const u32* cut_first,
               u32 n_items, u32 nnz, u32 n_vert, const int* center, u64* out, cudaStream_t s) {
  const u32 nch = (nnz + kCutSpan - 1) / kCutSpan;
  if (nch == 0) return 0;
  k_cut<<<nch, kCutThreads, 0, s>>>(row_ptr, col, nzv, cut_first, n_items, nnz, n_vert, center,
                                    out);
  return 1;
}

int launch_small_comp(const SmallComps& sc, u64* key, const u32* err, int num_sms, cudaStream_t s) {
  if (sc.ncomp == 0) return 0;
  const u32 blocks = (u32)min((long long)(sc.ncomp + 7) / 8, (long long)num_sms * 8);
  k_small_comp<<<blocks, 256, 0, s>>>(sc.comp_off, sc.comp_len, sc.ncomp, sc.comp_v, sc.adj, key,
                                      err);
  return 1;
}

cudaError_t components_phase1(const int* row_ptr, const int* col, const u32* nzv,
                              const u32* cut_first, u32 n_items, u32 n, u32 nnz, int num_sms,
                              const CompScratch& t, u32* excl, u32 counts[3], cudaStream_t s) {
  const u32 g = grid_for(n, num_sms);
  cudaError_t e;
  if ((e = cudaMemsetAsync(t.csize, 0, (size_t)n * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(t.fill, 0, (size_t)n * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(t.counters, 0, 3 * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(t.lane_of, 0xff, (size_t)n * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(excl, 0, ((size_t)n + 31) / 32 * 4, s)) != cudaSuccess) return e;
  k_iota<<<g, 256, 0, s>>>(t.parent, n);
  const u32 nch = (nnz + kCutSpan - 1) / kCutSpan;
  if (nch > 0)
    k_cc_hook<<<nch, kCutThreads, 0, s>>>(row_ptr, col, nzv, cut_first, n_items, nnz, n, t.parent);
  k_cc_finish<<<g, 256, 0, s>>>(t.parent, t.csize, n);
  k_small_roots<<<g, 256, 0, s>>>(t.parent, t.csize, n, t.root_off, t.comp_off, t.comp_len,
                                  t.counters);
  k_small_members<<<g, 256, 0, s>>>(row_ptr, t.parent, t.csize, t.root_off, n, t.fill, t.comp_v,
                                    t.lane_of, excl, t.counters);
  if ((e = cudaMemcpyAsync(counts, t.counters, 3 * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

cudaError_t components_phase2(const int* row_ptr, const int* col, const CompScratch& t,
                              const SmallComps& sc, int num_sms, cudaStream_t s) {
  if (sc.total > 0)
    k_small_adj<<<grid_for(sc.total, num_sms), 256, 0, s>>>(row_ptr, col, sc.comp_v, t.lane_of,
                                                             sc.total, sc.adj);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace ldd

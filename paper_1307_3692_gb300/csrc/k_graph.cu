// Per-graph tables, assignment and verification kernels (Miller, Peng, Xu 2013).
//
// finalize (Algorithm 1 step 4, Algorithm 2 step 2): a settled key
// (level << 32) | rank names the center order[rank]; the hop distance is the
// key's level minus the center's own start level, which is the level of the
// center's key (a center is its own center, so its key is its start key).
//
// cut (Definition 1.1, second condition; Section 4 notes the check costs
// O(m) work): edges {v, w} whose endpoints have different centers, each
// counted once, over the graph's grouped cut list (4 bytes per edge).
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
#include <algorithm>

#include "ldd_internal.cuh"

namespace ldd {

namespace {

constexpr u32 kFull = 0xffffffffu;

// Each thread takes kFinIpt vertices per step (coalesced across the warp) and
// issues their loads level by level (own keys, then the centers, then the
// centers' keys), so that the three dependent gathers of several vertices
// are in flight together.
constexpr int kFinIpt = 4;

__global__ void __launch_bounds__(256) k_finalize(const u64* __restrict__ key,
                                                  const u32* __restrict__ order,
                                                  const u32* __restrict__ solo, u32 n,
                                                  int* __restrict__ center, int* __restrict__ dist,
                                                  const u32* err) {
  if (*(volatile const u32*)err != 0u) return;  // outputs are not written after a failure
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 v0 = blockIdx.x * blockDim.x + threadIdx.x; v0 < n; v0 += stride * kFinIpt) {
    u32 v[kFinIpt], c[kFinIpt];
    bool live[kFinIpt], alone[kFinIpt];
    u64 k[kFinIpt], kc[kFinIpt];
#pragma unroll
    for (int q = 0; q < kFinIpt; ++q) {
      v[q] = v0 + (u32)q * stride;
      live[q] = v[q] < n;
      // alone in its component: the key is unused, the vertex is its own center
      alone[q] = live[q] && ((__ldg(solo + (v[q] >> 5)) >> (v[q] & 31)) & 1u);
      k[q] = (live[q] && !alone[q]) ? key[v[q]] : 0ull;
    }
#pragma unroll
    for (int q = 0; q < kFinIpt; ++q)
      c[q] = (live[q] && !alone[q]) ? order[min((u32)k[q], n - 1)] : v[q];
#pragma unroll
    for (int q = 0; q < kFinIpt; ++q)
      kc[q] = (live[q] && !alone[q]) ? key[c[q]] : k[q];
#pragma unroll
    for (int q = 0; q < kFinIpt; ++q)
      if (live[q]) {
        center[v[q]] = (int)c[q];
        dist[v[q]] = alone[q] ? 0 : (int)((u32)(k[q] >> 32) - (u32)(kc[q] >> 32));
      }
  }
}

// Labels of the hot table's vertices, gathered once per cut count.
__global__ void k_hot_centers(const u32* __restrict__ hot, u32 n_hot,
                              const int* __restrict__ center, int* __restrict__ hot_center) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_hot) hot_center[i] = center[hot[i]];
}

// Cut count over the grouped cut list (CutList in ldd_internal.cuh), in two
// streaming passes.  k_group_labels reads every group's cold label once.
// k_cut then streams the edges: each warp step covers 128 edges, one 16-byte
// load of 4 hot endpoints per lane; an edge finds its group from its block's
// first group and group-start mask (one popc), so its cold label is one
// gather from the per-group labels (consecutive edges share it).  Hot
// endpoints in the hot table read shared memory; others are one gather each.
// The next step's edge and block loads are issued before this step's label
// reads, and there is no block-wide synchronisation.
//
// U = true: a union of graphs (k_union.cu): hot[] and grp_v[] are already in
// the caller layout, and every member's count goes to its own counter, one
// atomic per warp step when the step's edges share a member.
constexpr int kCutThreads = 1024;

// Four groups per thread per step, their label gathers in flight together.
constexpr int kLabIpt = 4;

template <bool U>
__global__ void __launch_bounds__(256) k_group_labels(CutList cl, const int* __restrict__ center) {
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 g0 = blockIdx.x * blockDim.x + threadIdx.x; g0 < cl.ngrp; g0 += stride * kLabIpt) {
    int lab[kLabIpt];
#pragma unroll
    for (int q = 0; q < kLabIpt; ++q) {
      const u32 g = g0 + (u32)q * stride;
      lab[q] = g < cl.ngrp ? center[__ldg(cl.grp_v + g)] : 0;
    }
#pragma unroll
    for (int q = 0; q < kLabIpt; ++q) {
      const u32 g = g0 + (u32)q * stride;
      if (g >= cl.ngrp) break;
      if (U)  // member and label in one word: one gather per edge in k_cut
        reinterpret_cast<u64*>(cl.grp_lab)[g] = ((u64)__ldg(cl.grp_m + g) << 32) | (u32)lab[q];
      else
        cl.grp_lab[g] = lab[q];
    }
  }
}

__device__ __forceinline__ u32 bits_upto(u32 j) { return j >= 31u ? 0xffffffffu : (2u << j) - 1u; }

template <bool U>
__global__ void __launch_bounds__(kCutThreads, 1) k_cut(CutList cl, const int* __restrict__ center,
                                                        const int* __restrict__ hot_center,
                                                        u32 n_hot, u64* out) {
  extern __shared__ int4 cut_smem[];
  int* s_hot = reinterpret_cast<int*>(cut_smem);
  __shared__ unsigned long long wsum[kCutThreads / 32];
  const u32 tid = threadIdx.x, lane = tid & 31;
  if (!U) {
    const int4* hc4 = reinterpret_cast<const int4*>(hot_center);  // cudaMalloc'd: aligned
    for (u32 i = tid; i < n_hot / 4; i += blockDim.x) cut_smem[i] = __ldg(hc4 + i);
    for (u32 i = (n_hot & ~3u) + tid; i < n_hot; i += blockDim.x) s_hot[i] = hot_center[i];
    __syncthreads();
  }
  const int4* hot4 = reinterpret_cast<const int4*>(cl.hot);  // cudaMalloc'd: aligned
  const u32 nchunk = (cl.m + 127) / 128;                       // 128 edges per warp step
  const u32 stride = gridDim.x * (kCutThreads / 32);
  unsigned long long cnt = 0;
  u32 c = blockIdx.x * (kCutThreads / 32) + (tid >> 5);
  // lane's four edges: 4 lane .. 4 lane + 3 of the chunk, in block lane / 8
  auto load = [&](u32 cc, int4& h, u32& bg, u32& bm) {
    const u32 e0 = cc * 128 + 4 * lane;
    if (e0 + 3 < cl.m) {
      h = __ldcs(hot4 + (e0 >> 2));
    } else {
      h.x = e0 < cl.m ? cl.hot[e0] : 0;
      h.y = e0 + 1 < cl.m ? cl.hot[e0 + 1] : 0;
      h.z = e0 + 2 < cl.m ? cl.hot[e0 + 2] : 0;
      h.w = 0;
    }
    const u32 b = e0 >> 5;
    bg = b < cl.nblk ? __ldg(cl.blk_g + b) : 0u;
    bm = b < cl.nblk ? __ldg(cl.blk_mask + b) : 0u;
  };
  int4 h;
  u32 bg = 0, bm = 0;
  if (c < nchunk) load(c, h, bg, bm);
  for (; c < nchunk; c += stride) {
    int4 nh = make_int4(0, 0, 0, 0);
    u32 nbg = 0, nbm = 0;
    if (c + stride < nchunk) load(c + stride, nh, nbg, nbm);
    const u32 e0 = c * 128 + 4 * lane, j0 = (4 * lane) & 31u;
    const int hv[4] = {h.x, h.y, h.z, h.w};
    u32 g[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) g[q] = bg + __popc(bm & bits_upto(j0 + (u32)q));
    int cl_lab[4], hl[4];
    u32 gm[4];  // unions: the member of each edge
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool valid = e0 + (u32)q < cl.m;
      if (U) {
        const u64 lm = valid ? __ldg(reinterpret_cast<const u64*>(cl.grp_lab) + g[q]) : 0ull;
        cl_lab[q] = (int)(u32)lm;
        gm[q] = (u32)(lm >> 32);
        hl[q] = valid ? center[hv[q]] : 0;
      } else {
        cl_lab[q] = valid ? __ldg(cl.grp_lab + g[q]) : 0;
        hl[q] = valid ? (hv[q] < 0 ? s_hot[hv[q] & 0x7fffffff] : center[hv[q]]) : 0;
      }
    }
    if (U) {
      // per-member counts: the lane's edges, then the warp when all share a member
      const bool valid0 = e0 < cl.m;
      const u32 ms0 = valid0 ? gm[0] : 0xffffffffu;
      // members are sorted: the lane's edges share one if its first and last do
      const u32 qlast = valid0 ? min(3u, cl.m - 1 - e0) : 0u;
      u32 ms3 = ms0;
#pragma unroll
      for (int q = 1; q < 4; ++q)
        if ((u32)q == qlast) ms3 = gm[q];
      u32 mine = 0;
      bool split = ms3 != ms0;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (e0 + (u32)q < cl.m && cl_lab[q] != hl[q]) {
          if (!split) {
            ++mine;
          } else {
            atomicAdd(reinterpret_cast<unsigned long long*>(out + gm[q]), 1ull);
          }
        }
      const u32 act = __ballot_sync(0xffffffffu, valid0);
      if (act) {
        const u32 m0 = __shfl_sync(0xffffffffu, ms0, __ffs(act) - 1);
        const bool one = __all_sync(0xffffffffu, !valid0 || (!split && ms0 == m0));
        if (one) {
          u32 tot = mine;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
          if (lane == 0 && tot) atomicAdd(reinterpret_cast<unsigned long long*>(out + m0),
                                          (unsigned long long)tot);
        } else if (!split && mine) {
          atomicAdd(reinterpret_cast<unsigned long long*>(out + ms0), (unsigned long long)mine);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) cnt += e0 + (u32)q < cl.m && cl_lab[q] != hl[q];
    }
    h = nh;
    bg = nbg;
    bm = nbm;
  }
  if (!U) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kFull, cnt, o);
    if (lane == 0) wsum[tid >> 5] = cnt;
    __syncthreads();
    if (tid == 0) {
      unsigned long long tot = 0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += wsum[w];
      if (tot) atomicAdd(reinterpret_cast<unsigned long long*>(out), tot);
    }
  }
}

// blk_g and blk_mask of a union's concatenated groups (blk_mask zero on entry).
__global__ void k_cut_blocks(CutList cl) {
  for (u32 g = blockIdx.x * blockDim.x + threadIdx.x; g < cl.ngrp; g += gridDim.x * blockDim.x) {
    const u32 lo = cl.grp_off[g], hi = cl.grp_off[g + 1];
    if (lo & 31u) atomicOr(cl.blk_mask + (lo >> 5), 1u << (lo & 31u));
    for (u32 b = (lo + 31) / 32; b * 32 < hi; ++b) cl.blk_g[b] = g;
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

__global__ void k_cc_hook(const int2* __restrict__ up, u32 m_up, u32* parent) {
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < m_up; i += gridDim.x * blockDim.x) {
    const int2 e = up[i];
    cc_unite(parent, (u32)e.y, (u32)e.x);
  }
}

// Labelling from the CSR, after Afforest (Sutton, Ben-Nun, Barak 2018): every
// vertex is first linked to its r-th neighbour only (r = 0, 1), which joins
// nearly all of a large component; after compression the most common root c
// is found by sampling, and only the vertices outside c link their remaining
// arcs.  Every edge {v, w} with an end outside c is then linked from that end
// (the CSR holds both arcs), and edges inside c need nothing: the components
// are exact, with a fraction of the union-find work when one component holds
// most of the graph (R-MAT).
__global__ void k_cc_link_nth(const int* __restrict__ row_ptr, const int* __restrict__ col, u32 n,
                              int r, u32* parent) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int e = row_ptr[v] + r;
    if (e < row_ptr[v + 1]) {
      const u32 w = (u32)col[e];
      if (w < n && w != v) cc_unite(parent, v, w);
    }
  }
}

// Every vertex points straight at its root.  Only v's thread writes parent[v],
// and it writes the root, so concurrent walks through v stay valid.
__global__ void k_cc_compress(u32* parent, u32 n) {
  volatile u32* p = parent;
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    u32 r = p[v], nx;
    while ((nx = p[r]) != r) r = nx;
    p[v] = r;
  }
}

// The roots of `count` evenly spaced vertices, for the host to find the most
// common one.
__global__ void k_cc_sample(const u32* __restrict__ parent, u32 n, u32 count, u32* out) {
  const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = parent[(u32)((u64)i * n / count)];
}

// The arcs from the third on of every vertex outside component c: one lane per
// row of up to 32 arcs, the whole warp for a longer row.
__global__ void __launch_bounds__(256) k_cc_link_rest(const int* __restrict__ row_ptr,
                                                      const int* __restrict__ col, u32 n, u32 c,
                                                      u32* parent) {
  const u32 lane = threadIdx.x & 31;
  const u32 warps = gridDim.x * (blockDim.x / 32);
  for (u32 base = (blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * 32; base < n;
       base += warps * 32) {
    const u32 v = base + lane;
    int e0 = 0, e1 = 0;
    if (v < n) {
      e0 = row_ptr[v] + 2;
      e1 = row_ptr[v + 1];
      if (e0 < e1 && cc_root(parent, v) == c) e1 = e0;  // inside c: nothing to link
    }
    if (e1 - e0 <= 32)
      for (int e = e0; e < e1; ++e) {
        const u32 w = (u32)col[e];
        if (w < n && w != v) cc_unite(parent, v, w);
      }
    u32 lm = __ballot_sync(kFull, e1 - e0 > 32);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const u32 sv = __shfl_sync(kFull, v, src);
      const int b0 = __shfl_sync(kFull, e0, src), b1 = __shfl_sync(kFull, e1, src);
      for (int e = b0 + (int)lane; e < b1; e += 32) {
        const u32 w = (u32)col[e];
        if (w < n && w != sv) cc_unite(parent, sv, w);
      }
    }
  }
}

// Final labels and component sizes.  The walk only reads, and every store is
// a root, so concurrent walks stay valid.  Sizes are counted with one atomic
// per group of lanes that share a root; the vertices of component c (the
// common root, or ~0 for none) are counted per CTA, so that a giant
// component does not turn into millions of atomics on one address.
__global__ void __launch_bounds__(256) k_cc_finish(u32* parent, u32* csize, u32 n, u32 c) {
  __shared__ u32 s_c;
  if (threadIdx.x == 0) s_c = 0;
  __syncthreads();
  volatile u32* p = parent;
  const u32 lane = threadIdx.x & 31;
  const u32 stride = gridDim.x * blockDim.x;
  u32 in_c = 0;
  for (u32 base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
    const u32 v = base + lane;
    u32 r = 0xffffffffu;
    if (v < n) {
      r = v;
      u32 nx;
      while ((nx = p[r]) != r) r = nx;
      p[v] = r;
    }
    if (r == c && c != 0xffffffffu) {
      ++in_c;
      r = 0xffffffffu;
    }
    const u32 peers = __match_any_sync(kFull, r);
    if (r != 0xffffffffu && (int)lane == __ffs(peers) - 1) atomicAdd(csize + r, __popc(peers));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) in_c += __shfl_xor_sync(kFull, in_c, o);
  if (lane == 0 && in_c) atomicAdd(&s_c, in_c);
  __syncthreads();
  if (threadIdx.x == 0 && s_c) atomicAdd(csize + c, s_c);
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
// bit (no arcs, or a component of at most 32 vertices).  A warp owns whole
// words of the bitmasks (32 consecutive vertices), so it stores them without
// atomics, and it adds its BFS vertices and their arcs to the counters once.
__global__ void __launch_bounds__(256) k_small_members(const int* __restrict__ row_ptr,
                                                       const u32* __restrict__ parent,
                                                       const u32* __restrict__ csize,
                                                       const u32* __restrict__ root_off, u32 n,
                                                       u32* fill, u32* comp_v, u32* lane_of,
                                                       u32* excl, u32* solo, u32* counters) {
  const u32 lane = threadIdx.x & 31;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
    const u32 v = base + lane;
    bool is_solo = false, is_excl = false, bfs = false;
    u32 deg = 0;
    if (v < n) {
      const u32 r = parent[v];
      const u32 sz = csize[r];
      const bool small = sz <= kSmallComp;
      deg = (u32)(row_ptr[v + 1] - row_ptr[v]);
      if (small && sz >= 2) {
        const u32 pos = atomicAdd(fill + r, 1u);
        comp_v[root_off[r] + pos] = v;
        lane_of[v] = pos;
      }
      is_solo = sz == 1;
      is_excl = small || deg == 0;
      bfs = !is_excl;
    }
    const u32 solo_w = __ballot_sync(kFull, is_solo);
    const u32 excl_w = __ballot_sync(kFull, is_excl);
    const u32 nbfs = __popc(__ballot_sync(kFull, bfs));
    u32 arcs = bfs ? deg : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) arcs += __shfl_xor_sync(kFull, arcs, o);
    if (lane == 0) {
      solo[base >> 5] = solo_w;  // base is a multiple of 32: the warp owns the word
      excl[base >> 5] = excl_w;
      if (nbfs) {
        atomicAdd(counters + 2, nbfs);  // vertices the BFS settles
        atomicAdd(counters + 3, arcs);  // and their arcs
      }
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

// Largest value of x[0 .. n) (non-negative ints) into *out (zero on entry).
__global__ void __launch_bounds__(256) k_max_i32(const int* __restrict__ x, u32 n, u32* out) {
  u32 m = 0;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = max(m, (u32)max(x[i], 0));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// ---------------------------------------------------------------- residual graphs
// Blocks by repeated decomposition (Section 1's remark on Linial and Saks'
// block decompositions): after decomposing G_i, the arcs whose two ends
// share a piece form block i, and the others make up G_{i+1}.
//   * The count pass streams G_i's arcs with their source vertices (src, an
//     arc-aligned copy of the rows), kResIpt arcs per thread with all loads
//     first: a kept arc (v, w), centers different, adds one to kept[v] and
//     goes onto the kept list (its arc index, one reservation per warp); the
//     others get block i in arc_block (at their input arc id).  Rows of any
//     length cost the same, so hubs hold nobody up.
//   * After an exclusive scan of kept[] gives G_{i+1}'s row offsets (and a
//     copy of them as per-row cursors), the write pass takes the kept list
//     alone: each arc goes to its row's next place with its input arc id and
//     source, and each kept (v, w), v < w, is hooked into the union-find
//     forest of G_{i+1}'s components.  The order inside a row is free.
constexpr int kResIpt = 4;

struct ResArgs {
  const int* src;
  const int* col;
  const int* orig;       // input arc id of every arc (null: the arcs are the input's)
  const int* center;
  u32 n;
  u32 m;                 // arcs of G_i
  int block;
  int* arc_block;        // null: not recorded
  u32* kept;             // count pass: kept arcs per vertex
  unsigned long long* up_kept;
  u32* klist;            // count pass: the kept arcs' indices
  u32* n_kept;
  u32* cursor;           // write pass: next place of every row
  const u32* cid;        // write pass: every vertex's id in G_{i+1} (its rank among kept rows)
  int* new_col;
  int* new_orig;
  int* new_src;
  u32* parent;
};

__global__ void __launch_bounds__(256) k_residual_count(ResArgs a) {
  const u32 lane = threadIdx.x & 31;
  const u32 stride = gridDim.x * blockDim.x;
  u32 up = 0;
  // warp-uniform trip count: the kept-list reservation is a warp collective
  for (u32 b0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b0 < a.m; b0 += stride * kResIpt) {
    u32 v[kResIpt], w[kResIpt];
#pragma unroll
    for (int k = 0; k < kResIpt; ++k) {
      const u32 e = b0 + lane + (u32)k * stride;
      v[k] = e < a.m ? (u32)__ldcs(a.src + e) : 0xffffffffu;
      w[k] = e < a.m ? (u32)__ldcs(a.col + e) : 0xffffffffu;
    }
    int cv[kResIpt], cw[kResIpt];
#pragma unroll
    for (int k = 0; k < kResIpt; ++k) {
      cv[k] = v[k] < a.n ? __ldg(a.center + v[k]) : 0;
      cw[k] = w[k] < a.n ? __ldg(a.center + w[k]) : 0;
    }
#pragma unroll
    for (int k = 0; k < kResIpt; ++k) {
      const u32 e = b0 + lane + (u32)k * stride;
      const bool in = e < a.m && v[k] < a.n && w[k] < a.n;
      const bool keep = in && cv[k] != cw[k];
      if (in && !keep && a.arc_block) a.arc_block[a.orig ? __ldcs(a.orig + e) : (int)e] = a.block;
      const u32 km = __ballot_sync(kFull, keep);
      if (km) {  // kept arcs are few: one reservation per warp and step
        u32 at = 0;
        if (lane == (u32)(__ffs(km) - 1)) at = atomicAdd(a.n_kept, (u32)__popc(km));
        at = __shfl_sync(kFull, at, __ffs(km) - 1) + __popc(km & lanemask_lt());
        if (keep) {
          a.klist[at] = e;
          atomicAdd(a.kept + v[k], 1u);
          if (v[k] < w[k]) ++up;
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) up += __shfl_xor_sync(kFull, up, o);
  if (lane == 0 && up) atomicAdd(a.up_kept, (unsigned long long)up);
}

__global__ void __launch_bounds__(256) k_residual_write(ResArgs a) {
  const u32 nk = *a.n_kept;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < nk; i += gridDim.x * blockDim.x) {
    const u32 e = a.klist[i];
    const u32 v = (u32)a.src[e], w = (u32)a.col[e];
    const u32 at = atomicAdd(a.cursor + v, 1u);
    const u32 cv = a.cid[v], cw = a.cid[w];
    a.new_col[at] = (int)cw;
    a.new_orig[at] = a.orig ? a.orig[e] : (int)e;
    a.new_src[at] = (int)cv;
    if (cv < cw) cc_unite(a.parent, cw, cv);
  }
}

__global__ void __launch_bounds__(256) k_first_neighbours(const int* __restrict__ row_ptr,
                                                          const int* __restrict__ col, u32 n,
                                                          u32* first) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int e0 = row_ptr[v], e1 = row_ptr[v + 1];
    first[v] = e0 < e1 ? (u32)col[e0] : 0xffffffffu;
  }
}

// Compaction of G_{i+1} to the vertices that kept an arc.  off: the kept arcs'
// row offsets over G_i's n vertices (off[n] = all of them).
__global__ void __launch_bounds__(256) k_kept_flags(const int* __restrict__ off, u32 n,
                                                    u32* flag) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x)
    flag[v] = (v < n && off[v + 1] > off[v]) ? 1u : 0u;
}

// cid: exclusive scan of the flags (cid[n] = vertices of G_{i+1}).  Rows of
// G_{i+1} and its vertices' ids in the input graph.
__global__ void __launch_bounds__(256) k_compact_rows(const int* __restrict__ off,
                                                      const u32* __restrict__ cid, u32 n,
                                                      int* new_row, const u32* __restrict__ map,
                                                      u32* new_map) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
    if (v == n) {
      new_row[cid[n]] = off[n];
    } else if (off[v + 1] > off[v]) {
      const u32 c = cid[v];
      new_row[c] = off[v];
      new_map[c] = map ? map[v] : v;
    }
  }
}

// The shifts of G_{i+1}'s vertices, from the caller's vector over all n.
__global__ void __launch_bounds__(256) k_gather_shifts(const double* __restrict__ full,
                                                       const u32* __restrict__ map, u32 nc,
                                                       double* out) {
  for (u32 c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x)
    out[c] = full[map[c]];
}

// Every vertex alone (center itself, distance 0), then G_{i+1}'s results in
// the input graph's ids.
__global__ void __launch_bounds__(256) k_blocks_alone(u32 n, int* center, int* dist) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    center[v] = (int)v;
    dist[v] = 0;
  }
}
__global__ void __launch_bounds__(256) k_blocks_scatter(const int* __restrict__ cc,
                                                        const int* __restrict__ dc,
                                                        const u32* __restrict__ map, u32 nc,
                                                        int* center, int* dist) {
  for (u32 c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const u32 v = map[c];
    center[v] = (int)map[cc[c]];
    dist[v] = dc[c];
  }
}

// src[e] = v for every arc e of row v: a lane writes a row of up to 16 arcs,
// the whole warp a longer one (coalesced).
__global__ void __launch_bounds__(256) k_fill_src(const int* __restrict__ row, u32 n, int* src) {
  const u32 lane = threadIdx.x & 31;
  const u32 warps = gridDim.x * (blockDim.x / 32);
  for (u32 base = (blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * 32; base < n;
       base += warps * 32) {
    const u32 v = base + lane;
    int e0 = 0, e1 = 0;
    if (v < n) {
      e0 = row[v];
      e1 = row[v + 1];
    }
    if (e1 - e0 <= 16)
      for (int e = e0; e < e1; ++e) src[e] = (int)v;
    u32 lm = __ballot_sync(kFull, e1 - e0 > 16);
    while (lm) {
      const int sl = __ffs(lm) - 1;
      lm &= lm - 1;
      const int b0 = __shfl_sync(kFull, e0, sl), b1 = __shfl_sync(kFull, e1, sl);
      const int sv = (int)__shfl_sync(kFull, v, sl);
      for (int e = b0 + (int)lane; e < b1; e += 32) src[e] = sv;
    }
  }
}

// ---------------------------------------------------------------- fused cut counts
// The cut counts of two to four labelings of one graph (the decompositions of
// a pipelined batch) in one pass over the cut list.  The labelings are packed
// per vertex into one 16-byte word, lab4[v] = (c_0[v], .., c_3[v]) with unused
// slots 0, so that one gather per edge serves every labeling: the pass streams
// the cut list once instead of once per labeling, and makes as many L2 sector
// reads as a single count does.  The hot table's packed labels sit in shared
// memory up to kHot4Smem entries; the rest are read from global memory (hot
// vertices have many edges, so their lines stay cached).
constexpr u32 kHot4Smem = 12288;  // 192 KiB of packed labels per CTA

struct Labels4 {
  const int* c[4];
};

__global__ void __launch_bounds__(256) k_pack_labels(Labels4 L, int K, u32 n,
                                                     int4* __restrict__ lab4) {
  for (u32 v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int4 x;
    x.x = __ldg(L.c[0] + v);
    x.y = K > 1 ? __ldg(L.c[1] + v) : 0;
    x.z = K > 2 ? __ldg(L.c[2] + v) : 0;
    x.w = K > 3 ? __ldg(L.c[3] + v) : 0;
    lab4[v] = x;
  }
}

// out[i] = lab4[idx[i]]: the packed labels of the hot table or of every
// group's cold vertex; four gathers per thread in flight.
__global__ void __launch_bounds__(256) k_gather_labels4(const u32* __restrict__ idx, u32 cnt,
                                                        const int4* __restrict__ lab4,
                                                        int4* __restrict__ out) {
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < cnt; i0 += stride * kLabIpt) {
    int4 x[kLabIpt];
#pragma unroll
    for (int q = 0; q < kLabIpt; ++q) {
      const u32 i = i0 + (u32)q * stride;
      x[q] = i < cnt ? __ldg(lab4 + __ldg(idx + i)) : make_int4(0, 0, 0, 0);
    }
#pragma unroll
    for (int q = 0; q < kLabIpt; ++q) {
      const u32 i = i0 + (u32)q * stride;
      if (i < cnt) out[i] = x[q];
    }
  }
}

// k_cut's pass with packed labels: every edge compares the packed labels of
// its two endpoints and adds one to each labeling's count that differs.
// out[0 .. K) receive the counts (added).
__global__ void __launch_bounds__(kCutThreads, 1) k_cut4(CutList cl, const int4* __restrict__ lab4,
                                                         const int4* __restrict__ grp4,
                                                         const int4* __restrict__ hot4,
                                                         u32 n_hot, int K, u64* out) {
  extern __shared__ int4 cut_smem[];
  __shared__ unsigned long long wsum[kCutThreads / 32][4];
  const u32 tid = threadIdx.x, lane = tid & 31;
  const u32 nsm = min(n_hot, kHot4Smem);
  for (u32 i = tid; i < nsm; i += blockDim.x) cut_smem[i] = __ldg(hot4 + i);
  __syncthreads();
  const int4* hotv4 = reinterpret_cast<const int4*>(cl.hot);  // cudaMalloc'd: aligned
  const u32 nchunk = (cl.m + 127) / 128;                        // 128 edges per warp step
  const u32 stride = gridDim.x * (kCutThreads / 32);
  u32 cnt[4] = {0, 0, 0, 0};
  u32 c = blockIdx.x * (kCutThreads / 32) + (tid >> 5);
  // lane's four edges: 4 lane .. 4 lane + 3 of the chunk, in block lane / 8
  auto load = [&](u32 cc, int4& h, u32& bg, u32& bm) {
    const u32 e0 = cc * 128 + 4 * lane;
    if (e0 + 3 < cl.m) {
      h = __ldcs(hotv4 + (e0 >> 2));
    } else {
      h.x = e0 < cl.m ? cl.hot[e0] : 0;
      h.y = e0 + 1 < cl.m ? cl.hot[e0 + 1] : 0;
      h.z = e0 + 2 < cl.m ? cl.hot[e0 + 2] : 0;
      h.w = 0;
    }
    const u32 b = e0 >> 5;
    bg = b < cl.nblk ? __ldg(cl.blk_g + b) : 0u;
    bm = b < cl.nblk ? __ldg(cl.blk_mask + b) : 0u;
  };
  int4 h;
  u32 bg = 0, bm = 0;
  if (c < nchunk) load(c, h, bg, bm);
  for (; c < nchunk; c += stride) {
    int4 nh = make_int4(0, 0, 0, 0);
    u32 nbg = 0, nbm = 0;
    if (c + stride < nchunk) load(c + stride, nh, nbg, nbm);
    const u32 e0 = c * 128 + 4 * lane, j0 = (4 * lane) & 31u;
    const int hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (e0 + (u32)q >= cl.m) break;
      const u32 g = bg + __popc(bm & bits_upto(j0 + (u32)q));
      const int4 a = __ldg(grp4 + g);
      int4 b;
      if (hv[q] >= 0) {
        b = __ldg(lab4 + hv[q]);
      } else {
        const u32 i = (u32)hv[q] & 0x7fffffffu;
        b = i < nsm ? cut_smem[i] : __ldg(hot4 + i);
      }
      cnt[0] += a.x != b.x;
      cnt[1] += a.y != b.y;
      cnt[2] += a.z != b.z;
      cnt[3] += a.w != b.w;
    }
    h = nh;
    bg = nbg;
    bm = nbm;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    unsigned long long t = cnt[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFull, t, o);
    if (lane == 0) wsum[tid >> 5][k] = t;
  }
  __syncthreads();
  if (tid < (u32)K) {
    unsigned long long tot = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += wsum[w][tid];
    if (tot) atomicAdd(reinterpret_cast<unsigned long long*>(out + tid), tot);
  }
}

u32 grid_for(u32 n, int num_sms) {
  return (u32)max(1ll, min((long long)(n + 255) / 256, (long long)num_sms * 8));
}

}  // namespace

int launch_finalize(const u64* key, const u32* order, const u32* solo, u32 n, int* center,
                    int* dist, const u32* err, int num_sms, cudaStream_t s) {
  k_finalize<<<grid_for((n + kFinIpt - 1) / kFinIpt, num_sms), 256, 0, s>>>(key, order, solo, n,
                                                                         center, dist, err);
  return 1;
}

int launch_cut(const CutList& cl, const int* center, const u32* hot, u32 n_hot, int* hot_center,
               u64* out, int num_sms, cudaStream_t s) {
  if (cl.m == 0) return 0;
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaFuncSetAttribute(k_cut<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kHotSlots * sizeof(int)));
    attr_set[dev] = true;
  }
  int launches = 1;
  if (n_hot > 0) {
    k_hot_centers<<<(n_hot + 255) / 256, 256, 0, s>>>(hot, n_hot, center, hot_center);
    ++launches;
  }
  k_group_labels<false><<<grid_for((cl.ngrp + kLabIpt - 1) / kLabIpt, num_sms), 256, 0, s>>>(
      cl, center);
  const u32 g = (u32)max(1ll, min((long long)(cl.m + 4095) / 4096, (long long)num_sms));
  k_cut<false><<<g, kCutThreads, (size_t)n_hot * sizeof(int), s>>>(cl, center, hot_center, n_hot,
                                                                   out);
  return launches + 1;
}

int launch_cut4(const CutList& cl, const int* const* centers, int K, u32 n, const u32* hot,
                u32 n_hot, int4* lab4, int4* hot4, int4* grp4, u64* out, int num_sms,
                cudaStream_t s) {
  if (cl.m == 0 || K < 1 || K > 4) return 0;
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaFuncSetAttribute(k_cut4, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kHot4Smem * sizeof(int4)));
    attr_set[dev] = true;
  }
  Labels4 L = {{centers[0], K > 1 ? centers[1] : nullptr, K > 2 ? centers[2] : nullptr,
                K > 3 ? centers[3] : nullptr}};
  k_pack_labels<<<grid_for(n, num_sms), 256, 0, s>>>(L, K, n, lab4);
  int launches = 1;
  if (n_hot > 0) {
    k_gather_labels4<<<grid_for((n_hot + kLabIpt - 1) / kLabIpt, num_sms), 256, 0, s>>>(
        hot, n_hot, lab4, hot4);
    ++launches;
  }
  k_gather_labels4<<<grid_for((cl.ngrp + kLabIpt - 1) / kLabIpt, num_sms), 256, 0, s>>>(
      cl.grp_v, cl.ngrp, lab4, grp4);
  const u32 g = (u32)max(1ll, min((long long)(cl.m + 4095) / 4096, (long long)num_sms));
  k_cut4<<<g, kCutThreads, (size_t)min(n_hot, kHot4Smem) * sizeof(int4), s>>>(cl, lab4, grp4,
                                                                            hot4, n_hot, K, out);
  return launches + 2;
}

int launch_union_cut(const CutList& cl, const UnionOffsets& off, const u32* wmem,
                     const int* center, u64* cut, int num_sms, cudaStream_t s) {
  (void)off;
  (void)wmem;
  if (cl.m == 0) return 0;
  k_group_labels<true><<<grid_for((cl.ngrp + kLabIpt - 1) / kLabIpt, num_sms), 256, 0, s>>>(
      cl, center);
  const u32 g = (u32)max(1ll, min((long long)(cl.m + 4095) / 4096, (long long)num_sms));
  k_cut<true><<<g, kCutThreads, 0, s>>>(cl, center, nullptr, 0, cut);
  return 2;
}

int launch_cut_blocks(const CutList& cl, int num_sms, cudaStream_t s) {
  cudaMemsetAsync(cl.blk_mask, 0, (size_t)cl.nblk * 4, s);
  k_cut_blocks<<<grid_for(cl.ngrp ? cl.ngrp : 1, num_sms), 256, 0, s>>>(cl);
  return 1;
}

int launch_max_dist(const int* dist, u32 n, u32* out, int num_sms, cudaStream_t s) {
  cudaMemsetAsync(out, 0, sizeof(u32), s);
  k_max_i32<<<grid_for(n, num_sms), 256, 0, s>>>(dist, n, out);
  return 1;
}

int launch_small_comp(const SmallComps& sc, u64* key, const u32* err, int num_sms, cudaStream_t s) {
  if (sc.ncomp == 0) return 0;
  const u32 blocks = (u32)min((long long)(sc.ncomp + 7) / 8, (long long)num_sms * 8);
  k_small_comp<<<blocks, 256, 0, s>>>(sc.comp_off, sc.comp_len, sc.ncomp, sc.comp_v, sc.adj, key,
                                      err);
  return 1;
}

cudaError_t components_init(u32 n, int num_sms, const CompScratch& t, u32* excl, u32* solo,
                            cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(t.csize, 0, (size_t)n * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(t.fill, 0, (size_t)n * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(t.counters, 0, 4 * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(t.lane_of, 0xff, (size_t)n * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(excl, 0, ((size_t)n + 31) / 32 * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(solo, 0, ((size_t)n + 31) / 32 * 4, s)) != cudaSuccess) return e;
  k_iota<<<grid_for(n, num_sms), 256, 0, s>>>(t.parent, n);
  return cudaGetLastError();
}

cudaError_t components_phase1(const int* row_ptr, const int2* up, u32 m_up, u32 n, int num_sms,
                              const CompScratch& t, u32* excl, u32* solo, u32 counts[4],
                              cudaStream_t s) {
  cudaError_t e = components_init(n, num_sms, t, excl, solo, s);
  if (e != cudaSuccess) return e;
  if (m_up > 0) k_cc_hook<<<grid_for(m_up, num_sms), 256, 0, s>>>(up, m_up, t.parent);
  return components_label(row_ptr, n, num_sms, t, excl, solo, counts, s);
}

cudaError_t components_from_csr(const int* row_ptr, const int* col, u32 n, int num_sms,
                                const CompScratch& t, u32* excl, u32* solo, u32 counts[4],
                                cudaStream_t s) {
  cudaError_t e = components_init(n, num_sms, t, excl, solo, s);
  if (e != cudaSuccess) return e;
  const u32 g = grid_for(n, num_sms);
  for (int r = 0; r < 2; ++r) k_cc_link_nth<<<g, 256, 0, s>>>(row_ptr, col, n, r, t.parent);
  k_cc_compress<<<g, 256, 0, s>>>(t.parent, n);
  // the most common root of an even sample (root_off serves as the buffer; it
  // is written later by k_small_roots)
  const u32 count = min(n, 1024u);
  k_cc_sample<<<(count + 255) / 256, 256, 0, s>>>(t.parent, n, count, t.root_off);
  u32 roots[1024];
  if ((e = cudaMemcpyAsync(roots, t.root_off, count * 4, cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  std::sort(roots, roots + count);
  u32 c = roots[0], best = 0;
  for (u32 i = 0; i < count;) {
    u32 j = i;
    while (j < count && roots[j] == roots[i]) ++j;
    if (j - i > best) {
      best = j - i;
      c = roots[i];
    }
    i = j;
  }
  k_cc_link_rest<<<g, 256, 0, s>>>(row_ptr, col, n, c, t.parent);
  return components_label(row_ptr, n, num_sms, t, excl, solo, counts, s, c);
}

cudaError_t components_label(const int* row_ptr, u32 n, int num_sms, const CompScratch& t,
                             u32* excl, u32* solo, u32 counts[4], cudaStream_t s, u32 common) {
  const u32 g = grid_for(n, num_sms);
  cudaError_t e;
  k_cc_finish<<<g, 256, 0, s>>>(t.parent, t.csize, n, common);
  k_small_roots<<<g, 256, 0, s>>>(t.parent, t.csize, n, t.root_off, t.comp_off, t.comp_len,
                                  t.counters);
  k_small_members<<<g, 256, 0, s>>>(row_ptr, t.parent, t.csize, t.root_off, n, t.fill, t.comp_v,
                                    t.lane_of, excl, solo, t.counters);
  if ((e = cudaMemcpyAsync(counts, t.counters, 4 * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

int launch_residual(bool write, const int* src, const int* col, const int* orig,
                    const int* center, u32 n, u32 m, int block, int* arc_block, u32* kept,
                    unsigned long long* up_kept, u32* klist, u32* n_kept, u32* cursor,
                    const u32* cid, int* new_col, int* new_orig, int* new_src, u32* parent,
                    int num_sms, cudaStream_t s) {
  ResArgs a{src,     col,    orig,   center, n,   m,       block,    arc_block, kept,  up_kept,
            klist,   n_kept, cursor, cid,    new_col, new_orig, new_src, parent};
  if (write) {
    k_residual_write<<<num_sms * 4, 256, 0, s>>>(a);
  } else {
    if (m == 0) return 0;
    const u32 blocks = (u32)max(1ll, min(((long long)m + 256 * kResIpt - 1) / (256 * kResIpt),
                                         (long long)num_sms * 8));
    k_residual_count<<<blocks, 256, 0, s>>>(a);
  }
  return 1;
}

int launch_kept_flags(const int* off, u32 n, u32* flag, int num_sms, cudaStream_t s) {
  k_kept_flags<<<grid_for(n + 1, num_sms), 256, 0, s>>>(off, n, flag);
  return 1;
}

int launch_compact_rows(const int* off, const u32* cid, u32 n, int* new_row, const u32* map,
                        u32* new_map, int num_sms, cudaStream_t s) {
  k_compact_rows<<<grid_for(n + 1, num_sms), 256, 0, s>>>(off, cid, n, new_row, map, new_map);
  return 1;
}

int launch_gather_shifts(const double* full, const u32* map, u32 nc, double* out, int num_sms,
                         cudaStream_t s) {
  if (nc == 0) return 0;
  k_gather_shifts<<<grid_for(nc, num_sms), 256, 0, s>>>(full, map, nc, out);
  return 1;
}

int launch_blocks_output(const int* cc, const int* dc, const u32* map, u32 nc, u32 n, int* center,
                         int* dist, int num_sms, cudaStream_t s) {
  k_blocks_alone<<<grid_for(n, num_sms), 256, 0, s>>>(n, center, dist);
  if (nc > 0) k_blocks_scatter<<<grid_for(nc, num_sms), 256, 0, s>>>(cc, dc, map, nc, center, dist);
  return 2;
}

int launch_first_neighbours(const int* row_ptr, const int* col, u32 n, u32* first, int num_sms,
                            cudaStream_t s) {
  if (n == 0) return 0;
  k_first_neighbours<<<grid_for(n, num_sms), 256, 0, s>>>(row_ptr, col, n, first);
  return 1;
}

int launch_fill_src(const int* row, u32 n, int* src, int num_sms, cudaStream_t s) {
  if (n == 0) return 0;
  k_fill_src<<<grid_for(n, num_sms), 256, 0, s>>>(row, n, src);
  return 1;
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

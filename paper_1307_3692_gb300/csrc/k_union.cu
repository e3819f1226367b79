// Batches as disjoint unions (Miller, Peng, Xu 2013, Algorithm 2).
//
// Algorithm 2 assigns every vertex to the argmin over u of dist(u, v) - delta_u,
// and a vertex of another graph is at infinite distance.  So the decomposition
// of a disjoint union G_0 + G_1 + ... with the concatenated shifts is, member
// by member, the decomposition of each G_s with its own shifts: the integer
// levels of one member all move by the same constant (floor(delta_max) of the
// union instead of the member's), and the fraction ranks of one member keep
// their relative order (union ids preserve the members' id order).  A batch
// of graphs -- or of shift vectors of one graph -- therefore runs as one
// decomposition: one persistent BFS whose frontier holds every member's
// frontier, one rank, one finalize.
//
// Layout of the union.  Member s occupies union vertices
// [voff_s, voff_s + n_s) followed by pad_s = roundup(n_s, 32) - n_s isolated
// pad vertices, so that every member starts on a 32-vertex boundary and its
// per-vertex bitmask words are copied whole.  Arcs, cut-list edges and groups
// and small-component records are concatenated in member order with their
// vertex ids moved by voff_s.  The union's cut list has no hot table and
// holds caller-layout indices (the cut count reads the outputs).  Outputs use the caller's layout: member s's n_s
// entries at ooff_s = n_0 + ... + n_{s-1}, with member-local ids.
//
// Every table is built by one launch (k_union_concat, blockIdx.y = table);
// a block finds the member of its chunk's first element by a binary search
// over the table's member offsets, and its threads walk forward from there.
//
// Level alignment.  With one floor(delta_max) for the whole union, a member
// whose own largest shift is small would start late, and until then its
// unsettled vertices would sit in every bottom-up scan.  Each call therefore
// lifts member s's floors by max_t A_t - A_s, A_s the largest floor among
// the member's vertices that the round loop handles (k_union_spread,
// k_union_lift; applied by the rank's split), so that every member's first
// start is at round 0 and the members' frontiers grow and shrink together.
#include "ldd_internal.cuh"

namespace ldd {

namespace {

// Member s of off[0 .. k]: the last s with off[s] <= x (x < off[k]).  With
// empty members (equal offsets) this is the non-empty one holding x.
__device__ __forceinline__ u32 member_of(const u32* __restrict__ off, u32 k, u32 x) {
  u32 lo = 0, hi = k;  // off[lo] <= x < off[hi]
  while (hi - lo > 1) {
    const u32 mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Calls f(x, s) for every x in [0, X) with s = member_of(off, k, x * scale).  A block
// takes kConcatChunk consecutive elements at a time and finds the member of
// the first one once; each thread then walks forward from it (members are
// contiguous and ordered, and a thread's x only grows).
constexpr u32 kConcatChunk = 2048;

template <typename F>
__device__ __forceinline__ void for_each_member_elem(const u32* __restrict__ off, u32 k, u32 X,
                                                     F f, u32 scale = 1) {
  __shared__ u32 s_first;
  for (u32 base = blockIdx.x * kConcatChunk; base < X; base += gridDim.x * kConcatChunk) {
    __syncthreads();
    if (threadIdx.x == 0) s_first = member_of(off, k, base * scale);
    __syncthreads();
    u32 s = s_first;
    const u32 end = min(base + kConcatChunk, X);
    for (u32 x = base + threadIdx.x; x < end; x += blockDim.x) {
      while (__ldg(off + s + 1) <= x * scale) ++s;
      f(x, s);
    }
  }
}

__global__ void __launch_bounds__(256) k_union_concat(const UnionMember* __restrict__ mem,
                                                      UnionOffsets off, u32 k, UnionTables t) {
  switch (blockIdx.y) {
    case 0: {  // row_ptr: member rows moved by eoff; pads are empty rows
      const u32 N = off.v[k];
      if (blockIdx.x == 0 && threadIdx.x == 0) t.row[N] = (int)off.e[k];
      for_each_member_elem(off.v, k, N, [&](u32 u, u32 s) {
        const UnionMember& m = mem[s];
        const u32 v = u - off.v[s];
        t.row[u] = (int)(off.e[s] + (v < m.n ? (u32)__ldg(m.row + v) : m.nnz));
      });
      break;
    }
    case 1:  // col: neighbour ids moved by voff
      for_each_member_elem(off.e, k, off.e[k], [&](u32 e, u32 s) {
        t.col[e] = __ldg(mem[s].col + (e - off.e[s])) + (int)off.v[s];
      });
      break;
    case 2:  // cut list edges: hot-table slots resolved, ids moved to the caller layout
      for_each_member_elem(off.u, k, off.u[k], [&](u32 i, u32 s) {
        const UnionMember& m = mem[s];
        const int h = __ldg(m.cut_hot + (i - off.u[s]));
        const int hot = h < 0 ? (int)__ldg(m.hot + (h & 0x7fffffff)) : h;
        t.cut.hot[i] = hot + (int)off.o[s];  // caller layout: the cut reads outputs
      });
      break;
    case 8: {  // cut list groups: cold vertices (caller layout), members, edge offsets
      const u32 G = off.g[k];
      if (blockIdx.x == 0 && threadIdx.x == 0) t.cut.grp_off[G] = off.u[k];
      for_each_member_elem(off.g, k, G, [&](u32 i, u32 s) {
        const UnionMember& m = mem[s];
        t.cut.grp_v[i] = __ldg(m.grp_v + (i - off.g[s])) + off.o[s];
        t.cut.grp_m[i] = s;
        t.cut.grp_off[i] = __ldg(m.grp_off + (i - off.g[s])) + off.u[s];
      });
      break;
    }
    case 3:  // exclusion and singleton bitmasks: whole words, pad bits set
    case 7:  // and the member of every 32-vertex word (the rank's floor lift)
      for_each_member_elem(off.v, k, off.v[k] / 32, [&](u32 w, u32 s) {
        if (blockIdx.y == 7) {
          t.wmem[w] = s;
          return;
        }
        const UnionMember& m = mem[s];
        const u32 lw = w - off.v[s] / 32;
        const u32 lo = lw * 32;  // first local vertex of the word
        const u32 pad = lo + 32 <= m.n ? 0u : (lo >= m.n ? 0xffffffffu : ~0u << (m.n - lo));
        const u32 ex = lo < m.n ? __ldg(m.excl + lw) : 0u;
        const u32 so = lo < m.n ? __ldg(m.solo + lw) : 0u;
        t.excl[w] = ex | pad;
        t.solo[w] = so | pad;
      }, 32u);
      break;
    case 4:  // small components: member ranges and sizes
      for_each_member_elem(off.c, k, off.c[k], [&](u32 c, u32 s) {
        const UnionMember& m = mem[s];
        t.comp_off[c] = __ldg(m.comp_off + (c - off.c[s])) + off.m[s];
        t.comp_len[c] = __ldg(m.comp_len + (c - off.c[s]));
      });
      break;
    case 5:  // small components: member lists and lane adjacency masks
      for_each_member_elem(off.m, k, off.m[k], [&](u32 i, u32 s) {
        const UnionMember& m = mem[s];
        t.comp_v[i] = __ldg(m.comp_v + (i - off.m[s])) + off.v[s];
        t.adj[i] = __ldg(m.adj + (i - off.m[s]));
      });
      break;
    case 6:  // vertices the BFS handles, ascending (when every member lists them)
      if (!t.active) break;
      for_each_member_elem(off.a, k, off.a[k], [&](u32 i, u32 s) {
        t.active[i] = __ldg(mem[s].active + (i - off.a[s])) + off.v[s];
      });
      break;
    default: break;
  }
}

// floor(d) of a valid shift (finite, 0 <= d < 2^31), from the bits of d; 0
// for anything else (the rank's split rejects those shifts).
__device__ __forceinline__ int floor_of(double d) {
  const u64 b = (u64)__double_as_longlong(d);
  const u32 ex = (u32)(b >> 52) & 0x7ffu;
  if ((b >> 63) || ex < 1023u || ex >= 1023u + 31u) return 0;
  const u64 M = (b & ((1ull << 52) - 1)) | (1ull << 52);
  return (int)(M >> (52 - (ex - 1023u)));
}

// Concatenated input shifts (caller layout) to the union layout (pads get 0),
// and into amax[s] (zero on entry) the largest floor among member s's vertices
// that the round loop handles (excl bit clear): isolated vertices and small
// components never enter the rounds, so they must not set the alignment.  A
// warp's 32 consecutive union vertices belong to one member (members start on
// 32-vertex boundaries) and share one excl word, so each warp step ends in
// one atomicMax.
// Members are padded to multiples of 32 vertices, so every 32-vertex chunk
// of the union belongs to one member.  A warp takes kSpreadIpt consecutive
// chunks at a time, finds the member of the first once and walks forward for
// the others, and issues all their loads before any store.
constexpr int kSpreadIpt = 4;

__global__ void __launch_bounds__(256) k_union_spread(const double* __restrict__ in,
                                                      UnionOffsets off, u32 k,
                                                      const u32* __restrict__ excl,
                                                      double* __restrict__ out, int* amax) {
  const u32 N = off.v[k];
  const u32 lane = threadIdx.x & 31;
  const u32 span = 32u * kSpreadIpt;
  const u32 nwarps = gridDim.x * (blockDim.x / 32);
  for (u32 wb0 = (blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * span; wb0 < N;
       wb0 += nwarps * span) {
    u32 sm[kSpreadIpt];
    double d[kSpreadIpt];
    u32 m = member_of(off.v, k, wb0);
#pragma unroll
    for (int q = 0; q < kSpreadIpt; ++q) {
      const u32 wb = wb0 + (u32)q * 32;
      if (wb < N)
        while (__ldg(off.v + m + 1) <= wb) ++m;
      sm[q] = m;
      const u32 v = wb + lane - off.v[m];
      const u32 n = off.o[m + 1] - off.o[m];
      d[q] = (wb < N && v < n) ? __ldcs(in + off.o[m] + v) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kSpreadIpt; ++q) {
      const u32 wb = wb0 + (u32)q * 32;
      if (wb >= N) break;  // warp-uniform
      out[wb + lane] = d[q];
      int a = ((__ldg(excl + (wb >> 5)) >> lane) & 1u) ? 0 : floor_of(d[q]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
      if (lane == 0 && a > 0) atomicMax(amax + sm[q], a);
    }
  }
}

// lift[s] = max_t amax[t] - amax[s]: every member's largest shift then starts
// the round loop at round 0.  One CTA.
__global__ void __launch_bounds__(1024) k_union_lift(const int* __restrict__ amax, u32 k,
                                                     int* __restrict__ lift) {
  __shared__ int wmax[32];
  __shared__ int gmax;
  int m = 0;
  for (u32 s = threadIdx.x; s < k; s += blockDim.x) m = max(m, amax[s]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    int g = 0;
    for (u32 w = 0; w < blockDim.x / 32; ++w) g = max(g, wmax[w]);
    gmax = g;
  }
  __syncthreads();
  for (u32 s = threadIdx.x; s < k; s += blockDim.x) lift[s] = gmax - amax[s];
}

// Algorithm 1 step 4 in the caller's layout: output i is vertex v of member
// s, union vertex u = voff_s + v.  Its settled key names the center
// order[rank] (a union id of the same member); the member-local center id is
// that minus voff_s, and the hop distance is the key's level minus the
// center's own level.
// A warp takes 32 x kUFinIpt consecutive caller-layout entries at a time,
// finds the member of the first once and walks forward from it per entry;
// the loads of a lane's entries go out level by level (own keys, centers,
// centers' keys), so that their dependent gathers overlap.
constexpr int kUFinIpt = 4;

__global__ void __launch_bounds__(256) k_union_finalize(const u64* __restrict__ key,
                                                        const u32* __restrict__ order,
                                                        const u32* __restrict__ solo,
                                                        UnionOffsets off, u32 k,
                                                        int* __restrict__ center,
                                                        int* __restrict__ dist, const u32* err) {
  if (*(volatile const u32*)err != 0u) return;
  const u32 total = off.o[k], N = off.v[k];
  const u32 lane = threadIdx.x & 31;
  const u32 span = 32u * kUFinIpt;
  const u32 nwarps = gridDim.x * (blockDim.x / 32);
  for (u32 wbase = (blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) * span; wbase < total;
       wbase += nwarps * span) {
    const u32 s0 = member_of(off.o, k, wbase);
    u32 idx[kUFinIpt], sm[kUFinIpt], u[kUFinIpt], c[kUFinIpt];
    bool live[kUFinIpt], alone[kUFinIpt];
    u64 kv[kUFinIpt], kc[kUFinIpt];
#pragma unroll
    for (int q = 0; q < kUFinIpt; ++q) {
      idx[q] = wbase + (u32)q * 32 + lane;
      live[q] = idx[q] < total;
      u32 m = s0;
      if (live[q])
        while (__ldg(off.o + m + 1) <= idx[q]) ++m;
      sm[q] = m;
      u[q] = live[q] ? off.v[m] + (idx[q] - off.o[m]) : 0u;
      alone[q] = live[q] && ((__ldg(solo + (u[q] >> 5)) >> (u[q] & 31)) & 1u);
      kv[q] = (live[q] && !alone[q]) ? key[u[q]] : 0ull;
    }
#pragma unroll
    for (int q = 0; q < kUFinIpt; ++q)
      c[q] = (live[q] && !alone[q]) ? order[min((u32)kv[q], N - 1)] : u[q];
#pragma unroll
    for (int q = 0; q < kUFinIpt; ++q)
      kc[q] = (live[q] && !alone[q]) ? key[c[q]] : kv[q];
#pragma unroll
    for (int q = 0; q < kUFinIpt; ++q)
      if (live[q]) {
        center[idx[q]] = (int)(c[q] - off.v[sm[q]]);
        dist[idx[q]] = alone[q] ? 0 : (int)((u32)(kv[q] >> 32) - (u32)(kc[q] >> 32));
      }
  }
}

u32 blocks_for(u64 n, int num_sms) {
  return (u32)max(1ll, min((long long)((n + 255) / 256), (long long)num_sms * 8));
}

}  // namespace

int launch_union_concat(const UnionMember* mem, const UnionOffsets& off, u32 k,
                        const UnionTables& t, u64 largest, int num_sms, cudaStream_t s) {
  const u32 bx = (u32)max(1ll, min((long long)((largest + kConcatChunk - 1) / kConcatChunk),
                                   (long long)num_sms * 8));
  k_union_concat<<<dim3(bx, 9), 256, 0, s>>>(mem, off, k, t);
  launch_cut_blocks(t.cut, num_sms, s);  // after the groups are in place
  return 2;
}

int launch_union_spread(const double* in, const UnionOffsets& off, u32 k, u32 N,
                        const u32* excl, double* out, int* amax, int* lift, int num_sms,
                        cudaStream_t s) {
  cudaMemsetAsync(amax, 0, (size_t)k * sizeof(int), s);
  k_union_spread<<<blocks_for((N + kSpreadIpt - 1) / kSpreadIpt, num_sms), 256, 0, s>>>(
      in, off, k, excl, out, amax);
  k_union_lift<<<1, 1024, 0, s>>>(amax, k, lift);
  return 2;
}

int launch_union_finalize(const u64* key, const u32* order, const u32* solo,
                          const UnionOffsets& off, u32 k, u32 total, int* center, int* dist,
                          const u32* err, int num_sms, cudaStream_t s) {
  k_union_finalize<<<blocks_for((total + kUFinIpt - 1) / kUFinIpt, num_sms), 256, 0, s>>>(
      key, order, solo, off, k, center, dist, err);
  return 1;
}

}  // namespace ldd

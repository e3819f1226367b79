// Round-synchronous, delayed-start multi-source BFS (Algorithm 1 step 3;
// Section 4 of Miller, Peng, Xu 2013), as one persistent cooperative kernel.
//
// State: key[v] = (level << 32) | rank, initialised to v's own start label
// (level R_v = floor(delta_max) - floor(delta_v)).  Round r expands the
// frontier F_r = {v : final level of v is r}: every arc (v, w) offers
// key[v] + 2^32 to w with a 64-bit atomicMin.  Because key[v] is final once
// round r - 1 has finished, and an offer made in round r carries level r + 1,
// the minimum over all offers is the exact label the paper's super-source
// shortest path assigns (Section 4), including the fraction tie-break.
//
// F_{r+1} is built during round r from two disjoint sources:
//   * pushes: the one atomicMin that lowers w's level from > r + 1 to r + 1
//     appends w (its return value identifies it uniquely);
//   * delayed starts (Section 4: the super-source edge of length L is used
//     when the frontier reaches L): vertices of start bucket r + 1 whose key
//     still has level r + 1.  A push in round r can only lower their rank
//     part, so this test is stable while round r runs.
// Appends are warp-aggregated: one 64-bit atomicAdd per warp reserves
// (items << 32 | edges), giving every appended vertex its queue slot and the
// exclusive edge offset of its adjacency list in the next frontier.  The next
// round then splits the frontier's edges into equal spans, one per CTA step,
// whatever the degree skew: a CTA loads the window of queue items that cover
// its span into shared memory and finds each edge's item with a block-wide
// max-scan.
//
// Direction-optimising rounds (Beamer, Asanovic, Patterson 2012): when the
// frontier's arcs outweigh the arcs of the still-unsettled vertices, a round
// runs bottom-up instead: every unsettled vertex w scans its neighbours for
// keys of level r and keeps the smallest key + 2^32.  The scan can stop once it
// holds (r + 1, minrank_r), where minrank_r is the smallest rank among level-r
// keys: nothing can beat it.  minrank_r is tracked exactly during round r - 1
// as the minimum over every successful key update and every appended start
// (each final level-r key is one of these, and each of these is >= the final
// key of its vertex).  Only w's own thread writes key[w] in such a round, and a
// vertex being lowered to level r + 1 is never read as a level-r key, so no
// atomics are needed.  On a union of graphs (k_union.cu) the floor is per
// member: the smallest level-r rank of w's own member, since no other member's
// key can reach w; it is computed when a round goes bottom-up, by one pass
// over the frontier list (every level-r vertex is on it) and one more grid
// barrier.  The first bottom-up round of a run examines every
// vertex the BFS owns; each round lists the vertices still above level r + 1,
// and the next bottom-up round examines only those.
//
// Rounds with an empty frontier jump straight to the next non-empty start
// bucket; the loop stops as soon as every vertex with an arc is settled.
// Graphs whose vertices have at most kLdMaxDegree arcs run low-degree rounds
// (a plain vertex list, a thread per frontier vertex), and a single such graph
// relaxes up to eight levels between two grid barriers (windows of levels,
// below).  All device-side waits are bounded: a barrier that does not complete
// within the spin limit sets kErrTimeout and the kernel returns.
#include <cstddef>

#include "ldd_internal.cuh"

namespace ldd {

namespace {

constexpr u32 kFull = 0xffffffffu;
constexpr int kEdgeBatch = 4;  // arcs per thread in flight
constexpr int kWinBatch = 3;   // window items per thread in flight
// candidates per lane in flight in a bottom-up round: three with one CTA per
// SM (up to 128 registers), two with two CTAs per SM (64 registers: more
// would spill); measured on R-MAT 22 (0.132 ms against 0.140 with two, 0.137
// with four) and on 64 R-MAT 20 copies as a union (3.4 ms against 4.0 with
// three)
constexpr int pull_width(int per_sm) { return per_sm >= 2 ? 2 : 3; }
constexpr int kPullLong = 32;  // longer adjacency lists are scanned by the whole warp
constexpr int kPullCoop = 4;   // neighbours per lane per step of a warp-wide scan
// Unions of at most this many members keep their per-member floors in shared
// memory (two tables after Smem); larger unions use the global table directly.
constexpr u32 kSmemMembers = 4096;
constexpr int kLdBatch = 8;    // low-degree rounds: arcs per frontier vertex and step
constexpr int kLdItems = 1;    // low-degree rounds: items per thread in flight

struct Smem {
  int owner[kBfsMaxSpan];
  int rowd[kBfsMaxSpan + 1];
  u64 cand[kBfsMaxSpan + 1];
  int wtot[kBfsThreads / 32];
  u32 minrank;  // this CTA's smallest successful next-level rank in the round
  u32 stop;     // thread 0 saw an error bit: the whole CTA leaves the loop
  // the next round's frontier counter, bottom-up floor and unsettled-list
  // length, read by thread 0 as the barrier releases
  u64 next_c;
  u32 next_minrank;
  u32 next_ucnt;
  int next_lo, next_hi;  // the next round's start bucket (lvl + 1) bounds
  u32 next_ovf;          // the next round's overflow-list length (windows)
  u32 lcnt[3];           // windows: local-queue lengths, rotating (read, fill, clear)
  u32 nstart;            // a scan's result, shared by the CTA
};
// Windows of levels keep two local queues whose entries carry a vertex, the
// key it was pushed with and its adjacency range (20 bytes, as four arrays).
// The first queue sits in the memory the edge-balanced rounds use for their
// span windows.  With two CTAs per SM the second shares it; with one, which
// has the room, it gets as much again after Smem.
constexpr size_t kSpanBytes = sizeof(int) * kBfsMaxSpan * 2 + sizeof(u64) * kBfsMaxSpan;
static_assert(offsetof(Smem, owner) == 0 && offsetof(Smem, rowd) < offsetof(Smem, cand) &&
                  offsetof(Smem, cand) + sizeof(u64) * (kBfsMaxSpan + 1) >= kSpanBytes,
              "the span-window arrays lead Smem and cover its first kSpanBytes bytes");
constexpr size_t kLqEntry = sizeof(u64) + 3 * sizeof(u32);
constexpr int lq_cap(int per_sm) {
  return (int)((per_sm >= 2 ? kSpanBytes / 2 : kSpanBytes) / kLqEntry) / 32 * 32;
}
constexpr size_t lq_extra(int per_sm) { return per_sm >= 2 ? 0 : kSpanBytes; }
// the entries a local queue takes: the tuning's limit, if any, else all that fit
template <int kCap>
__device__ __forceinline__ u32 lq_limit(const BfsArgs& a) {
  return a.window_queue ? min(a.window_queue, (u32)kCap) : (u32)kCap;
}
struct LocalQueue {
  u64* key;
  u32* rs;
  u32* re;
  u32* v;
};
template <int kCap>
__device__ __forceinline__ LocalQueue lq_buf(Smem& s, int b) {
  unsigned char* span = reinterpret_cast<unsigned char*>(&s.owner[0]);
  unsigned char* base;
  if ((size_t)kCap * kLqEntry * 2 <= kSpanBytes) base = span + (size_t)b * kCap * kLqEntry;
  else base = b == 0 ? span : reinterpret_cast<unsigned char*>(&s) + sizeof(Smem);
  LocalQueue q;
  q.key = reinterpret_cast<u64*>(base);
  q.rs = reinterpret_cast<u32*>(q.key + kCap);
  q.re = q.rs + kCap;
  q.v = q.re + kCap;
  return q;
}

// Grid-wide barrier on a monotonic arrival counter: the k-th barrier of a
// launch completes when the counter reaches k * nblocks (+ phantom), so
// arrival is one fire-and-forget add and nobody has to reset anything.
// Before arriving, thread 0 publishes this CTA's smallest next-level rank to
// ctl->minrank[post] (and resets the CTA value).  The poll is an acquire
// load, so once it sees every arrival the round's writes of all CTAs are
// visible.  The wait is bounded: after `limit` polls (or once any CTA has
// recorded an error) it sets kErrTimeout and returns.  Thread 0 then reads,
// in one round trip, the error word and the next round's state (slot `post`
// of the frontier counter, bottom-up floor and unsettled-list length, and the
// bounds of start bucket blevel unless it is negative) into shared memory, so that every thread of the CTA sees the same values and
// takes the same branch after the barrier (a thread that left the loop alone
// would leave the others at a CTA barrier).  phantom > 0 waits for CTAs that
// do not exist: the barrier can then only end by running out of polls, which
// is how the timeout path is tested.
constexpr u32 kNoPost = 0xffffffffu;  // grid_barrier: a barrier inside a round

__device__ __forceinline__ void grid_barrier(Control* ctl, u32& gen, u32 nblocks, u32 phantom,
                                             u32 limit, u32 post, const int* bptr, int blevel,
                                             Smem& s) {
  __syncthreads();
  if (threadIdx.x == 0) {
    if (post != kNoPost && s.minrank != 0xffffffffu) atomicMin(&ctl->minrank[post], s.minrank);
    if (post != kNoPost) s.minrank = 0xffffffffu;
    ++gen;
    const u64 target = (u64)gen * nblocks + phantom;
    __threadfence();
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(&ctl->bar), "l"(1ull) : "memory");
    u32 spins = 0;
    for (;;) {
      u64 seen;
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(seen) : "l"(&ctl->bar) : "memory");
      if (seen >= target) break;
      if (++spins > limit || ld_acquire_u32(&ctl->err) != 0u) {
        atomicOr(&ctl->err, kErrTimeout);
        __threadfence();
        break;
      }
      if (spins > 64) __nanosleep(20);
    }
    const u32 err = ld_cg_u32(&ctl->err);
    if (post != kNoPost) {
      s.next_c = ld_cg_u64(&ctl->qctr[post]);
      s.next_minrank = ld_cg_u32(&ctl->minrank[post]);
      s.next_ucnt = ld_cg_u32(&ctl->ucnt[post]);
      s.next_ovf = ld_cg_u32(&ctl->ovf[post]);
      s.next_lo = s.next_hi = 0;
      if (blevel >= 0) {  // bounds of start bucket blevel, for the round after the barrier
        s.next_lo = __ldg(bptr + blevel);
        s.next_hi = __ldg(bptr + blevel + 1);
      }
    }
    s.stop = err != 0u ? 1u : 0u;
  }
  __syncthreads();
}

__device__ __forceinline__ u32 warp_min(u32 x) { return __reduce_min_sync(kFull, x); }

// Exclusive prefix over the warp of small counts x < 2^kBits (and, in *tot,
// their sum), by one ballot per bit instead of a chain of shuffles.
template <int kBits>
__device__ __forceinline__ u32 warp_excl_small(u32 x, u32* tot) {
  const u32 lt = lanemask_lt();
  u32 pre = 0, sum = 0;
#pragma unroll
  for (int b = 0; b < kBits; ++b) {
    const u32 m = __ballot_sync(kFull, (x >> b) & 1u);
    pre += (u32)__popc(m & lt) << b;
    sum += (u32)__popc(m) << b;
  }
  *tot = sum;
  return pre;
}
template <int K>
constexpr int bits_for() { return K < 2 ? 1 : K < 4 ? 2 : K < 8 ? 3 : K < 16 ? 4 : K < 32 ? 5 : 6; }


// First item of this warp in a grid-stride loop over groups of 32 x k items,
// numbered so that consecutive groups go to different CTAs (warp w of CTA b
// takes group w * gridDim.x + b): a round with fewer items than threads still
// spreads over every SM instead of filling the leading CTAs.  The stride is
// gridDim.x * blockDim.x * k.  rev: CTAs in reverse order.
__device__ __forceinline__ u32 warp_first_item(u32 k, bool rev = false) {
  const u32 b = rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
  return ((threadIdx.x >> 5) * gridDim.x + b) * 32u * k;
}

__device__ __forceinline__ u64 warp_min64(u64 x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = min(x, (u64)__shfl_xor_sync(kFull, x, o));
  return x;
}

// Records a successful next-level key (vertex v, rank) for the bottom-up
// floor of the next round: the thread's running minimum, folded into the
// CTA's and the grid's at the barrier.  Unions track nothing here: their floor
// is per member (another member's smaller rank can never reach v), and it is
// computed from the frontier list only when a round goes bottom-up
// (member_floors), since keeping up to kmem minima per CTA in every round
// cost more than the rare bottom-up rounds of a batch gain from it.
template <bool U>
__device__ __forceinline__ void note_rank(const BfsArgs& a, u32 slot, bool valid, u32 v, u32 rank,
                                          u32& myrank, u32* s_acc) {
  (void)a;
  (void)slot;
  (void)v;
  (void)s_acc;
  if (!U && valid) myrank = min(myrank, rank);
}

// Unions: the per-member floors of level-L keys (the smallest rank among each
// member's keys of the frontier's level) from the frontier list qv of Q
// vertices, into slot `slot` of a.mrank (all ~0 on entry).  A warp whose
// vertices share one member makes one update; small unions gather the minima
// per CTA in shared memory (s_acc) and flush them.  The caller then waits at a
// grid barrier before the floors are read.
__device__ __forceinline__ void member_floors(const BfsArgs& a, const u32* qv, u32 Q, u32 slot,
                                              u32* s_acc) {
  const u32 lane = threadIdx.x & 31;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 base = warp_first_item(1); base < Q; base += stride) {
    const u32 i = base + lane;
    const bool valid = i < Q;
    u32 v = 0, m = 0xffffffffu, r = 0xffffffffu;
    if (valid) {
      v = ld_cg_u32(qv + i);
      m = __ldg(a.wmem + (v >> 5));
      r = (u32)ld_cg_u64(a.key + v);
    }
    const u32 act = __ballot_sync(kFull, valid);
    const u32 m0 = __shfl_sync(kFull, m, __ffs(act) - 1);
    const bool one = __all_sync(kFull, !valid || m == m0);
    const u32 rr = one ? warp_min(r) : r;
    if ((one && lane == 0) || (!one && valid)) {
      const u32 mm = one ? m0 : m;
      if (s_acc) {
        if (rr < s_acc[mm]) atomicMin(s_acc + mm, rr);
      } else {
        u32* p = a.mrank + (size_t)slot * a.kmem + mm;
        if (rr < ld_cg_u32(p)) atomicMin(p, rr);
      }
    }
  }
}

// Union: the CTA's per-member minima into slot `slot` of a.mrank, and the
// shared table reset.  Called by the whole CTA between __syncthreads.
__device__ __forceinline__ void flush_members(const BfsArgs& a, u32 slot, u32* s_acc) {
  for (u32 m = threadIdx.x; m < a.kmem; m += blockDim.x) {
    const u32 r = s_acc[m];
    if (r != 0xffffffffu) {
      u32* p = a.mrank + (size_t)slot * a.kmem + m;
      if (r < ld_cg_u32(p)) atomicMin(p, r);
      s_acc[m] = 0xffffffffu;
    }
  }
}

// Appends to the frontier every vertex v[i] whose bit i is set in `mask`, for
// up to K candidates per lane, with one atomicAdd per warp: the warp scans
// (count << 32 | degree sum) over its lanes, reserves that many queue slots
// and edge offsets, and every lane writes its vertices in slot order.
// qi: frontier counter index (rotates over 3), qb: queue buffer (ping-pong).
// Low-degree mode: the frontier is the plain vertex list qv (items in the
// counter's high word, its low word unused), so an append is one reservation
// per warp and one store per vertex, with no adjacency range to load.
template <int K>
__device__ __forceinline__ void warp_append_ld(u32 mask, const u32 (&v)[K], const BfsArgs& a,
                                               int qi, int qb) {
  const u32 lane = threadIdx.x & 31;
  u32 tot;
  const u32 excl = warp_excl_small<bits_for<K>()>(__popc(mask), &tot);
  if (tot == 0) return;
  u32 base = 0;
  if (lane == 0) base = (u32)(atomicAdd(&a.ctl->qctr[qi], (u64)tot << 32) >> 32);
  u32 slot = __shfl_sync(kFull, base, 0) + excl;
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (mask >> i & 1u) a.qv[qb][slot++] = v[i];
}

template <int K, bool LD>
__device__ __forceinline__ void warp_append(u32 mask, const u32 (&v)[K], const BfsArgs& a, int qi,
                                            int qb) {
  if (LD) {
    warp_append_ld<K>(mask, v, a, qi, qb);
    return;
  }
  const u32 lane = threadIdx.x & 31;
  int rs[K], dg[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    rs[i] = 0;
    dg[i] = 0;
    if (mask >> i & 1u) {
      rs[i] = __ldg(a.row_ptr + v[i]);
      dg[i] = __ldg(a.row_ptr + v[i] + 1) - rs[i];
    }
  }
  u32 cnt = 0, dsum = 0;
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (dg[i] <= 0) {
      mask &= ~(1u << i);  // a vertex without arcs has nothing to expand
    } else {
      ++cnt;
      dsum += (u32)dg[i];
    }
  if (!__any_sync(kFull, mask != 0u)) return;
  const u64 mine = ((u64)cnt << 32) | dsum;
  u64 incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 y = __shfl_up_sync(kFull, incl, o);
    if (lane >= (u32)o) incl += y;
  }
  const u64 tot = __shfl_sync(kFull, incl, 31);
  u64 base = 0;
  if (lane == 0) base = atomicAdd(&a.ctl->qctr[qi], tot);
  base = __shfl_sync(kFull, base, 0) + (incl - mine);
  u32 slot = (u32)(base >> 32), off = (u32)base;
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (mask >> i & 1u) {
      a.qv[qb][slot] = v[i];
      a.qrow[qb][slot] = rs[i];
      a.qoff[qb][slot] = off;
      const u32 end = off + (u32)dg[i];
      for (u32 c = (off + kBfsBase - 1) / kBfsBase; c * kBfsBase < end; ++c) a.cf[qb][c] = slot;
      ++slot;
      off = end;
    }
}

// Unclaimed vertices of start bucket rr join the frontier of level rr.
template <bool U>
__device__ __forceinline__ void append_bucket(const BfsArgs& a, int rr, const u32* rv, int qi,
                                              int qb, u32& myrank, u32* s_acc, int lo = -1,
                                              int hi = -1) {
  if (lo < 0) {  // bounds not known yet
    lo = __ldg(a.bptr + rr);
    hi = __ldg(a.bptr + rr + 1);
  }
  const u32 cnt = (u32)(hi - lo);
  const u32 lane = threadIdx.x & 31;
  const u32 stride = gridDim.x * blockDim.x;
  // trailing CTAs first: in a small round the leading CTAs are expanding
  for (u32 base = warp_first_item(1, true); base < cnt; base += stride) {
    const u32 i = base + lane;
    u32 u[1] = {0};
    bool want = false;
    u64 k = 0;
    if (i < cnt) {
      u[0] = __ldg(rv + lo + i);
      k = ld_cg_u64(a.key + u[0]);
      want = (u32)(k >> 32) == (u32)rr;
    }
    note_rank<U>(a, (u32)qi, want, u[0], (u32)k, myrank, s_acc);
    warp_append<1, false>(want ? 1u : 0u, u, a, qi, qb);
  }
}

template <bool U>
__device__ __forceinline__ void expand(const BfsArgs& a, Smem& s, int cur, u32 Q, u32 E, int lvl,
                                       int qi, int qb, u32& myrank, u32* s_acc) {
  const u32 nb = (E + kBfsBase - 1) / kBfsBase;
  u32 k = (nb + gridDim.x - 1) / gridDim.x;
  k = max(1u, min(k, a.span / kBfsBase));
  const u32 nsuper = (nb + k - 1) / k;
  const u32* cf = a.cf[cur];
  const u32* qv = a.qv[cur];
  const int* qrow = a.qrow[cur];
  const u32* qoff = a.qoff[cur];
  const u32 lvl_next = (u32)lvl + 1;
  const bool probe = E >= a.probe_min_arcs;  // smaller frontiers skip the key probe
  for (u32 sc = blockIdx.x; sc < nsuper; sc += gridDim.x) {
    const u32 b0 = sc * k, b1 = min(b0 + k, nb);
    const u32 e0 = b0 * kBfsBase, e1 = min(b1 * kBfsBase, E);
    const u32 i0 = ld_cg_u32(cf + b0);
    const u32 ilast = (b1 < nb) ? ld_cg_u32(cf + b1) : Q - 1;
    const int nwin = (int)(ilast - i0) + 1;
    const int len = (int)(e1 - e0);
    if (nwin > kBfsMaxSpan + 1 || nwin < 1 || ilast >= Q) {  // window invariant broken
      if (threadIdx.x == 0) atomicOr(&a.ctl->err, kErrInternal);
      return;
    }
    for (int j = threadIdx.x; j < len; j += kBfsThreads) s.owner[j] = 0;
    __syncthreads();
    // window: queue items covering [e0, e1); loads batched for memory-level parallelism
    for (int j0 = 0; j0 < nwin; j0 += kBfsThreads * kWinBatch) {
      u32 off[kWinBatch], v[kWinBatch];
      int row[kWinBatch];
#pragma unroll
      for (int i = 0; i < kWinBatch; ++i) {
        const int j = j0 + i * kBfsThreads + (int)threadIdx.x;
        off[i] = e1;
        if (j < nwin) {
          off[i] = ld_cg_u32(qoff + i0 + j);
          v[i] = ld_cg_u32(qv + i0 + j);
          row[i] = ld_cg_i32(qrow + i0 + j);
        }
      }
      u64 kv[kWinBatch];
#pragma unroll
      for (int i = 0; i < kWinBatch; ++i)
        if (off[i] < e1) kv[i] = ld_cg_u64(a.key + v[i]);
#pragma unroll
      for (int i = 0; i < kWinBatch; ++i)
        if (off[i] < e1) {
          const int j = j0 + i * kBfsThreads + (int)threadIdx.x;
          s.rowd[j] = row[i] - (int)off[i];
          s.cand[j] = kv[i] + kLevelOne;
          atomicMax(&s.owner[off[i] > e0 ? off[i] - e0 : 0u], j);
        }
    }
    __syncthreads();
    block_max_scan<kBfsThreads, kBfsMaxSpan>(s.owner, len, s.wtot);
    __syncthreads();
    // edges: all loads of a batch first, then all probes, then the atomics
    for (int base = 0; base < len; base += kBfsThreads * kEdgeBatch) {
      u32 w[kEdgeBatch];
      u64 cand[kEdgeBatch];
#pragma unroll
      for (int i = 0; i < kEdgeBatch; ++i) {
        const int kk = base + i * kBfsThreads + (int)threadIdx.x;
        w[i] = 0xffffffffu;
        cand[i] = 0;
        if (kk < len) {
          const int j = s.owner[kk];
          cand[i] = s.cand[j];
          w[i] = (u32)__ldg(a.col + (s.rowd[j] + (int)(e0 + kk)));
        }
      }
      u64 cur[kEdgeBatch];  // probe before the atomic only when there are many arcs
#pragma unroll
      for (int i = 0; i < kEdgeBatch; ++i)
        cur[i] = (w[i] < a.n) ? (probe ? ld_cg_u64(a.key + w[i]) : ~0ull) : 0ull;
      u32 mask = 0, won = 0;
#pragma unroll
      for (int i = 0; i < kEdgeBatch; ++i)
        if (cand[i] < cur[i]) {
          const u64 old = atomicMin(a.key + w[i], cand[i]);
          if (old > cand[i]) won |= 1u << i;
          if ((u32)(old >> 32) > lvl_next) mask |= 1u << i;
        }
#pragma unroll
      for (int i = 0; i < kEdgeBatch; ++i)
        note_rank<U>(a, (u32)qi, (won >> i) & 1u, w[i], (u32)cand[i], myrank, s_acc);
      warp_append<kEdgeBatch, false>(mask, w, a, qi, qb);
    }
    __syncthreads();
  }
}

// Low-degree round (every vertex of the graph has at most kLdMaxDegree
// arcs): one pass over Q frontier vertices (the list qv_cur) and the cnt
// entries of start bucket rb (from lo in rv), a thread per item.
//   * A frontier vertex v offers key[v] + 2^32 to each of its neighbours
//     (64-bit atomicMin, after a probe of the key when `probe`), kLdBatch arcs
//     per step, and appends the neighbours whose level it lowered to lvl + 1.
//   * A start-bucket entry u joins the next frontier if its key still has its
//     start level rb (Section 4's delayed start; stable during the round, see
//     the file comment).
// v's key and adjacency range, and the bucket entries' keys, load in one round
// trip, and the bucket test runs beside the expansion instead of after it: a
// thin round is a short chain of dependent loads.  A thread takes kLdItems
// items at a time (a warp 32 kLdItems consecutive ones) and interleaves their
// loads, so that a round with more items than threads still costs about one
// such chain.  `pushed` adds the arcs offered.
template <bool U>
__device__ __forceinline__ void expand_ld(const BfsArgs& a, const u32* qv_cur, u32 Q, u32 lvl_next,
                                          const u32* rv, int lo, u32 cnt, u32 rb, bool probe,
                                          int qi, int qb, u32& myrank, u32* s_acc, u64& pushed) {
  constexpr u32 kNone = 0xffffffffu;
  constexpr int KI = kLdItems;
  constexpr int KA = kLdItems * kLdBatch;
  const u32 lane = threadIdx.x & 31;
  const u32 total = Q + cnt;
  const u32 stride = gridDim.x * blockDim.x * KI;
  for (u32 base = warp_first_item(KI); base < total; base += stride) {
    u32 v[KI];
    bool front[KI], buck[KI];
#pragma unroll
    for (int t = 0; t < KI; ++t) {
      const u32 i = base + (u32)t * 32 + lane;
      front[t] = i < Q;
      buck[t] = !front[t] && i < total;
      v[t] = 0;
      if (front[t]) v[t] = ld_cg_u32(qv_cur + i);
      else if (buck[t]) v[t] = __ldg(rv + lo + (int)(i - Q));
    }
    u64 kv[KI];
    int rs[KI], re[KI];
#pragma unroll
    for (int t = 0; t < KI; ++t) {
      kv[t] = 0;
      rs[t] = 0;
      re[t] = 0;
      if (front[t] || buck[t]) kv[t] = ld_cg_u64(a.key + v[t]);
      if (front[t]) {
        rs[t] = __ldg(a.row_ptr + v[t]);
        re[t] = __ldg(a.row_ptr + v[t] + 1);
      }
    }
    u32 smask = 0;
#pragma unroll
    for (int t = 0; t < KI; ++t) {
      const bool start = buck[t] && (u32)(kv[t] >> 32) == rb;
      if (start) smask |= 1u << t;
      note_rank<U>(a, (u32)qi, start, v[t], (u32)kv[t], myrank, s_acc);
    }
    warp_append<KI, true>(smask, v, a, qi, qb);
    int nch = 0;
#pragma unroll
    for (int t = 0; t < KI; ++t) {
      pushed += (u64)(re[t] - rs[t]);
      nch = max(nch, (re[t] - rs[t] + kLdBatch - 1) / kLdBatch);
    }
    nch = (int)__reduce_max_sync(kFull, (u32)nch);
    for (int ch = 0; ch < nch; ++ch) {
      u32 w[KA];
#pragma unroll
      for (int t = 0; t < KI; ++t)
#pragma unroll
        for (int q = 0; q < kLdBatch; ++q) {
          const int e = rs[t] + ch * kLdBatch + q;
          w[t * kLdBatch + q] = e < re[t] ? (u32)__ldg(a.col + e) : kNone;
        }
      u64 cur[KA];
#pragma unroll
      for (int x = 0; x < KA; ++x)
        cur[x] = (w[x] < a.n) ? (probe ? ld_cg_u64(a.key + w[x]) : ~0ull) : 0ull;
      u32 mask = 0, won = 0;
#pragma unroll
      for (int x = 0; x < KA; ++x) {
        const u64 cand = kv[x / kLdBatch] + kLevelOne;
        if (cand < cur[x]) {
          const u64 old = atomicMin(a.key + w[x], cand);
          if (old > cand) won |= 1u << x;
          if ((u32)(old >> 32) > lvl_next) mask |= 1u << x;
        }
      }
#pragma unroll
      for (int x = 0; x < KA; ++x)
        note_rank<U>(a, (u32)qi, (won >> x) & 1u, w[x], (u32)(kv[x / kLdBatch] + kLevelOne),
                     myrank, s_acc);
      warp_append<KA, true>(mask, w, a, qi, qb);
    }
  }
}

// ---------------------------------------------------------------- windows of levels
// Low-degree rounds may run a window of levels [L, H) between two grid
// barriers instead of one level.  Each CTA expands its share of the level-L
// frontier (and of the overflow list of the last window), then keeps going on
// its own: every vertex whose key it lowers to a level below H goes into the
// CTA's local queue (shared memory) and is expanded by the same CTA at the
// next local level, with only a CTA barrier in between; vertices lowered to
// level H go to the global queue for the next round.  Start bucket lv + 1 is
// checked at local level lv, as in a one-level round.
//
// Exactness: keys only decrease, and the fixed point of the min over all
// offers does not depend on the order in which they are made (Section 4's
// shortest path, label-correcting).  Every successful atomicMin makes its
// vertex be expanded again: it is pushed with the level it got, to a local
// queue, to the global queue (the first time it reaches level H), or -- when
// a local queue is full -- to the overflow list that the next round expands.
// A global-queue or overflow entry whose vertex has meanwhile been lowered to
// a smaller level is skipped, since its lowerer pushed it again; a local entry
// carries the key it was pushed with, and if that key is outdated, its offers
// are dominated by those of the better one.  Past level H - 1 a CTA works its
// local queue down until it is empty.  A CTA may run ahead of another
// inside a window, so a vertex can first get a worse key and be expanded
// twice (the statistics count every expansion); the result is the same.  A
// start test inside a window may let a vertex start that a slower CTA lowers
// later: it is expanded again with the better key.  At the end of a window
// every key below level H is final unless an overflow entry is pending, and
// the loop then runs another window before any bottom-up round.
//
// Once a window has run, the number of settled vertices is no longer counted
// exactly; an empty frontier then scans the start buckets from the current
// level for the next one that still holds an unclaimed vertex (one pass and
// one grid barrier) instead of stopping when every vertex is settled.

// Pushes vertex w[i] with key k[i] and adjacency range [rs[i], re[i]) for
// every bit i of mask: to the CTA's local queue nb while it has room, the rest
// (as vertex and level) to the overflow list of the next round.
template <int K, int kCap>
__device__ __forceinline__ void window_push(u32 mask, const u32 (&w)[K], const u64 (&k)[K],
                                            const int (&rs)[K], const int (&re)[K],
                                            const BfsArgs& a, Smem& s, int nb, int nc, int qi,
                                            int qb) {
  const u32 lane = threadIdx.x & 31;
  u32 tot;
  const u32 excl = warp_excl_small<bits_for<K>()>(__popc(mask), &tot);
  if (tot == 0) return;
  u32 base = 0;
  if (lane == 0) base = atomicAdd(&s.lcnt[nc], tot);
  base = __shfl_sync(kFull, base, 0) + excl;
  const LocalQueue lq = lq_buf<kCap>(s, nb);
  const u32 cap = lq_limit<kCap>(a);
  u32 spill = 0;
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (mask >> i & 1u) {
      if (base < cap) {
        lq.key[base] = k[i];
        lq.rs[base] = (u32)rs[i];
        lq.re[base] = (u32)re[i];
        lq.v[base] = w[i];
      } else {
        spill |= 1u << i;
      }
      ++base;
    }
  // a full local queue: the rest waits for the next round on the overflow list
  if (!__any_sync(kFull, spill != 0u)) return;
  u32 stot;
  const u32 sexcl = warp_excl_small<bits_for<K>()>(__popc(spill), &stot);
  u32 sbase = 0;
  if (lane == 0) sbase = atomicAdd(&a.ctl->ovf[qi], stot);
  sbase = __shfl_sync(kFull, sbase, 0) + sexcl;
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (spill >> i & 1u) {
      if (sbase < a.n) {
        reinterpret_cast<u32*>(a.qrow[qb])[sbase] = w[i];
        a.qoff[qb][sbase] = (u32)(k[i] >> 32);
      } else {
        atomicOr(&a.ctl->err, kErrInternal);  // more pushes than vertices: cannot happen
      }
      ++sbase;
    }
}

// Expands one item per lane -- valid: key kv, adjacency range [rs, re) -- in a
// window whose end is H: kv + 2^32 is offered to the neighbours.  Winners
// below H go to the local queue nb with the key they got and their adjacency
// range (loaded beside the atomicMin, not after it), winners at H that reach
// it for the first time to the global queue qb.  A kv that is no longer the
// vertex's key (it was lowered again, and its lowerer pushed it again) only
// makes offers that the better key dominates.  Every lane of the warp calls
// this.
template <bool U, int kCap>
__device__ __forceinline__ void window_expand(const BfsArgs& a, Smem& s, bool valid, u64 kv,
                                              int rs, int re, u32 H, int nb, int nc, int qi,
                                              int qb,
                                              u32& myrank, u32* s_acc, u64& pushed,
                                              u64& expanded) {
  constexpr u32 kNone = 0xffffffffu;
  if (!valid) re = rs;
  else ++expanded;
  pushed += (u64)(re - rs);
  const u64 cand = kv + kLevelOne;
  const u32 cl = (u32)(cand >> 32);
  const int nch = (int)__reduce_max_sync(kFull, (u32)((re - rs + kLdBatch - 1) / kLdBatch));
  for (int ch = 0; ch < nch; ++ch) {
    const int e0 = rs + ch * kLdBatch;
    u32 w[kLdBatch];
#pragma unroll
    for (int q = 0; q < kLdBatch; ++q) w[q] = (e0 + q < re) ? (u32)__ldg(a.col + e0 + q) : kNone;
    u64 kk[kLdBatch];
    int wrs[kLdBatch], wre[kLdBatch];
    u32 local = 0, glob = 0, won = 0;
#pragma unroll
    for (int q = 0; q < kLdBatch; ++q) {
      kk[q] = cand;
      wrs[q] = 0;
      wre[q] = 0;
      if (w[q] < a.n) {
        if (cl < H) {  // the range of a vertex that may be pushed locally, beside the atomic
          wrs[q] = __ldg(a.row_ptr + w[q]);
          wre[q] = __ldg(a.row_ptr + w[q] + 1);
        }
        const u64 old = atomicMin(a.key + w[q], cand);
        if (old > cand) {
          won |= 1u << q;
          if (cl < H) local |= 1u << q;
          else if ((u32)(old >> 32) > H) glob |= 1u << q;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kLdBatch; ++q)  // the next round's bottom-up floor: level-H keys
      note_rank<U>(a, (u32)qi, ((won >> q) & 1u) && cl == H, w[q], (u32)cand, myrank, s_acc);
    window_push<kLdBatch, kCap>(local, w, kk, wrs, wre, a, s, nb, nc, qi, qb);
    warp_append<kLdBatch, true>(glob, w, a, qi, qb);
  }
}

// One window of levels [L, H): the level-L frontier (Q entries of qv_cur) and
// the nov overflow entries of the last round (qrow/qoff of side qcur, vertex
// and level), then local levels L .. H - 1, then whatever the CTA's local
// queue still holds.
// Only pushes that find the local queue full wait for the next round (on the
// overflow list).  `expanded` counts expansions.
template <bool U, int kCap>
__device__ __forceinline__ void window_ld(const BfsArgs& a, Smem& s, const u32* rv, int A,
                                          u32 Q, u32 nov, int qcur, u32 L, u32 H, int qi, int qb,
                                          u32& myrank, u32* s_acc, u64& pushed, u64& expanded) {
  const u32 lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s.lcnt[0] = 0;
    s.lcnt[1] = 0;
    s.lcnt[2] = 0;
  }
  __syncthreads();
  // Start buckets are read one level ahead: at level lv this thread's first
  // entry of bucket lv + 1 is known (its key is requested as the level
  // starts, beside the expansions) and its first entry of bucket lv + 2 and
  // the bounds of bucket lv + 3 are requested.  A key read before the level's
  // expansions can only be higher than after them: a start taken on it that a
  // correction undercuts is an entry that its expansion skips.
  constexpr u32 kNoItem = 0xffffffffu;
  const u32 i0 = warp_first_item(1, true) + lane;  // this thread's first entry of a bucket
  const u32 gstride = gridDim.x * blockDim.x;
  auto bucket_ok = [&](u32 r) { return (int)r <= A && r <= H; };
  int b1lo = 0, b1hi = 0, b2lo = 0, b2hi = 0;  // buckets lv + 1 and lv + 2
  if (bucket_ok(L + 1)) {
    b1lo = __ldg(a.bptr + L + 1);
    b1hi = __ldg(a.bptr + L + 2);
  }
  if (bucket_ok(L + 2)) {
    b2lo = __ldg(a.bptr + L + 2);
    b2hi = __ldg(a.bptr + L + 3);
  }
  u32 pu = kNoItem;  // this thread's first entry of bucket lv + 1
  if (i0 < (u32)(b1hi - b1lo)) pu = __ldg(rv + b1lo + (int)i0);
  int lb = 0;  // the local queue being read (level lv); the other one is filled
  int cr = 0;  // the counter of the queue being read; (cr + 1) % 3 counts the filled one
  for (u32 lv = L;; ++lv) {
    const int nb = lb ^ 1;
    const int nc = cr == 2 ? 0 : cr + 1;
    // the third counter, read last at level lv - 1 and filled next at level
    // lv + 1, is cleared now: one CTA barrier per level
    if (threadIdx.x == 0) s.lcnt[nc == 2 ? 0 : nc + 1] = 0;
    const u32 nloc = min(s.lcnt[cr], lq_limit<kCap>(a));  // the same for the whole CTA
    // Past the window's last level the CTA goes on with its own queue until
    // it is empty: entries of overflow from an earlier window run behind the
    // frontier, and their chains end here instead of one hop per round.
    if (lv >= H && nloc == 0) break;
    u64 pk = 0;  // its key and adjacency range
    int pr0 = 0, pr1 = 0;
    if (pu != kNoItem) {
      pk = ld_cg_u64(a.key + pu);
      pr0 = __ldg(a.row_ptr + pu);
      pr1 = __ldg(a.row_ptr + pu + 1);
    }
    u32 pu2 = kNoItem;
    if (i0 < (u32)(b2hi - b2lo)) pu2 = __ldg(rv + b2lo + (int)i0);
    int b3lo = 0, b3hi = 0;
    if (bucket_ok(lv + 3)) {
      b3lo = __ldg(a.bptr + lv + 3);
      b3hi = __ldg(a.bptr + lv + 4);
    }
    // (1) the window's first level: the global frontier and the overflow list,
    // whose keys and ranges are loaded here
    if (lv == L) {
      const u32 total = Q + nov;
      for (u32 base = warp_first_item(1); base < total; base += gridDim.x * blockDim.x) {
        const u32 i = base + lane;
        u32 v = 0, lev = L;
        if (i < Q) {
          v = ld_cg_u32(a.qv[qcur] + i);
        } else if (i < total) {
          v = ld_cg_u32(reinterpret_cast<const u32*>(a.qrow[qcur]) + (i - Q));
          lev = ld_cg_u32(a.qoff[qcur] + (i - Q));
        }
        u64 kv = 0;
        int rs = 0, re = 0;
        bool ok = i < total;
        if (ok) {
          kv = ld_cg_u64(a.key + v);
          rs = __ldg(a.row_ptr + v);
          re = __ldg(a.row_ptr + v + 1);
          ok = (u32)(kv >> 32) >= lev;  // lowered since: its lowerer pushed it again
        }
        window_expand<U, kCap>(a, s, ok, kv, rs, re, H, nb, nc, qi, qb, myrank, s_acc, pushed,
                               expanded);
      }
    }
    // (2) this CTA's local queue of level lv: keys and ranges come with the entries
    {
      const LocalQueue lq = lq_buf<kCap>(s, lb);
      for (u32 base = threadIdx.x & ~31u; base < nloc; base += blockDim.x) {
        const u32 i = base + lane;
        const bool ok = i < nloc;
        window_expand<U, kCap>(a, s, ok, ok ? lq.key[i] : 0ull, ok ? (int)lq.rs[i] : 0,
                               ok ? (int)lq.re[i] : 0, H, nb, nc, qi, qb, myrank, s_acc, pushed,
                               expanded);
      }
    }
    // (3) start bucket lv + 1: a vertex whose key still has its start level joins level lv + 1
    if (bucket_ok(lv + 1)) {
      const u32 cnt = (u32)(b1hi - b1lo);
      for (u32 base = i0 - lane; base < cnt; base += gstride) {  // warp-uniform
        const u32 i = base + lane;
        u32 u[1] = {0};
        u64 k[1] = {0};
        int urs[1] = {0}, ure[1] = {0};
        bool start = false;
        if (i < cnt) {
          if (i == i0) {  // the entry read ahead
            u[0] = pu;
            k[0] = pk;
            urs[0] = pr0;
            ure[0] = pr1;
          } else {
            u[0] = __ldg(rv + b1lo + (int)i);
            k[0] = ld_cg_u64(a.key + u[0]);
            urs[0] = __ldg(a.row_ptr + u[0]);
            ure[0] = __ldg(a.row_ptr + u[0] + 1);
          }
          start = (u32)(k[0] >> 32) == lv + 1;
        }
        if (lv + 1 < H) {
          window_push<1, kCap>(start ? 1u : 0u, u, k, urs, ure, a, s, nb, nc, qi, qb);
        } else {
          note_rank<U>(a, (u32)qi, start, u[0], (u32)k[0], myrank, s_acc);
          warp_append<1, true>(start ? 1u : 0u, u, a, qi, qb);
        }
      }
    }
    __syncthreads();  // every push of level lv + 1 is in; level lv's queue is read
    lb = nb;
    cr = nc;
    pu = pu2;
    b1lo = b2lo;
    b1hi = b2hi;
    b2lo = b3lo;
    b2hi = b3hi;
  }
}

// The smallest start level >= from among start-bucket entries whose key still
// has their start level (a vertex nobody has claimed), into ctl->nstart[slot]
// as ~level by atomicMax (0 if none); the caller waits at a grid barrier.
__device__ __forceinline__ void scan_unclaimed(const BfsArgs& a, const u32* rk, const u32* rv,
                                               int from, int A, u32 slot) {
  if (from > A) return;
  const int lo = __ldg(a.bptr + from), hi = __ldg(a.bptr + A + 1);
  u32 best = 0;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; (int)i < hi - lo;
       i += gridDim.x * blockDim.x) {
    const u32 r = __ldg(rk + lo + (int)i);
    const u64 k = ld_cg_u64(a.key + __ldg(rv + lo + (int)i));
    if ((u32)(k >> 32) == r) best = max(best, ~r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(kFull, best, o));
  if ((threadIdx.x & 31) == 0 && best) atomicMax(&a.ctl->nstart[slot], best);
}

// Folds a thread's smallest rank into the CTA's (lane 0 of each warp) and resets it.
__device__ __forceinline__ void post_cta_min(Smem& s, u32& myrank) {
  const u32 wm = warp_min(myrank);
  if ((threadIdx.x & 31) == 0 && wm != 0xffffffffu) atomicMin(&s.minrank, wm);
  myrank = 0xffffffffu;
}

// The two appends of a bottom-up step in one pass.  The vertices of `mask`
// join the next frontier; their adjacency ranges [rs, re) are known already,
// so, unlike warp_append, no row_ptr round trip comes first.  The vertices of
// `keep` join the list of the next bottom-up round.  Lane 0 sends both
// reservations before waiting for either.
template <int K, bool LD>
__device__ __forceinline__ void pull_append(u32 mask, u32 keep, const u32 (&v)[K],
                                            const int (&rs)[K], const int (&re)[K],
                                            const BfsArgs& a, int qi, int qb, u32* list,
                                            u32* lcount) {
  const u32 lane = threadIdx.x & 31;
  u32 cnt = 0, dsum = 0;
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (mask >> i & 1u) {
      if (re[i] <= rs[i]) {
        mask &= ~(1u << i);  // a vertex without arcs has nothing to expand
      } else {
        ++cnt;
        dsum += (u32)(re[i] - rs[i]);
      }
    }
  const u32 kc = __popc(keep);
  if (!__any_sync(kFull, mask != 0u || keep != 0u)) return;
  const u64 mine = ((u64)cnt << 32) | (LD ? 0u : dsum);
  u64 incl = mine;
  u32 kincl = kc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 y = __shfl_up_sync(kFull, incl, o);
    const u32 ky = __shfl_up_sync(kFull, kincl, o);
    if (lane >= (u32)o) {
      incl += y;
      kincl += ky;
    }
  }
  const u64 tot = __shfl_sync(kFull, incl, 31);
  const u32 ktot = __shfl_sync(kFull, kincl, 31);
  u64 base = 0;
  u32 kbase = 0;
  if (lane == 0) {
    if (tot) base = atomicAdd(&a.ctl->qctr[qi], tot);
    if (ktot) kbase = atomicAdd(lcount, ktot);
  }
  base = __shfl_sync(kFull, base, 0) + (incl - mine);
  kbase = __shfl_sync(kFull, kbase, 0) + (kincl - kc);
  u32 slot = (u32)(base >> 32), off = (u32)base;
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (mask >> i & 1u) {
      a.qv[qb][slot] = v[i];
      if (!LD) {
        const u32 dg = (u32)(re[i] - rs[i]);
        a.qrow[qb][slot] = rs[i];
        a.qoff[qb][slot] = off;
        const u32 end = off + dg;
        for (u32 c = (off + kBfsBase - 1) / kBfsBase; c * kBfsBase < end; ++c) a.cf[qb][c] = slot;
        off = end;
      }
      ++slot;
    }
#pragma unroll
  for (int i = 0; i < K; ++i)
    if (keep >> i & 1u) list[kbase++] = v[i];
}

// Bottom-up round from level lvl (see the file comment).  Candidates are every
// vertex not in excl (from_list = false; a.active lists them when it is set)
// or the list `cand` of ncand vertices.
// Each lane takes kPullV candidates at a time and advances their neighbour
// scans in lock-step, one neighbour each per step, so that up to kPullV
// independent loads are in flight per lane.  A scan's first probe is the
// candidate's first neighbour from the per-graph table (when there is one),
// loaded beside its key, so it needs no col round trip.  Adds the arcs it
// scans and the vertices it examines to the statistics.
template <bool U, bool LD, int kPullV>
__device__ __forceinline__ void pull_round(const BfsArgs& a, int lvl, u32 minrank, u32 mslot,
                                           int qi, int qb, bool from_list, const u32* cand,
                                           u32 ncand, u32* ulist_out, u32* ucnt_out,
                                           u32& myrank, u32* s_acc, const u32* s_floor) {
  constexpr u32 kNone = 0xffffffffu;
  u32 scanned = 0, examined = 0;
  const u32 lane = threadIdx.x & 31;
  const u32 L = (u32)lvl;
  if (!from_list && a.active) {  // the first bottom-up round: the BFS's own vertices
    from_list = true;
    cand = a.active;
    ncand = a.n_active;
  }
  const u32 total = from_list ? ncand : a.n;
  // Units of 32 kPullV candidates.  A single graph deals about three fifths
  // of them out in advance, kd per warp (warps interleaved across CTAs as
  // everywhere), a union only every warp's first; the rest go to whichever
  // warp asks next, one atomic ticket per unit, so a warp held up by hub scans
  // takes fewer units instead of holding the round.  (R-MAT 22 round loop
  // 0.143 -> 0.136 ms; 64 R-MAT 20 copies as a union 5.2 -> 4.0 ms, where
  // dealing three fifths in advance gave 4.9 ms.)
  constexpr u32 kUnit = 32u * kPullV;
  const u32 W = gridDim.x * (blockDim.x >> 5);
  const u32 kd = U ? 1u : max(1u, ((total + kUnit - 1) / kUnit / W) * 3 / 5);
  u32* const next_unit = &a.ctl->pull_ctr[mslot];
  auto unit_base = [&](u32 ticket) {  // lane 0's ticket: the unit's first candidate
    return (kd * W + __shfl_sync(kFull, ticket, 0)) * kUnit;
  };
  // The passes are software-pipelined: pass p + 1's candidates are requested
  // when pass p starts, and their keys and adjacency ranges while pass p makes
  // its appends, so a pass waits only on its neighbour scans and its appends.
  auto load_ids = [&](u32 b, u32 (&w)[kPullV]) {
#pragma unroll
    for (int j = 0; j < kPullV; ++j) {
      const u32 i = b + (u32)j * 32 + lane;
      w[j] = kNone;
      if (from_list) {
        if (i < total) w[j] = ld_cg_u32(cand + i);
      } else if (i < total) {
        const u32 ex = __ldg(a.excl + (i >> 5));  // same word for the whole warp
        if (!((ex >> lane) & 1u)) w[j] = i;
      }
    }
  };
  // the key, the adjacency range and the first neighbour together: one round
  // trip, and the scan's first probe needs no col load
  auto load_keys = [&](const u32 (&w)[kPullV], u64 (&kw)[kPullV], int (&e)[kPullV],
                       int (&re)[kPullV], u32 (&f)[kPullV]) {
#pragma unroll
    for (int j = 0; j < kPullV; ++j) {
      kw[j] = 0ull;
      e[j] = 0;
      re[j] = 0;
      f[j] = kNone;
      if (w[j] != kNone) {
        kw[j] = ld_cg_u64(a.key + w[j]);
        e[j] = __ldg(a.row_ptr + w[j]);
        re[j] = __ldg(a.row_ptr + w[j] + 1);
        if (a.first) f[j] = __ldg(a.first + w[j]);
      }
    }
  };
  u32 base = warp_first_item(kPullV);
  u32 w[kPullV], f[kPullV];
  u64 kw[kPullV];
  int e[kPullV], re[kPullV];
  load_ids(base, w);
  load_keys(w, kw, e, re, f);
  const u32 gw = base / kUnit;  // this warp's first unit
  auto dealt_base = [&](u32 p) { return (p * W + gw) * kUnit; };  // its pass p < kd
  u32 pass = 0, ticket = 0;
  if (lane == 0 && kd <= 1 && base < total) ticket = atomicAdd(next_unit, 1u);
  u32 nbase = kd > 1 ? dealt_base(1) : (base < total ? unit_base(ticket) : total);
  while (base < total) {
    u32 wn[kPullV];  // the next pass's candidates, in flight during this pass
    load_ids(nbase, wn);
    // the ticket for the pass after the next: its atomic returns during this pass
    if (lane == 0 && pass + 2 >= kd && nbase < total) ticket = atomicAdd(next_unit, 1u);
    int rs0[kPullV], re0[kPullV];  // the adjacency ranges, for the appends
#pragma unroll
    for (int j = 0; j < kPullV; ++j) {
      rs0[j] = e[j];
      re0[j] = re[j];
    }
    u64 best[kPullV];
    u32 fr[kPullV];  // floor rank: nothing beats (L + 1, fr); union: w's own member's
#pragma unroll
    for (int j = 0; j < kPullV; ++j) {
      fr[j] = minrank;
      if (U && w[j] != kNone) {
        const u32 m = __ldg(a.wmem + (w[j] >> 5));
        fr[j] = s_floor ? s_floor[m] : ld_cg_u32(a.mrank + (size_t)mslot * a.kmem + m);
      }
    }
    const u64 lvl_key = (u64)(L + 1) << 32;
#pragma unroll
    for (int j = 0; j < kPullV; ++j) {
      best[j] = kw[j];
      if (w[j] != kNone) ++examined;
      if (!((u32)(kw[j] >> 32) > L && kw[j] > (lvl_key | fr[j]))) re[j] = e[j];  // settled or unbeatable
      if (U && fr[j] == 0xffffffffu) re[j] = e[j];  // w's member has no level-L key
    }
    // one neighbour of every still-scanning candidate per step, for at most
    // kPullLong steps: most scans stop at their first neighbours
    for (int step = 0; step < kPullLong; ++step) {
      bool any = false;
      u32 vv[kPullV];
#pragma unroll
      for (int j = 0; j < kPullV; ++j) {
        vv[j] = kNone;
        if (e[j] < re[j]) {
          vv[j] = (step == 0 && a.first) ? f[j] : (u32)__ldg(a.col + e[j]);
          ++e[j];
          ++scanned;
          any = true;
        }
      }
      if (!any) break;
      u64 kv[kPullV];
#pragma unroll
      for (int j = 0; j < kPullV; ++j) kv[j] = (vv[j] < a.n) ? ld_cg_u64(a.key + vv[j]) : ~0ull;
#pragma unroll
      for (int j = 0; j < kPullV; ++j) {
        if ((u32)(kv[j] >> 32) == L) best[j] = min(best[j], kv[j] + kLevelOne);
        if (best[j] <= (lvl_key | fr[j])) re[j] = e[j];  // nothing can beat (L + 1, fr)
      }
    }
    // scans still going after kPullLong neighbours (hubs with no early exit):
    // the warp takes them one at a time, 32 x kPullCoop coalesced neighbours
    // per step, with the same early exit per step
#pragma unroll
    for (int j = 0; j < kPullV; ++j) {
      u32 lm = __ballot_sync(kFull, e[j] < re[j]);
      while (lm) {
        const int src = __ffs(lm) - 1;
        lm &= lm - 1;
        const int eb = __shfl_sync(kFull, e[j], src), ee = __shfl_sync(kFull, re[j], src);
        const u64 fj = lvl_key | __shfl_sync(kFull, fr[j], src);
        u64 b = __shfl_sync(kFull, best[j], src);
        int pos = eb;
        while (pos < ee) {
          u32 vq[kPullCoop];
#pragma unroll
          for (int q = 0; q < kPullCoop; ++q) {
            const int idx = pos + q * 32 + (int)lane;
            vq[q] = idx < ee ? (u32)__ldg(a.col + idx) : kNone;
          }
          u64 lb = ~0ull;
#pragma unroll
          for (int q = 0; q < kPullCoop; ++q) {
            const u64 kq = vq[q] < a.n ? ld_cg_u64(a.key + vq[q]) : ~0ull;
            if ((u32)(kq >> 32) == L) lb = min(lb, kq + kLevelOne);
          }
          b = min(b, warp_min64(lb));
          pos += 32 * kPullCoop;
          if (b <= fj) break;  // warp-uniform: nothing can beat (L + 1, minrank)
        }
        if ((int)lane == src) {
          best[j] = b;
          scanned += (u32)(min(pos, ee) - eb);
        }
      }
    }
    u64 kwn[kPullV];  // the next pass's keys and ranges, beside this pass's appends
    int en[kPullV], ren[kPullV];
    u32 fnn[kPullV];
    load_keys(wn, kwn, en, ren, fnn);
    u32 mask = 0, keep = 0, won = 0;
#pragma unroll
    for (int j = 0; j < kPullV; ++j) {
      const bool pending = w[j] != kNone && (u32)(kw[j] >> 32) > L;
      if (pending && best[j] < kw[j]) {
        a.key[w[j]] = best[j];  // only this thread writes key[w] in a bottom-up round
        won |= 1u << j;
        if ((u32)(kw[j] >> 32) > L + 1) mask |= 1u << j;
      }
      // still above level L + 1: examined again by a following bottom-up round
      if (pending && (u32)(min(best[j], kw[j]) >> 32) > L + 1) keep |= 1u << j;
    }
#pragma unroll
    for (int j = 0; j < kPullV; ++j)
      note_rank<U>(a, (u32)qi, (won >> j) & 1u, w[j], (u32)best[j], myrank, s_acc);
    pull_append<kPullV, LD>(mask, keep, w, rs0, re0, a, qi, qb, ulist_out, ucnt_out);
#pragma unroll
    for (int j = 0; j < kPullV; ++j) {
      w[j] = wn[j];
      kw[j] = kwn[j];
      e[j] = en[j];
      re[j] = ren[j];
      f[j] = fnn[j];
    }
    base = nbase;
    ++pass;
    nbase = pass + 1 < kd ? dealt_base(pass + 1) : (base < total ? unit_base(ticket) : total);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    scanned += __shfl_xor_sync(kFull, scanned, o);
    examined += __shfl_xor_sync(kFull, examined, o);
  }
  if (lane == 0) {
    if (scanned) atomicAdd(&a.ctl->pull_arcs, (u64)scanned);
    if (examined) atomicAdd(&a.ctl->pull_verts, (u64)examined);
  }
}

// U: a union of graphs (per-member bottom-up floors); a separate instance so
// that the plain kernel carries none of it.  kPerSm: the CTAs per SM the
// instance is built for.  One CTA per SM leaves it 128 registers per thread
// (no spills) and the cheapest grid barrier, the best for thin frontiers and
// single graphs; two give twice the warps, the best for the wide bottom-up
// rounds of many-seed unions.  The launch parameter bfs_blocks_per_sm picks
// the instance.
template <bool U, int kPerSm, bool LD>
__global__ void __launch_bounds__(kBfsThreads, kPerSm) k_bfs(BfsArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  // union with few enough members: per-member next-level minima and
  // current-level floors in shared memory, after Smem
  u32* s_acc = (U && a.kmem <= kSmemMembers)
                   ? reinterpret_cast<u32*>(smem_raw + sizeof(Smem) + (LD ? lq_extra(kPerSm) : 0))
                   : nullptr;
  u32* s_floor = s_acc ? s_acc + kSmemMembers : nullptr;
  if (s_acc)
    for (u32 m = threadIdx.x; m < a.kmem; m += blockDim.x) s_acc[m] = 0xffffffffu;
  Control* ctl = a.ctl;
  if (threadIdx.x == 0) {
    s.minrank = 0xffffffffu;
    s.stop = ld_acquire_u32(&ctl->err) != 0u ? 1u : 0u;  // validation failed upstream
  }
  __syncthreads();
  if (s.stop) return;  // CTA-uniform: read once by thread 0
  const int A = ctl->A;
  const u32 par_r = __popc(ctl->mask_r) & 1u;
  const u32* rk = a.rk[par_r];
  const u32* rv = a.rv[par_r];
  const u32 G = gridDim.x;
  u32 gen = 0;
  u32 myrank = 0xffffffffu;  // this thread's smallest successful next-level rank

  u64 pushed = 0;  // low-degree mode: arcs offered by this thread
  // Level 0: the vertices with the largest integer shift part start.
  if (LD) {
    const int lo = __ldg(a.bptr), hi = __ldg(a.bptr + 1);
    expand_ld<U>(a, nullptr, 0, 0, rv, lo, (u32)(hi - lo), 0, false, 0, 0, myrank, s_acc, pushed);
  } else {
    append_bucket<U>(a, 0, rv, 0, 0, myrank, s_acc);
  }
  post_cta_min(s, myrank);
  grid_barrier(ctl, gen, G, a.bar_phantom, a.spin_limit, 0, a.bptr, A >= 1 ? 1 : -1, s);
  const bool profiler = blockIdx.x == 0 && threadIdx.x == 0;
  if (profiler) {
    const long long t = clock64();
    ctl->round_clk[0][0] = ctl->round_clk[0][1] = ctl->round_clk[0][2] = t;
    ctl->round_kind[0] = kRoundSkip;
  }

  u64 settled = 0, edges = 0;
  u64 items = 0;     // vertices expanded (a window may expand a vertex twice)
  u64 expanded = 0;  // this thread's expansions inside windows
  u32 phase = 0, pulls = 0, nwin = 0, overflowed = 0;
  u32 wdepth = a.window_levels;  // levels of the next window
  u64 push_arcs = 0;
  int lvl = 0;
  bool pulling = false;
  bool windowed = false;  // a window has run: settled vertices are no longer counted exactly
  // No correct run needs more rounds than this (each round settles a level or
  // jumps to a start bucket); a loop that would is stopped with an error
  // instead of holding the GPU.
  const u64 max_rounds = 2ull * ((u64)a.n_active + (u64)A) + 1024;
  for (;;) {
    if (s.stop) break;  // set by the last barrier, the same for every thread of the CTA
    if (phase > max_rounds) {  // the same for every thread of every CTA
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->err, kErrInternal);
      break;
    }
    const u64 c = s.next_c;  // slot phase % 3, read as the last barrier released
    const int nb_lo = s.next_lo, nb_hi = s.next_hi;  // start bucket lvl + 1 (if lvl + 1 <= A)
    const u32 Q = (u32)(c >> 32);
    // overflow entries of the last window (more than n cannot have been written:
    // that sets kErrInternal, and the loop stops at the barrier)
    const u32 nov = LD ? min(s.next_ovf, a.n) : 0u;
    // low-degree mode keeps no arc count: the frontier's arcs are estimated
    // from the mean degree (direction choice and probe threshold only)
    const u32 E = LD ? (u32)min((u64)Q * a.nnz_active / max(a.n_active, 1u), 0xffffffffull)
                     : (u32)c;
    settled += Q;
    if (!windowed && settled >= a.n_active) break;  // every vertex the BFS owns has its final key
    const u32 minrank = s.next_minrank;
    const u32 ncand = s.next_ucnt;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      ctl->qctr[(phase + 2) % 3] = 0;
      ctl->minrank[(phase + 2) % 3] = 0xffffffffu;
      ctl->ucnt[(phase + 2) % 3] = 0;
      ctl->ovf[(phase + 2) % 3] = 0;
      ctl->nstart[(phase + 2) % 3] = 0;
      ctl->pull_ctr[(phase + 2) % 3] = 0;
    }
    if (U)  // the members' floors of the slot that the next round fills
      for (u32 m = blockIdx.x * blockDim.x + threadIdx.x; m < a.kmem; m += G * blockDim.x)
        a.mrank[(size_t)((phase + 2) % 3) * a.kmem + m] = 0xffffffffu;
    const int qi = (int)((phase + 1) % 3), qb = (int)((phase + 1) & 1);
    int nlvl;
    // a window of levels: low-degree rounds whose frontier is thin enough, and
    // always while overflow entries of the last window wait
    bool window = false;
    u32 H = 0;
    if (LD && a.window_levels > 1 && (nov > 0 || (Q > 0 && Q <= a.window_max_q))) {
      // The window's depth adapts: halved while the last window's local queues
      // overflowed by more than a quarter of the frontier, doubled again (up
      // to the tuning's) once nothing overflowed; and cut before the first
      // start bucket it would take in locally (buckets lvl + 1 .. H - 1) that
      // holds more than window_max_q vertices.  One level only drains the
      // overflow.  The same for every thread: nov, Q and bptr are.
      if (nov > (Q >> 2)) wdepth = max(wdepth >> 1, 1u);
      else if (nov == 0) wdepth = min(wdepth << 1, a.window_levels);
      u32 d = 1;
      for (; d < wdepth; ++d) {
        const int r = lvl + (int)d;
        if (r <= A && (u32)(__ldg(a.bptr + r + 1) - __ldg(a.bptr + r)) > a.window_max_q) break;
      }
      window = d > 1 || nov > 0;
      H = (u32)lvl + d;
    }
    if (window) {
      edges += E;
      pulling = false;
      window_ld<U, lq_cap(kPerSm)>(a, s, rv, A, Q, nov, (int)(phase & 1), (u32)lvl, H, qi, qb, myrank, s_acc,
                   pushed, expanded);
      if (profiler && phase + 1 < (u32)kRoundProfile) ctl->round_clk[phase + 1][0] = clock64();
      windowed = true;
      ++nwin;
      overflowed += nov;
      nlvl = (int)H;
    } else if (Q > 0) {
      items += Q;
      edges += E;
      const u64 unsettled_arcs = a.nnz_active > edges ? a.nnz_active - edges : 0;
      const bool was_pulling = pulling;
      if (!pulling && (u64)E * a.pull_alpha > unsettled_arcs &&
          (u64)E * a.pull_gamma > a.n_active)
        pulling = true;
      else if (pulling && (u64)Q * a.pull_beta < a.n_active)
        pulling = false;
      if (pulling) {
        if (U) {  // this level's per-member floors, from the frontier list
          member_floors(a, a.qv[phase & 1], Q, phase % 3, s_acc);
          if (s_acc) {
            __syncthreads();
            flush_members(a, phase % 3, s_acc);
          }
          grid_barrier(ctl, gen, G, a.bar_phantom, a.spin_limit, kNoPost, a.bptr, -1, s);
          if (s.stop) break;
          if (s_floor) {  // read once per CTA
            for (u32 m = threadIdx.x; m < a.kmem; m += blockDim.x)
              s_floor[m] = ld_cg_u32(a.mrank + (size_t)(phase % 3) * a.kmem + m);
            __syncthreads();
          }
        }
        pull_round<U, LD, pull_width(kPerSm)>(a, lvl, minrank, phase % 3, qi, qb, was_pulling,
                                              a.ulist[phase & 1], ncand, a.ulist[(phase + 1) & 1],
                                              &ctl->ucnt[qi], myrank, s_acc, s_floor);
        ++pulls;
        if (profiler && phase + 1 < (u32)kRoundProfile) ctl->round_clk[phase + 1][0] = clock64();
        if (lvl + 1 <= A) {
          if (LD) {
            expand_ld<U>(a, nullptr, 0, 0, rv, nb_lo, (u32)(nb_hi - nb_lo), (u32)lvl + 1, false,
                         qi, qb, myrank, s_acc, pushed);
          } else {
            append_bucket<U>(a, lvl + 1, rv, qi, qb, myrank, s_acc, nb_lo, nb_hi);
          }
        }
      } else if (LD) {  // expansion and start bucket lvl + 1 in one pass
        expand_ld<U>(a, a.qv[phase & 1], Q, (u32)lvl + 1, rv, nb_lo, (u32)(nb_hi - nb_lo),
                     (u32)lvl + 1, E >= a.probe_min_arcs, qi, qb, myrank, s_acc, pushed);
        if (profiler && phase + 1 < (u32)kRoundProfile) ctl->round_clk[phase + 1][0] = clock64();
      } else {
        expand<U>(a, s, (int)(phase & 1), Q, E, lvl, qi, qb, myrank, s_acc);
        push_arcs += E;
        if (profiler && phase + 1 < (u32)kRoundProfile) ctl->round_clk[phase + 1][0] = clock64();
        if (lvl + 1 <= A) append_bucket<U>(a, lvl + 1, rv, qi, qb, myrank, s_acc, nb_lo, nb_hi);
      }
      nlvl = lvl + 1;
    } else {
      if (lvl + 1 > A) break;
      int rr;
      if (windowed) {  // the next start level that still holds an unclaimed vertex
        scan_unclaimed(a, rk, rv, lvl + 1, A, phase % 3);
        grid_barrier(ctl, gen, G, a.bar_phantom, a.spin_limit, kNoPost, a.bptr, -1, s);
        if (s.stop) break;
        if (threadIdx.x == 0) s.nstart = ld_cg_u32(&ctl->nstart[phase % 3]);
        __syncthreads();
        if (s.nstart == 0u) break;  // none: every vertex the BFS owns is settled
        rr = (int)~s.nstart;
      } else {
        const int start = __ldg(a.bptr + lvl + 1);
        if ((u32)start >= a.n) break;
        rr = (int)__ldg(rk + start);  // next non-empty start bucket
        if (rr > A) break;            // only vertices the BFS does not handle remain
      }
      if (profiler && phase + 1 < (u32)kRoundProfile) ctl->round_clk[phase + 1][0] = clock64();
      if (LD) {
        const int lo = __ldg(a.bptr + rr), hi = __ldg(a.bptr + rr + 1);
        expand_ld<U>(a, nullptr, 0, 0, rv, lo, (u32)(hi - lo), (u32)rr, false, qi, qb, myrank,
                     s_acc, pushed);
      } else {
        append_bucket<U>(a, rr, rv, qi, qb, myrank, s_acc);
      }
      // this round left no unsettled list: a bottom-up round after it starts
      // from every vertex the loop owns
      pulling = false;
      nlvl = rr;
    }
    if (profiler && phase + 1 < (u32)kRoundProfile) ctl->round_clk[phase + 1][1] = clock64();
    post_cta_min(s, myrank);
    grid_barrier(ctl, gen, G, a.bar_phantom, a.spin_limit, (u32)qi, a.bptr,
                 nlvl + 1 <= A ? nlvl + 1 : -1, s);
    ++phase;
    lvl = nlvl;
    if (profiler && phase < (u32)kRoundProfile) {
      ctl->round_clk[phase][2] = clock64();
      ctl->round_kind[phase] = Q == 0 ? kRoundSkip : (pulling ? kRoundPull : kRoundPush);
    }
  }
  if (LD) {  // every thread's offered arcs (the estimate above is not a count) and expansions
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      pushed += __shfl_xor_sync(kFull, pushed, o);
      expanded += __shfl_xor_sync(kFull, expanded, o);
    }
    if ((threadIdx.x & 31) == 0 && pushed) atomicAdd(&ctl->push_arcs, pushed);
    if ((threadIdx.x & 31) == 0 && expanded) atomicAdd(&ctl->items, expanded);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->pull_rounds = pulls;
    if (!LD) ctl->push_arcs = push_arcs;
    ctl->rounds = phase;
    ctl->last_level = lvl;
    atomicAdd(&ctl->items, windowed ? items : settled);
    ctl->edges = edges;
    ctl->windows = nwin;
    ctl->overflowed = overflowed;
  }
}

}  // namespace

size_t bfs_smem_bytes() { return sizeof(Smem); }

namespace {
size_t bfs_smem(bool u, int per_sm, bool ld) {
  return sizeof(Smem) + (ld ? lq_extra(per_sm) : 0) + (u ? 2 * kSmemMembers * sizeof(u32) : 0);
}

const void* bfs_kernel(bool u, int per_sm, bool ld) {
  if (ld) {
    if (u) return per_sm >= 2 ? (const void*)k_bfs<true, 2, true> : (const void*)k_bfs<true, 1, true>;
    return per_sm >= 2 ? (const void*)k_bfs<false, 2, true> : (const void*)k_bfs<false, 1, true>;
  }
  if (u) return per_sm >= 2 ? (const void*)k_bfs<true, 2, false> : (const void*)k_bfs<true, 1, false>;
  return per_sm >= 2 ? (const void*)k_bfs<false, 2, false> : (const void*)k_bfs<false, 1, false>;
}
}  // namespace

int bfs_grid_size(int num_sms, int* blocks_per_sm) {
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !attr_set[dev]) {
    for (int u = 0; u < 2; ++u)
      for (int p = 1; p <= 2; ++p)
        for (int ld = 0; ld < 2; ++ld)
          cudaFuncSetAttribute(bfs_kernel(u != 0, p, ld != 0),
                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)bfs_smem(u != 0, p, ld != 0));
    attr_set[dev] = true;
  }
  // the most CTAs per SM (1 or 2) that every instance built for it reaches
  int per_sm = 2;
  for (int u = 0; u < 2; ++u)
    for (int p = 1; p <= 2; ++p)
      for (int ld = 0; ld < 2; ++ld) {
        int got = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&got, bfs_kernel(u != 0, p, ld != 0),
                                                          kBfsThreads, bfs_smem(u != 0, p, ld != 0)) !=
            cudaSuccess)
          return -1;
        if (got < 1) return -1;
        if (got < p) per_sm = min(per_sm, got);
      }
  *blocks_per_sm = per_sm;
  return per_sm * num_sms;
}

int launch_bfs(const BfsArgs& a, int grid, int per_sm, cudaStream_t s, cudaError_t* err) {
  BfsArgs copy = a;
  void* args[] = {&copy};
  *err = cudaLaunchCooperativeKernel(bfs_kernel(a.mrank != nullptr, per_sm, a.low_degree != 0),
                                     dim3(grid),
                                     dim3(kBfsThreads), args,
                                     bfs_smem(a.mrank != nullptr, per_sm, a.low_degree != 0), s);
  return *err == cudaSuccess ? 1 : -1;
}

}  // namespace ldd

// Start keys of the delayed-start BFS (Section 4 of Miller, Peng, Xu 2013).
//
//  1. split (Algorithm 1 step 2, Section 4): a_u = floor(delta_u),
//     f_u = delta_u - a_u (exact in FP64), A = max a_u = floor(delta_max).
//  2. fraction rank (Section 4: the fractional parts are tie-breakers within
//     an integer level and can be replaced by a permutation): rank_u = the
//     position of u in the order (f_u descending, u ascending), order[rank] = u.
//  3. keys: key_u = ((A - a_u) << 32) | rank_u, i.e. u's own start label at
//     round R_u = A - a_u.
//  4. start buckets (Section 4: the super-source edge of length L is looked at
//     when the frontier reaches distance L): the vertices the BFS handles,
//     grouped by R_u (any order inside a group); bptr[r] = start of group r,
//     r = 0 .. A + 1.
//
// Fraction rank, fast path (most-significant-digit bucketing): the bucket of u
// is the top B bits of ~floor(f_u * 2^32), which is monotone in f_u, with
// 2^B about n / 16 so that buckets hold ~16 vertices.  One pass over the
// shifts drops a 16-byte record (bits of f_u, a_u, u) into a free slot of its
// bucket (kSlotCap slots each); an exclusive scan of the bucket counts gives
// every bucket's first rank; tiles of buckets staged in shared memory then
// rank every member exactly by (f descending, u ascending) with the full FP64
// fractions, one thread per record, and write order[] and the keys directly.
// Vertices alone in their component are not ranked (their center is
// themselves).  A full bucket (crafted shifts, e.g. all fractions equal)
// makes the host redo the rank with the exact path: a stable LSD radix sort
// of the order-preserving bits of f (8 "onesweep" passes of 8 bits) over all
// vertices.
//
// Batches (disjoint unions of member graphs, k_union.cu): every member's
// floors are lifted by one integer, lift_s = max_t A_t - A_s, so that each
// member's own largest shift starts at round 0 and the members' rounds run in
// step.  A constant added to every level of one member changes no comparison
// inside that member, and members never compete.
//
// Start buckets: a counting sort by R_u (histogram while the keys are built,
// an exclusive scan that is bptr, and a scatter in which each CTA reserves its
// range of every group with one atomic).
#include <algorithm>

#include "ldd_internal.cuh"

namespace ldd {

namespace {

constexpr u32 kFull = 0xffffffffu;
constexpr u32 kSlotCap = 64;                  // record slots per fraction bucket (mean <= 16)
constexpr int kScanThreads = 256;
constexpr int kScanIpt = 16;
constexpr int kScanTile = kScanThreads * kScanIpt;
constexpr u32 kRBins = 4096;                  // start rounds counted in shared memory
constexpr int kRChunk = 16;                   // vertices per thread in the start-bucket scatter

__device__ __forceinline__ bool failed(const Control* ctl) {
  return *(volatile const u32*)&ctl->err != 0u;
}

// Adds one count per valid lane to sh[digit]: one atomic when the warp agrees.
__device__ __forceinline__ void hist_add(u32* sh, u32 digit, bool valid, u32 lane) {
  const u32 act = __ballot_sync(kFull, valid);
  if (act == 0) return;
  const int first = __ffs(act) - 1;
  const u32 d0 = __shfl_sync(kFull, digit, first);
  if (__all_sync(kFull, !valid || digit == d0)) {
    if ((int)lane == first) atomicAdd(&sh[d0], (u32)__popc(act));
  } else if (valid) {
    atomicAdd(&sh[digit], 1u);
  }
}

// Splits a shift d into a = floor(d) and the IEEE-754 bits of its fraction
// f = d - a (exact), with integer operations on d's bits only: FP64
// arithmetic is slow on this part and the split runs once per vertex.  The
// bits of a non-negative double order like its value, so fb orders the
// fractions.  d = -0 counts as +0.  NaN or d < 0 sets kErrShiftArg, d >= 2^31
// (or +inf) kErrShiftRange; a = 0 and fb = 0 then.
__device__ __forceinline__ void split_bits(double d, u32& err, int& a, u64& fb) {
  constexpr u64 kMan = (1ull << 52) - 1;
  const u64 b = (u64)__double_as_longlong(d);
  const u32 ex = (u32)(b >> 52) & 0x7ffu;
  a = 0;
  fb = 0;
  if (ex == 0x7ffu && (b & kMan) != 0) {  // NaN, either sign
    err |= kErrShiftArg;
  } else if (b >> 63) {                   // negative; -0 is +0
    if (b << 1) err |= kErrShiftArg;
  } else if (ex >= 1023u + 31u) {         // >= 2^31 or +inf
    err |= kErrShiftRange;
  } else if (ex < 1023u) {                // d < 1: a = 0, f = d
    fb = b;
  } else {
    const u32 E = ex - 1023u;             // d = M * 2^(E - 52), 0 <= E <= 30
    const u64 M = (b & kMan) | (1ull << 52);
    a = (int)(M >> (52 - E));
    const u64 fr = M & ((1ull << (52 - E)) - 1);  // f = fr * 2^(E - 52)
    if (fr) {
      const int p = 63 - __clzll((long long)fr);  // leading bit of fr: f in [2^(p+E-52), 2^(p+E-51))
      fb = ((u64)(p + (int)E - 52 + 1023) << 52) | ((fr << (52 - p)) & kMan);
    }
  }
}

__device__ __forceinline__ void finish_split(u32 err, int amax, Control* ctl) {
  __shared__ int s_amax;
  __shared__ u32 s_err;
  if (threadIdx.x == 0) {
    s_amax = 0;
    s_err = 0;
  }
  __syncthreads();
  if (err) atomicOr(&s_err, err);
  atomicMax(&s_amax, amax);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_err) atomicOr(&ctl->err, s_err);
    atomicMax(&ctl->A, s_amax);
  }
}

// ---------------------------------------------------------------- fast path
// Top B bits of ~floor(f * 2^32) for the fraction with bits fb: larger
// fractions get smaller buckets.  f = M * 2^(Ef - 52) with Ef <= -1, so
// floor(f * 2^32) = M >> (20 - Ef) < 2^32.
__device__ __forceinline__ u32 bucket_of(u64 fb, int B) {
  const u32 ef = (u32)(fb >> 52);
  const u64 M = (fb & ((1ull << 52) - 1)) | (ef ? (1ull << 52) : 0ull);
  const int Ef = ef ? (int)ef - 1023 : -1022;
  const int sh = 20 - Ef;
  const u32 code = sh >= 64 ? 0u : (u32)(M >> sh);
  return (~code) >> (32 - B);
}

// Pass 1, the only read of the shifts (vertices u0 .. n-1 per launch; one
// launch per chunk while the shifts are still arriving): split and validate
// every shift, and
// drop a record into the next free slot of u's bucket unless u is alone in
// its component.  Record: x = bits of f_u; y = (a_u << 32) | u, with bit 31
// set when the BFS does not handle u (u < 2^30).  Vertices the BFS handles are
// also counted by their floor a_u into acnt (the start-round histogram in
// reverse order; acnt is all zero on entry).  Each thread takes kPlaceIpt
// vertices per step so that their loads and slot atomics overlap: two below
// 2^24 vertices, four above (the single graphs gain from more resident warps,
// the larger unions from more loads in flight).  A full bucket sends the host
// to the exact path.
constexpr u32 kPlaceWideFrom = 1u << 24;

// Adds one to the count of floor value a for every lane with take set, one
// atomic per distinct a in the warp; floors below kRBins go to the CTA's
// shared histogram.  A floor beyond the table (a + 2 > cap) sets kErrBucketCap.
__device__ __forceinline__ void count_floor(int a, bool take, u32* sh, u32* acnt, u32 cap,
                                            u32& err) {
  const u32 act = __ballot_sync(kFull, take);
  if (!act) return;
  const u32 peers = __match_any_sync(kFull, take ? (u32)a : 0xffffffffu) & act;
  if (take && (peers & lanemask_lt()) == 0) {
    const u32 c = (u32)__popc(peers);
    if ((u32)a < kRBins) atomicAdd(&sh[a], c);
    else if ((u64)(u32)a + 2 <= cap) atomicAdd(acnt + a, c);
    else err |= kErrBucketCap;
  }
}

template <int kPlaceIpt>
__global__ void __launch_bounds__(256) k_bplace(const double* __restrict__ delta,
                                                const u32* __restrict__ solo,
                                                const u32* __restrict__ excl, u32 u0, u32 n,
                                                int B, u32* __restrict__ cnt,
                                                ulonglong2* __restrict__ slots,
                                                u32* acnt, u32 cap,
                                                const u32* __restrict__ wmem,
                                                const int* __restrict__ lift, Control* ctl) {
  __shared__ u32 sh[kRBins];
  const u32 tid = threadIdx.x, lane = tid & 31;
  for (u32 i = tid; i < kRBins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  int amax = 0;
  u32 err = 0;
  const u32 stride = gridDim.x * blockDim.x;
  // warp-uniform trip count: the histogram adds are warp collectives
  for (u32 wb = u0 + blockIdx.x * blockDim.x + (tid & ~31u); wb < n; wb += stride * kPlaceIpt) {
    double d[kPlaceIpt];
#pragma unroll
    for (int k = 0; k < kPlaceIpt; ++k) {
      const u32 u = wb + lane + (u32)k * stride;
      d[k] = (u < n) ? __ldcs(delta + u) : 0.0;
    }
    u32 bkt[kPlaceIpt], pos[kPlaceIpt];
    int fl[kPlaceIpt];
    bool own[kPlaceIpt];
    ulonglong2 rec[kPlaceIpt];
#pragma unroll
    for (int k = 0; k < kPlaceIpt; ++k) {
      const u32 u = wb + lane + (u32)k * stride;
      bkt[k] = 0xffffffffu;
      fl[k] = 0;
      own[k] = false;
      if (u < n) {
        u64 fb;
        split_bits(d[k], err, fl[k], fb);
        if (lift) fl[k] += __ldg(lift + __ldg(wmem + (u >> 5)));
        amax = max(amax, fl[k]);
        if (!((__ldg(solo + (u >> 5)) >> (u & 31)) & 1u)) {
          const u32 out = (__ldg(excl + (u >> 5)) >> (u & 31)) & 1u;
          own[k] = out == 0u;
          bkt[k] = bucket_of(fb, B);
          rec[k] = make_ulonglong2(fb, ((u64)(u32)fl[k] << 32) | u | (out << 31));
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kPlaceIpt; ++k) pos[k] = bkt[k] != 0xffffffffu ? atomicAdd(cnt + bkt[k], 1u) : 0u;
#pragma unroll
    for (int k = 0; k < kPlaceIpt; ++k) count_floor(fl[k], own[k], sh, acnt, cap, err);
#pragma unroll
    for (int k = 0; k < kPlaceIpt; ++k) {
      if (bkt[k] == 0xffffffffu) continue;
      if (pos[k] < kSlotCap) slots[(size_t)bkt[k] * kSlotCap + pos[k]] = rec[k];
      else err |= kErrRankRetry;
    }
  }
  __syncthreads();
  for (u32 i = tid; i < kRBins; i += blockDim.x)
    if (sh[i] && (u64)i + 2 <= cap) atomicAdd(acnt + i, sh[i]);
    else if (sh[i]) err |= kErrBucketCap;
  finish_split(err, amax, ctl);
}

// True if record o comes before record me in (f descending, id ascending).
__device__ __forceinline__ bool rec_before(const ulonglong2 o, const ulonglong2 me) {
  const u32 uo = (u32)o.y & 0x7fffffffu, um = (u32)me.y & 0x7fffffffu;
  return o.x > me.x || (o.x == me.x && uo < um);
}

// Writes what rank p of record rec gives: order[p] = u and u's start key
// ((A - a_u) << 32) | p.  Returns true if u goes into a start bucket (the BFS
// handles u).
__device__ __forceinline__ bool emit_key(bool valid, const ulonglong2 rec, u32 p, u32 n, int A,
                                         u32* __restrict__ order, u64* __restrict__ key) {
  const u32 u = (u32)rec.y & 0x7fffffffu;
  if (!(valid && p < n && u < n)) return false;
  const u32 R = (u32)(A - (int)(u32)(rec.y >> 32));
  order[p] = u;
  key[u] = ((u64)R << 32) | p;
  return !((u32)rec.y >> 31);
}

// Places u into start bucket R (bv[pos] = u, rk[pos] = R, pos from the
// bucket's global cursor), one atomic per distinct R in the warp.  Called by
// the whole warp.
__device__ __forceinline__ void place_start_warp(bool take, u32 u, u32 R, u32 n, u32* rcur,
                                                 u32* __restrict__ bv, u32* __restrict__ rk) {
  const u32 lane = threadIdx.x & 31;
  const u32 act = __ballot_sync(kFull, take);
  if (!act) return;
  const u32 peers = __match_any_sync(kFull, take ? R : 0xffffffffu) & act;
  const int leader = take ? __ffs(peers) - 1 : (int)lane;
  u32 base = 0;
  if (take && (int)lane == leader) base = atomicAdd(rcur + R, (u32)__popc(peers));
  base = __shfl_sync(kFull, base, leader);
  if (take) {
    const u32 pos = base + (u32)__popc(peers & lanemask_lt());
    if (pos < n) {
      bv[pos] = u;
      rk[pos] = R;
    }
  }
}

// Pass 2: CTAs take tiles of kTileBuckets consecutive buckets, in ticket
// order.  The tile's records (bucket b's len = start[b + 1] - start[b] records
// sit in slots [b * kSlotCap, b * kSlotCap + len)) are staged densely in
// shared memory in bucket order: first every position learns its bucket and
// the bucket's span of positions (one warp per bucket, shared memory only),
// then one thread per position copies its record.  Every thread then ranks
// one record against the members of its own bucket: rank = start[b] + the
// number of members before it in (f descending, id ascending), comparing the
// fraction bits alone unless another member has the same bits; and writes
// order[] and the key.  The tile's vertices then go into their start buckets:
// counted per start round in shared memory, one global reservation per round
// and tile, then written.  A tile with more than kTileRecs records (crowded
// fractions just short of a slot overflow) is ranked from global memory
// instead, and with more than kSortRBins start rounds the reservations are
// per warp.
constexpr u32 kTileBuckets = 64;   // <= threads per CTA (one capacity check each); < 256
constexpr u32 kTileRecs = 1280;    // < 2^16: spans are two 16-bit positions
constexpr u32 kSortRBins = 2048;
constexpr int kBsortPerSm = 5;     // resident CTAs per SM: 5 x 39 KB shared, <= 51 registers

struct BsortSmem {
  u64 fx[kTileRecs];         // fraction bits of the tile's records, bucket order
  u64 fy[kTileRecs];         // (a_u << 32) | u | (not handled by the BFS) << 31
  u32 span[kTileRecs];       // (first << 16) | end: the record's bucket as tile positions
  u32 loc[kTileRecs];        // record's offset within its start round's share of the tile
  u32 rc[kSortRBins];        // the tile's count per start round, then its base in the round
  u32 st[kTileBuckets + 1];  // global first rank of every bucket of the tile, and the end
  unsigned char bi[kTileRecs];  // record's bucket within the tile
  u32 tile;
};

__global__ void __launch_bounds__(256, kBsortPerSm)
    k_bsort(const u32* __restrict__ start, u32 nbkt, const ulonglong2* __restrict__ slots, u32 n,
            u32* __restrict__ order, u64* __restrict__ key, u32* rcur, u32* __restrict__ bv,
            u32* __restrict__ rk, u32* ticket, Control* ctl) {
  extern __shared__ __align__(16) unsigned char bsort_raw[];
  BsortSmem& sm = *reinterpret_cast<BsortSmem*>(bsort_raw);
  if (failed(ctl)) return;
  const int A = ctl->A;
  const bool small = (u32)A < kSortRBins;
  const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  if (small)
    for (u32 i = tid; i <= (u32)A; i += blockDim.x) sm.rc[i] = 0;
  const u32 ntiles = (nbkt + kTileBuckets - 1) / kTileBuckets;
  for (;;) {
    __syncthreads();  // previous tile done with sm
    if (tid == 0) sm.tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const u32 t = sm.tile;
    if (t >= ntiles) break;
    const u32 b0 = t * kTileBuckets;
    const u32 nb = min(kTileBuckets, nbkt - b0);
    for (u32 i = tid; i <= nb; i += blockDim.x) sm.st[i] = start[b0 + i];
    __syncthreads();
    // a bucket beyond kSlotCap cannot reach here (k_bplace flags it); checked anyway
    const bool full = tid < nb && sm.st[tid + 1] - sm.st[tid] > kSlotCap;
    const bool overfull = __syncthreads_or(full) != 0;
    const u32 total = sm.st[nb] - sm.st[0];
    if (!overfull && total <= kTileRecs) {
      for (u32 i = warp; i < nb; i += nwarp) {
        const u32 s0 = sm.st[i] - sm.st[0], e = sm.st[i + 1] - sm.st[0];
        for (u32 q = s0 + lane; q < e; q += 32) {
          sm.span[q] = (s0 << 16) | e;
          sm.bi[q] = (unsigned char)i;
        }
      }
      __syncthreads();
#pragma unroll 4
      for (u32 q = tid; q < total; q += blockDim.x) {
        const u32 i = sm.bi[q];
        const ulonglong2 rec = slots[(size_t)(b0 + i) * kSlotCap + (q - (sm.span[q] >> 16))];
        sm.fx[q] = rec.x;
        sm.fy[q] = rec.y;
      }
      __syncthreads();
      for (u32 q0 = 0; q0 < total; q0 += blockDim.x) {
        const u32 q = q0 + tid;
        const bool valid = q < total;
        ulonglong2 me = make_ulonglong2(0ull, 0ull);
        u32 p = 0;
        if (valid) {
          me = make_ulonglong2(sm.fx[q], sm.fy[q]);
          const u32 sp = sm.span[q], lo = sp >> 16, hi = sp & 0xffffu;
          u32 r = 0, eq = 0;
          for (u32 j = lo; j < hi; ++j) {
            const u64 x = sm.fx[j];
            r += x > me.x ? 1u : 0u;
            eq += x == me.x ? 1u : 0u;
          }
          if (eq > 1) {  // another member with the same fraction: the smaller id goes first
            const u32 um = (u32)me.y & 0x7fffffffu;
            for (u32 j = lo; j < hi; ++j)
              r += (sm.fx[j] == me.x && ((u32)sm.fy[j] & 0x7fffffffu) < um) ? 1u : 0u;
          }
          p = sm.st[0] + lo + r;
        }
        const bool take = emit_key(valid, me, p, n, A, order, key);
        const u32 R = (u32)(A - (int)(u32)(me.y >> 32));
        if (small) {
          if (take) sm.loc[q] = atomicAdd(&sm.rc[R], 1u);
        } else {
          place_start_warp(take, (u32)me.y & 0x7fffffffu, R, n, rcur, bv, rk);
        }
      }
      if (small) {
        __syncthreads();
        for (u32 i = tid; i <= (u32)A; i += blockDim.x) {
          const u32 c = sm.rc[i];
          sm.rc[i] = c ? atomicAdd(rcur + i, c) : 0u;  // this tile's base in round i
        }
        __syncthreads();
        for (u32 q = tid; q < total; q += blockDim.x) {
          const u64 y = sm.fy[q];
          const u32 u = (u32)y & 0x7fffffffu;
          if (((u32)y >> 31) || u >= n) continue;
          const u32 R = (u32)(A - (int)(u32)(y >> 32));
          const u32 pos = sm.rc[R] + sm.loc[q];
          if (pos < n) {
            bv[pos] = u;
            rk[pos] = R;
          }
        }
        __syncthreads();
        for (u32 i = tid; i <= (u32)A; i += blockDim.x) sm.rc[i] = 0;
      }
    } else {
      // one warp per bucket, records read from global memory
      for (u32 i = warp; i < nb; i += nwarp) {
        const u32 s0 = sm.st[i], len = sm.st[i + 1] - sm.st[i];
        if (len > kSlotCap) continue;  // cannot happen: k_bplace flags a full bucket
        const ulonglong2* bs = slots + (size_t)(b0 + i) * kSlotCap;
        for (u32 i0 = 0; i0 < len; i0 += 32) {
          const u32 q = i0 + lane;
          const bool valid = q < len;
          const ulonglong2 me = valid ? bs[q] : make_ulonglong2(0ull, 0ull);
          u32 r = 0;
          for (u32 j = 0; j < len; ++j) r += rec_before(bs[j], me) ? 1u : 0u;
          const bool take = emit_key(valid, me, s0 + r, n, A, order, key);
          place_start_warp(take, (u32)me.y & 0x7fffffffu, (u32)(A - (int)(u32)(me.y >> 32)), n,
                           rcur, bv, rk);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- exact path
__global__ void __launch_bounds__(256) k_split64(const double* __restrict__ delta, u32 n,
                                                 int* __restrict__ a_out, u64* __restrict__ kout,
                                                 u32* __restrict__ vout,
                                                 const u32* __restrict__ wmem,
                                                 const int* __restrict__ lift, Control* ctl) {
  __shared__ u32 sh[kFracDigits][256];
  const u32 tid = threadIdx.x, lane = tid & 31;
  for (u32 i = tid; i < kFracDigits * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  int amax = 0;
  u32 err = 0;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 base = blockIdx.x * blockDim.x + (tid & ~31u); base < n; base += stride) {
    const u32 idx = base + lane;
    const bool valid = idx < n;
    u64 key = 0;
    if (valid) {
      int a;
      u64 fb;
      split_bits(delta[idx], err, a, fb);
      if (lift) a += __ldg(lift + __ldg(wmem + (idx >> 5)));
      key = ~fb;  // ascending key: f descending
      a_out[idx] = a;
      kout[idx] = key;
      vout[idx] = idx;
      amax = max(amax, a);
    }
#pragma unroll
    for (int dg = 0; dg < kFracDigits; ++dg)
      hist_add(sh[dg], (u32)(key >> (8 * dg)) & 255u, valid, lane);
  }
  __syncthreads();
  for (u32 i = tid; i < kFracDigits * 256; i += blockDim.x) {
    const u32 c = (&sh[0][0])[i];
    if (c) atomicAdd(&(&ctl->hist_f[0][0])[i], c);
  }
  finish_split(err, amax, ctl);
}

// Exclusive offsets of every digit histogram; a digit whose keys all share
// one value needs no pass.  One CTA of 256 threads.
__global__ void __launch_bounds__(256) k_scan_digits(const u32* __restrict__ hist,
                                                     u32* __restrict__ off, u32* mask, int ndig,
                                                     u32 n) {
  __shared__ u32 s_warp[8];
  __shared__ int s_const;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  u32 m = 0;
  for (int d = 0; d < ndig; ++d) {
    const u32 h = hist[d * 256 + t];
    if (t == 0) s_const = 0;
    __syncthreads();
    if (h == n) s_const = 1;
    u32 x = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    u32 wbase = 0;
    for (int i = 0; i < w; ++i) wbase += s_warp[i];
    off[d * 256 + t] = wbase + x - h;
    if (!s_const) m |= 1u << d;
    __syncthreads();
  }
  if (t == 0) *mask = (n == 0) ? 0u : m;
}

constexpr int kSortWarps = kSortThreads / 32;

struct SortSmem {
  u64 keys[kSortTile];         // the tile, staged in sorted order for the write-out
  u32 vals[kSortTile];
  u32 whist[kSortWarps][256];  // per-warp digit counts, then per-warp offsets
  u32 tile_excl[256];          // start of each digit's run inside the tile
  u32 base[256];               // global start of this tile's run of each digit
  u32 wsum[kSortWarps];
  u32 tile;
  u32 bad;
};

// One stable LSD pass on digit `pass` (bits shift..shift+7) of 64-bit keys.
// Buffers are a ping-pong pair; the input side is the parity of the passes run
// before.  Each 4096-key tile ranks its keys per digit in shared memory with
// warp match, finds its global offsets by decoupled look-back over the
// preceding tiles, and writes each digit's run out contiguously.
__global__ void __launch_bounds__(kSortThreads) k_onesweep(
    u64* __restrict__ k0, u32* __restrict__ v0, u64* __restrict__ k1, u32* __restrict__ v1, u32 n,
    int pass, int shift, const u32* __restrict__ mask_ptr, const u32* __restrict__ digit_off,
    u64* __restrict__ status, u32* __restrict__ tile_ctr, u32 epoch, u32* err, u32 spin_limit) {
  const u32 mask = *mask_ptr;
  if (!((mask >> pass) & 1u) || *(volatile u32*)err != 0u) return;
  const int par = __popc(mask & ((1u << pass) - 1u)) & 1;
  const u64* kin = par ? k1 : k0;
  const u32* vin = par ? v1 : v0;
  u64* kout = par ? k0 : k1;
  u32* vout = par ? v0 : v1;

  extern __shared__ __align__(16) unsigned char sort_smem_raw[];
  SortSmem& sm = *reinterpret_cast<SortSmem*>(sort_smem_raw);
  const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    sm.tile = atomicAdd(tile_ctr, 1u);
    sm.bad = 0;
  }
  for (u32 i = tid; i < kSortWarps * 256; i += kSortThreads) (&sm.whist[0][0])[i] = 0;
  __syncthreads();
  const u32 tile = sm.tile;
  const u32 tile0 = tile * kSortTile;
  const u32 base = tile0 + warp * (32 * kSortIpt);

  u64 key[kSortIpt];
  u32 val[kSortIpt];
  u32 rk[kSortIpt];
#pragma unroll
  for (int k = 0; k < kSortIpt; ++k) {
    const u32 idx = base + k * 32 + lane;
    key[k] = (idx < n) ? kin[idx] : 0ull;
    val[k] = (idx < n) ? vin[idx] : 0u;
  }
  const u32 lt = lanemask_lt();
#pragma unroll
  for (int k = 0; k < kSortIpt; ++k) {
    const u32 idx = base + k * 32 + lane;
    const bool valid = idx < n;
    const u32 dg = (u32)(key[k] >> shift) & 255u;
    const u32 d = valid ? dg : 256u + lane;
    const u32 peers = __match_any_sync(kFull, d);
    const u32 cnt = valid ? sm.whist[warp][dg] : 0u;
    rk[k] = cnt + __popc(peers & lt);
    __syncwarp();
    if (valid && (peers & lt) == 0) sm.whist[warp][dg] = cnt + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  const u32 dg = tid;  // thread tid owns digit tid
  u32 run = 0;
#pragma unroll
  for (int w = 0; w < kSortWarps; ++w) {
    const u32 c = sm.whist[w][dg];
    sm.whist[w][dg] = run;
    run += c;
  }
  u64* mine = status + (u64)tile * 256 + dg;
  const u64 tag = (u64)epoch << 32;
  if (tile == 0) st_volatile_u64(mine, tag | (2ull << 30) | run);
  else st_volatile_u64(mine, tag | (1ull << 30) | run);
  {
    u32 x = run;  // exclusive scan of the digit totals over the tile
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(kFull, x, o);
      if (lane >= (u32)o) x += y;
    }
    if (lane == 31) sm.wsum[warp] = x;
    __syncthreads();
    u32 pre = 0;
    for (u32 w = 0; w < warp; ++w) pre += sm.wsum[w];
    sm.tile_excl[dg] = pre + x - run;
  }
  u32 excl = 0;
  if (tile > 0) {
    int p = (int)tile - 1;
    u32 spins = 0;
    while (p >= 0) {
      const u64 sv = ld_volatile_u64(status + (u64)p * 256 + dg);
      if ((u32)(sv >> 32) != epoch) {
        if (++spins > spin_limit) {
          atomicOr(err, kErrTimeout);
          sm.bad = 1;
          break;
        }
        if (spins > 16) __nanosleep(64);
        continue;
      }
      excl += (u32)sv & 0x3fffffffu;
      if ((((u32)sv) >> 30) == 2u) break;
      --p;
    }
    st_volatile_u64(mine, tag | (2ull << 30) | (excl + run));
  }
  sm.base[dg] = digit_off[dg] + excl;
  __syncthreads();
  if (sm.bad) return;  // offsets unknown: write nothing
#pragma unroll
  for (int k = 0; k < kSortIpt; ++k) {
    const u32 idx = base + k * 32 + lane;
    if (idx < n) {
      const u32 d = (u32)(key[k] >> shift) & 255u;
      const u32 local = sm.tile_excl[d] + sm.whist[warp][d] + rk[k];
      sm.keys[local] = key[k];
      sm.vals[local] = val[k];
    }
  }
  __syncthreads();
  const u32 tile_n = min((u32)kSortTile, n - tile0);
  for (u32 i = tid; i < tile_n; i += kSortThreads) {
    const u64 kv = sm.keys[i];
    const u32 d = (u32)(kv >> shift) & 255u;
    const u32 pos = sm.base[d] + (i - sm.tile_excl[d]);
    if (pos < n) {
      kout[pos] = kv;
      vout[pos] = sm.vals[i];
    }
  }
}

// order[p] = u and rank[u] = p for the sorted fraction order (exact path).
__global__ void __launch_bounds__(256) k_rank_scatter(const u32* __restrict__ v0,
                                                      const u32* __restrict__ v1, Control* ctl,
                                                      u32 n, u32* __restrict__ order,
                                                      u32* __restrict__ rank) {
  if (failed(ctl)) return;
  const u32* vals = (__popc(ctl->mask_f) & 1u) ? v1 : v0;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    u32 u = vals[p];
    if (u >= n) {  // cannot happen for a permutation; never index with it
      atomicOr(&ctl->err, kErrInternal);
      u = 0;
    }
    order[p] = u;
    rank[u] = p;
  }
}

// ---------------------------------------------------------------- device scan
// In-place exclusive scan of data[0 .. len), single pass with decoupled
// look-back over 4096-element tiles.  len = A + 2 when len_from_A (the
// start-round histogram), else len_host.  With rev_src (fast path), the input
// is the floor histogram read in reverse, data[r] = rev_src[A - r] for
// r = 0 .. A and 0 for r = A + 1, and rev_src is cleared on the way (all zero
// for the next decomposition); a table of fewer than A + 2 entries (cap) sets
// kErrBucketCap.  Optionally copies the result to copy[] and records the
// largest input value in *maxv.  Tiles take tickets in order, so every tile's
// predecessors are running or done; every wait is bounded (spin_limit polls,
// then kErrTimeout).  One warp looks back over 32 predecessor tiles at a time.
// stall = 1 makes tile 0 wait, like the others, on a predecessor that does not
// exist, so that every look-back runs out of polls (tests of the timeout path).
__global__ void __launch_bounds__(kScanThreads) k_scan_excl(u32* data, u32* copy, u32 len_host,
                                                            int len_from_A, u64* __restrict__ status,
                                                            u32 epoch, u32* tile_ctr, u32* maxv,
                                                            u32* rev_src, u32 cap, Control* ctl,
                                                            u32 spin_limit, u32 stall) {
  __shared__ u32 s_tile, s_excl, s_bad;
  __shared__ u32 s_wsum[kScanThreads / 32];
  __shared__ u32 s_wmax[kScanThreads / 32];
  if (failed(ctl)) {
    // an upstream error skips the scan; the floor counts are still cleared, so
    // a decomposition queued behind this one starts from zero counts
    if (rev_src) {
      const u32 end = (u32)min((u64)(u32)ctl->A + 1, (u64)cap);
      for (u32 r = blockIdx.x * blockDim.x + threadIdx.x; r < end; r += gridDim.x * blockDim.x)
        rev_src[r] = 0;
    }
    return;
  }
  const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(tile_ctr, 1u);
    s_bad = 0;
    s_excl = 0;
  }
  __syncthreads();
  const u32 tile = s_tile;
  const int A = ctl->A;
  if (rev_src && (u64)A + 2 > cap) {
    if (tile == 0 && tid == 0) atomicOr(&ctl->err, kErrBucketCap);
    for (u32 r = tile * kScanTile + tid; r < min(cap, (tile + 1) * kScanTile); r += blockDim.x)
      rev_src[r] = 0;  // cleared as above
    return;
  }
  const u32 len = len_from_A ? (u32)A + 2u : len_host;
  const u32 t0 = tile * kScanTile;
  if (t0 >= len) return;  // tiles past the end: no later tile needs them
  const u32 my0 = t0 + tid * kScanIpt;
  u32 v[kScanIpt];
  u32 tot = 0, mx = 0;
#pragma unroll
  for (int i = 0; i < kScanIpt; ++i) {
    const u32 r = my0 + i;
    if (rev_src) {
      v[i] = 0;
      if (r <= (u32)A) {
        v[i] = rev_src[(u32)A - r];
        rev_src[(u32)A - r] = 0;
      }
    } else {
      v[i] = (r < len) ? data[r] : 0u;
    }
    tot += v[i];
    mx = max(mx, v[i]);
  }
  u32 x = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(kFull, x, o);
    if (lane >= (u32)o) x += y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  if (lane == 31) s_wsum[warp] = x;
  if (lane == 0) s_wmax[warp] = mx;
  __syncthreads();
  u32 wpre = 0, tile_tot = 0, tile_max = 0;
  for (u32 w = 0; w < kScanThreads / 32; ++w) {
    if (w < warp) wpre += s_wsum[w];
    tile_tot += s_wsum[w];
    tile_max = max(tile_max, s_wmax[w]);
  }
  if (warp == 0) {
    const u64 tag = (u64)epoch << 32;
    u64* mine = status + tile;
    if (tile == 0 && !stall) {
      if (lane == 0) st_volatile_u64(mine, tag | (2ull << 30) | tile_tot);
    } else {
      if (lane == 0) st_volatile_u64(mine, tag | (1ull << 30) | tile_tot);
      u32 excl = 0;
      int p = (int)tile - 1;
      u32 spins = 0;
      bool bad = false;
      while (p >= 0 || stall) {
        // lane l looks at tile p - l; "before tile 0" counts as an inclusive
        // prefix of 0 (with stall: as a tile that never reports)
        const int q = p - (int)lane;
        const u64 sv = (q >= 0) ? ld_volatile_u64(status + q) : (stall ? 0ull : (tag | (2ull << 30)));
        const bool ready = (u32)(sv >> 32) == epoch;
        const bool pref = ready && ((((u32)sv) >> 30) == 2u);
        const u32 pmask = __ballot_sync(kFull, pref);
        const u32 limit = pmask ? (u32)(__ffs(pmask) - 1) : 31u;  // lanes 0..limit are needed
        const u32 rmask = __ballot_sync(kFull, ready);
        const u32 need = (limit == 31u) ? kFull : ((2u << limit) - 1u);
        if ((rmask & need) != need) {
          if (++spins > spin_limit) {
            bad = true;
            break;
          }
          if (spins > 16) __nanosleep(64);
          continue;
        }
        u32 val = (lane <= limit) ? ((u32)sv & 0x3fffffffu) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(kFull, val, o);
        excl += val;
        if (pmask) break;
        p -= 32;
      }
      if (lane == 0) {
        if (bad) {
          atomicOr(&ctl->err, kErrTimeout);
          s_bad = 1;
        } else {
          st_volatile_u64(mine, tag | (2ull << 30) | (excl + tile_tot));
        }
        s_excl = excl;
      }
    }
  }
  __syncthreads();
  if (s_bad) return;
  if (tid == 0 && maxv && tile_max) atomicMax(maxv, tile_max);
  u32 run = s_excl + wpre + x - tot;
#pragma unroll
  for (int i = 0; i < kScanIpt; ++i) {
    if (my0 + i < len) {
      data[my0 + i] = run;
      if (copy) copy[my0 + i] = run;
    }
    run += v[i];
  }
}

// ---------------------------------------------------------------- keys and start buckets
__global__ void __launch_bounds__(256) k_zero_rounds(int* bptr, u32 cap, Control* ctl) {
  if (failed(ctl)) return;
  if ((u64)ctl->A + 2 > cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->err, kErrBucketCap);
    return;
  }
  const u32 len = (u32)ctl->A + 2u;
  for (u32 r = blockIdx.x * blockDim.x + threadIdx.x; r < len; r += gridDim.x * blockDim.x)
    bptr[r] = 0;
}

// In vertex order: key_u = ((A - a_u) << 32) | rank_u, and the count of every
// start round R_u among the vertices the BFS handles (into rcnt).
__global__ void __launch_bounds__(256) k_keys(const int* __restrict__ a,
                                              const u32* __restrict__ rank,
                                              const u32* __restrict__ excl, Control* ctl, u32 n,
                                              u64* __restrict__ key, u32* rcnt) {
  __shared__ u32 sh[kRBins];
  if (failed(ctl)) return;
  const int A = ctl->A;
  const bool small = (u32)A + 1u <= kRBins;
  const u32 tid = threadIdx.x, lane = tid & 31;
  if (small)
    for (u32 i = tid; i <= (u32)A; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 base = blockIdx.x * blockDim.x + (tid & ~31u); base < n; base += stride) {
    const u32 u = base + lane;
    bool count = false;
    u32 R = 0;
    if (u < n) {
      R = (u32)(A - a[u]);
      key[u] = ((u64)R << 32) | rank[u];
      count = !(excl[u >> 5] >> (u & 31) & 1u);
    }
    const u32 act = __ballot_sync(kFull, count);
    if (act) {
      const u32 peers = __match_any_sync(kFull, count ? R : 0xffffffffu) & act;
      if (count && (peers & lanemask_lt()) == 0) {
        const u32 c = __popc(peers);
        if (small) atomicAdd(&sh[R], c);
        else atomicAdd(rcnt + R, c);
      }
    }
  }
  __syncthreads();
  if (small)
    for (u32 i = tid; i <= (u32)A; i += blockDim.x)
      if (sh[i]) atomicAdd(rcnt + i, sh[i]);
}

// Start-bucket scatter: bv[pos] = u, rk[pos] = R_u for every vertex the BFS
// handles.  With few rounds, each CTA counts its chunk in shared memory and
// reserves its range of every group with one atomic; otherwise one atomic per
// warp and round.
__global__ void __launch_bounds__(256) k_rscatter(const int* __restrict__ a,
                                                  const u32* __restrict__ excl, Control* ctl,
                                                  u32 n, u32* cursor, u32* __restrict__ bv,
                                                  u32* __restrict__ rk) {
  __shared__ u32 s_cnt[kRBins];
  if (failed(ctl)) return;
  const int A = ctl->A;
  const bool small = (u32)A + 1u <= kRBins;
  const u32 tid = threadIdx.x, lane = tid & 31;
  const u32 chunk = blockDim.x * kRChunk;
  for (u32 c0 = blockIdx.x * chunk; c0 < n; c0 += gridDim.x * chunk) {
    if (small) {
      for (u32 i = tid; i <= (u32)A; i += blockDim.x) s_cnt[i] = 0;
      __syncthreads();
    }
    u32 R[kRChunk];
    u32 local[kRChunk];
#pragma unroll
    for (int k = 0; k < kRChunk; ++k) {
      const u32 u = c0 + (u32)k * blockDim.x + tid;
      bool take = false;
      R[k] = 0xffffffffu;
      if (u < n) {
        take = !(excl[u >> 5] >> (u & 31) & 1u);
        if (take) R[k] = (u32)(A - a[u]);
      }
      local[k] = 0;
      const u32 act = __ballot_sync(kFull, take);
      if (act) {
        const u32 peers = __match_any_sync(kFull, R[k]) & act;
        const int leader = take ? __ffs(peers) - 1 : (int)lane;
        u32 got = 0;
        if (take && (int)lane == leader)
          got = small ? atomicAdd(&s_cnt[R[k]], (u32)__popc(peers))
                      : atomicAdd(cursor + R[k], (u32)__popc(peers));
        got = __shfl_sync(kFull, got, leader);
        local[k] = got + __popc(peers & lanemask_lt());
      }
    }
    if (small) {
      __syncthreads();
      for (u32 i = tid; i <= (u32)A; i += blockDim.x) {
        const u32 c = s_cnt[i];
        s_cnt[i] = c ? atomicAdd(cursor + i, c) : 0u;  // this chunk's base in group i
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kRChunk; ++k) {
      const u32 u = c0 + (u32)k * blockDim.x + tid;
      if (R[k] != 0xffffffffu) {
        const u32 pos = (small ? s_cnt[R[k]] : 0u) + local[k];
        if (pos < n) {
          bv[pos] = u;
          rk[pos] = R[k];
        }
      }
    }
    if (small) __syncthreads();
  }
}

// ---------------------------------------------------------------- ranked variant
// Section 4: the fractional parts of the shifts only order the vertices of one
// integer level, and a random permutation of the vertices can stand in for
// them.  Input: the integer parts a_u (levels[u] >= 0) and the permutation
// (perm[u] = u's tie-break position, smaller first).  The rank is perm itself;
// order[perm[u]] = u, with a duplicate position detected by the exchange
// (order is all ones on entry).  Bad input sets kErrPermArg.
__global__ void __launch_bounds__(256) k_ranked_split(const int* __restrict__ levels,
                                                      const int* __restrict__ perm, u32 n,
                                                      int* __restrict__ a_out, u32* order,
                                                      Control* ctl) {
  int amax = 0;
  u32 err = 0;
  for (u32 u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const int a = levels[u];
    const int p = perm[u];
    if (a < 0 || p < 0 || (u32)p >= n) {
      err |= kErrPermArg;
      a_out[u] = 0;
      continue;
    }
    a_out[u] = a;
    amax = max(amax, a);
    if (atomicExch(order + p, u) != 0xffffffffu) err |= kErrPermArg;  // p taken twice
  }
  finish_split(err, amax, ctl);
}

u32 grid_stride_blocks(u32 n, int num_sms) {
  return (u32)max(1ll, min((long long)(n + 255) / 256, (long long)num_sms * 8));
}

void allow_bsort_smem() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  if (!done[dev]) {
    cudaFuncSetAttribute(k_bsort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(BsortSmem));
    done[dev] = true;
  }
}

// CTAs of a k_bplace instance resident on one SM: its grid is one full wave.
int bplace_blocks_per_sm(bool wide) {
  static int per_sm[2][64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 4;
  int& b = per_sm[wide ? 1 : 0][dev];
  if (b <= 0) {
    const void* fn = wide ? (const void*)k_bplace<4> : (const void*)k_bplace<2>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, 256, 0) != cudaSuccess || b < 1) {
      cudaGetLastError();
      b = 4;
    }
  }
  return b;
}

void allow_sort_smem() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  if (!done[dev]) {
    cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(SortSmem));
    done[dev] = true;
  }
}

}  // namespace

u32 fraction_bucket_bits(u32 n) {
  u32 b = 1;
  while (b < 26 && (1ull << (b + 4)) < n) ++b;  // about 16 vertices per bucket
  return b;
}

size_t rank_status_words(u32 n, u32 bptr_cap) {
  const u32 nbkt = 1u << fraction_bucket_bits(n);
  return std::max<size_t>((nbkt + 1 + kScanTile - 1) / kScanTile,
                          ((size_t)bptr_cap + kScanTile - 1) / kScanTile);
}

size_t fraction_slot_bytes(u32 n) {
  return ((size_t)1 << fraction_bucket_bits(n)) * kSlotCap * sizeof(ulonglong2);
}

int launch_rank_and_buckets(const RankBufs& r, bool exact64, cudaStream_t s,
                            const ShiftChunks* chunks) {
  const u32 n = r.n;
  Control* ctl = r.ctl;
  const u32 gs = grid_stride_blocks(n, r.num_sms);
  int launches = 0;
  const u32 rtiles = (r.bptr_cap + kScanTile - 1) / kScanTile;
  u32* rcnt = reinterpret_cast<u32*>(r.bptr);
  if (!exact64) {
    // split + records + floor counts; bucket starts; round counts (the scan
    // below makes them bptr); ranks, keys and the start buckets in one pass
    const u32 B = fraction_bucket_bits(n), nbkt = 1u << B;
    u32* cnt = reinterpret_cast<u32*>(r.k1);  // [nbkt + 1] counts, then first ranks
    ulonglong2* slots = reinterpret_cast<ulonglong2*>(r.slots);
    if (r.acnt_dirty) cudaMemsetAsync(r.acnt, 0, (size_t)r.bptr_cap * 4, s);
    cudaMemsetAsync(cnt, 0, (size_t)(nbkt + 1) * 4, s);
    const int nchunk = chunks ? chunks->n : 0;
    u32 lo = 0;
    for (int c = 0; c <= nchunk; ++c) {
      // chunk c is vertices [lo, hi), complete once its event has fired
      const u32 hi = c < nchunk ? std::min(chunks->end[c], n) : n;
      if (c < nchunk) cudaStreamWaitEvent(s, chunks->ev[c], 0);
      if (hi <= lo) continue;
      const u32 m = hi - lo;
      const bool wide = n >= kPlaceWideFrom;
      const int ipt = wide ? 4 : 2;
      const u32 place_grid =
          (u32)min((long long)(m + 256 * ipt - 1) / (256 * ipt),
                   (long long)r.num_sms * bplace_blocks_per_sm(wide));
      if (wide)
        k_bplace<4><<<max(place_grid, 1u), 256, 0, s>>>(r.shift, r.solo, r.excl, lo, hi, (int)B,
                                                        cnt, slots, r.acnt, r.bptr_cap, r.wmem,
                                                        r.lift, ctl);
      else
        k_bplace<2><<<max(place_grid, 1u), 256, 0, s>>>(r.shift, r.solo, r.excl, lo, hi, (int)B,
                                                        cnt, slots, r.acnt, r.bptr_cap, r.wmem,
                                                        r.lift, ctl);
      ++launches;
      lo = hi;
    }
    k_scan_excl<<<(nbkt + 1 + kScanTile - 1) / kScanTile, kScanThreads, 0, s>>>(
        cnt, nullptr, nbkt + 1, 0, r.status, ++(*r.epoch), &ctl->tile_ctr[0], nullptr, nullptr, 0,
        ctl, r.lookback_limit, r.stall_lookback);
    k_scan_excl<<<rtiles, kScanThreads, 0, s>>>(rcnt, r.rcur, 0, 1, r.status, ++(*r.epoch),
                                                 &ctl->tile_ctr[1], nullptr, r.acnt, r.bptr_cap,
                                                 ctl, r.lookback_limit, r.stall_lookback);
    allow_bsort_smem();
    const u32 ntiles = (nbkt + kTileBuckets - 1) / kTileBuckets;
    const u32 sort_grid = (u32)min((long long)ntiles, (long long)r.num_sms * kBsortPerSm);
    k_bsort<<<sort_grid, 256, sizeof(BsortSmem), s>>>(
        cnt, nbkt, slots, n, r.order, r.key, r.rcur, r.v0, reinterpret_cast<u32*>(r.k0),
        &ctl->tile_ctr[kFracDigits + kRoundDigits - 1], ctl);
    return launches + 3;
  }
  // exact path: stable LSD radix sort of all fractions, then keys and the
  // start-round counting sort (groups in any order inside)
  u32* rank = reinterpret_cast<u32*>(r.k1) + n;  // k1 holds 2 max(n, 64) 32-bit words
  if (chunks)
    for (int c = 0; c < chunks->n; ++c) cudaStreamWaitEvent(s, chunks->ev[c], 0);
  allow_sort_smem();
  k_split64<<<gs, 256, 0, s>>>(r.shift, n, r.a, r.k0, r.v0, r.wmem, r.lift, ctl);
  k_scan_digits<<<1, 256, 0, s>>>(&ctl->hist_f[0][0], &ctl->off_f[0][0], &ctl->mask_f,
                                  kFracDigits, n);
  launches += 2;
  const u32 ntiles = (n + kSortTile - 1) / kSortTile;
  for (int d = 0; d < kFracDigits; ++d) {
    k_onesweep<<<ntiles, kSortThreads, sizeof(SortSmem), s>>>(
        r.k0, r.v0, r.k1, r.v1, n, d, 8 * d, &ctl->mask_f, ctl->off_f[d], r.status,
        &ctl->tile_ctr[2 + d], ++(*r.epoch), &ctl->err, r.lookback_limit);
    ++launches;
  }
  k_rank_scatter<<<gs, 256, 0, s>>>(r.v0, r.v1, ctl, n, r.order, rank);
  k_zero_rounds<<<grid_stride_blocks(r.bptr_cap, r.num_sms), 256, 0, s>>>(r.bptr, r.bptr_cap,
                                                                            ctl);
  k_keys<<<gs, 256, 0, s>>>(r.a, rank, r.excl, ctl, n, r.key, rcnt);
  k_scan_excl<<<rtiles, kScanThreads, 0, s>>>(rcnt, r.rcur, 0, 1, r.status, ++(*r.epoch),
                                               &ctl->tile_ctr[1], nullptr, nullptr, 0, ctl,
                                               r.lookback_limit, r.stall_lookback);
  k_rscatter<<<(u32)min((long long)(n + 256 * kRChunk - 1) / (256 * kRChunk),
                        (long long)r.num_sms * 8),
               256, 0, s>>>(r.a, r.excl, ctl, n, r.rcur, r.v0, reinterpret_cast<u32*>(r.k0));
  return launches + 5;
}

int launch_exclusive_scan(u32* data, u32 len, u64* status, u32* epoch, u32* tile_ctr,
                          Control* ctl, u32 spin_limit, cudaStream_t s, u32* copy) {
  const u32 tiles = (len + kScanTile - 1) / kScanTile;
  if (tiles == 0) return 0;
  k_scan_excl<<<tiles, kScanThreads, 0, s>>>(data, copy, len, 0, status, ++(*epoch), tile_ctr,
                                             nullptr, nullptr, 0, ctl, spin_limit, 0);
  return 1;
}

int launch_ranked_and_buckets(const RankBufs& r, const int* levels, const int* perm,
                              cudaStream_t s) {
  const u32 n = r.n;
  Control* ctl = r.ctl;
  const u32 gs = grid_stride_blocks(n, r.num_sms);
  const u32 rtiles = (r.bptr_cap + kScanTile - 1) / kScanTile;
  u32* rcnt = reinterpret_cast<u32*>(r.bptr);
  const u32* rank = reinterpret_cast<const u32*>(perm);
  cudaMemsetAsync(r.order, 0xff, (size_t)n * 4, s);
  k_ranked_split<<<gs, 256, 0, s>>>(levels, perm, n, r.a, r.order, ctl);
  k_zero_rounds<<<grid_stride_blocks(r.bptr_cap, r.num_sms), 256, 0, s>>>(r.bptr, r.bptr_cap,
                                                                            ctl);
  k_keys<<<gs, 256, 0, s>>>(r.a, rank, r.excl, ctl, n, r.key, rcnt);
  k_scan_excl<<<rtiles, kScanThreads, 0, s>>>(rcnt, r.rcur, 0, 1, r.status, ++(*r.epoch),
                                               &ctl->tile_ctr[1], nullptr, nullptr, 0, ctl,
                                               r.lookback_limit, r.stall_lookback);
  k_rscatter<<<(u32)min((long long)(n + 256 * kRChunk - 1) / (256 * kRChunk),
                        (long long)r.num_sms * 8),
               256, 0, s>>>(r.a, r.excl, ctl, n, r.rcur, r.v0, reinterpret_cast<u32*>(r.k0));
  return 5;
}

}  // namespace ldd

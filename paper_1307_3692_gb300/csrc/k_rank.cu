// Start keys of the delayed-start BFS (Section 4 of Miller, Peng, Xu 2013).
//
//  1. split (Algorithm 1 step 2, Section 4): a_u = floor(delta_u),
//     f_u = delta_u - a_u (exact in FP64), A = max a_u = floor(delta_max).
//  2. fraction rank (Section 4: the fractional parts are tie-breakers within
//     an integer level and can be replaced by a permutation): the stable order
//     of (f_u descending, u ascending) gives order[rank] = u.
//  3. keys: key_u = ((A - a_u) << 32) | rank_u, i.e. u's own start label at
//     round R_u = A - a_u.
//  4. start buckets (Section 4: the super-source edge of length L is looked at
//     when the frontier reaches distance L): stable sort of the vertices by
//     R_u, and bptr[r] = first position with R >= r, for r = 0 .. A + 1.
//     Vertices the BFS does not handle (no arcs, or a component small enough
//     for the warp solver) sort with R = A + 1, after every real bucket.
//
// Fraction rank, fast path: c_u = floor(f_u * 2^32) is a 32-bit code that is
// monotone in f_u, so a stable LSD sort of ~c_u (4 passes of 8 bits) orders
// the vertices by f descending except inside runs of equal codes, where they
// are in id order.  A fix-up pass sorts every such run of at most 32 vertices
// by the exact (f descending, id ascending); a run longer than 32 whose
// fractions are not all equal (never seen with drawn shifts, possible with
// crafted ones) makes the host redo the rank with the exact 64-bit path:
// the order-preserving bits of f itself as the key, 8 passes.
//
// The radix sort is a single-pass-per-digit ("onesweep") LSD sort: one kernel
// per 8-bit digit; each 4096-key tile ranks its keys in shared memory with
// warp match, publishes its per-digit counts and finds its global offsets by
// decoupled look-back over the preceding tiles.  Digits that are the same
// for every key are skipped (their pass is a no-op).
#include "ldd_internal.cuh"

namespace ldd {

namespace {

constexpr u32 kFull = 0xffffffffu;
constexpr u32 kLookbackSpinLimit = 1u << 24;  // ~1 s of polling, then kErrTimeout
constexpr int kRunMax = 32;                   // longest run of equal codes sorted in place

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

// Exact fraction of a validated shift, with -0 folded into +0.
__device__ __forceinline__ double frac_of(double d) {
  const double f = d - floor(d);
  return f == 0.0 ? 0.0 : f;
}

// Split.  KeyT = u32: key = ~floor(f * 2^32); KeyT = u64: key = ~bits(f).
template <typename KeyT>
__global__ void __launch_bounds__(256) k_split(const double* __restrict__ delta, u32 n,
                                               int* __restrict__ a_out, KeyT* __restrict__ kout,
                                               u32* __restrict__ vout, Control* ctl) {
  constexpr int kDigits = (int)sizeof(KeyT);
  __shared__ u32 sh[kDigits][256];
  __shared__ int s_amax;
  __shared__ u32 s_err;
  const u32 tid = threadIdx.x, lane = tid & 31;
  for (u32 i = tid; i < kDigits * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
  if (tid == 0) {
    s_amax = 0;
    s_err = 0;
  }
  __syncthreads();
  int amax = 0;
  u32 err = 0;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 base = blockIdx.x * blockDim.x + (tid & ~31u); base < n; base += stride) {
    const u32 idx = base + lane;
    const bool valid = idx < n;
    KeyT key = 0;
    if (valid) {
      const double d = delta[idx];
      int a = 0;
      double f = 0.0;
      if (!(d >= 0.0)) {
        err |= kErrShiftArg;
      } else if (!(d < 2147483648.0)) {
        err |= kErrShiftRange;
      } else {
        const double fl = floor(d);
        a = (int)fl;
        f = d - fl;  // exact: fl <= d < 2 fl, or fl = 0
      }
      if (sizeof(KeyT) == 4) {
        key = (KeyT)~(u32)floor(f * 4294967296.0);  // f * 2^32 < 2^32, exact scaling
      } else {
        key = (KeyT)~(f == 0.0 ? 0ull : (u64)__double_as_longlong(f));
      }
      a_out[idx] = a;
      kout[idx] = key;
      vout[idx] = idx;
      amax = max(amax, a);
    }
#pragma unroll
    for (int dg = 0; dg < kDigits; ++dg)
      hist_add(sh[dg], (u32)(key >> (8 * dg)) & 255u, valid, lane);
  }
  if (err) atomicOr(&s_err, err);
  atomicMax(&s_amax, amax);
  __syncthreads();
  if (tid == 0) {
    if (s_err) atomicOr(&ctl->err, s_err);
    atomicMax(&ctl->A, s_amax);
  }
  for (u32 i = tid; i < kDigits * 256; i += blockDim.x) {
    const u32 c = (&sh[0][0])[i];
    if (c) atomicAdd(&(&ctl->hist_f[0][0])[i], c);
  }
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

template <typename KeyT>
struct SortSmem {
  KeyT keys[kSortTile];             // the tile, staged in sorted order for the write-out
  u32 vals[kSortTile];
  u32 whist[kSortWarps][256];       // per-warp digit counts, then per-warp offsets
  u32 tile_excl[256];               // start of each digit's run inside the tile
  u32 base[256];                    // global start of this tile's run of each digit
  u32 wsum[kSortWarps];
  u32 tile;
  u32 bad;
};

// One stable LSD pass on digit `pass` (bits shift..shift+7).  Buffers are a
// ping-pong pair; the input side is the parity of the passes run before.  The
// tile is reordered by digit in shared memory first, so that the write-out of
// each digit's run is contiguous and coalesced.
template <typename KeyT>
__global__ void __launch_bounds__(kSortThreads) k_onesweep(
    KeyT* __restrict__ k0, u32* __restrict__ v0, KeyT* __restrict__ k1, u32* __restrict__ v1,
    u32 n, int pass, int shift, const u32* __restrict__ mask_ptr,
    const u32* __restrict__ digit_off, u64* __restrict__ status, u32* __restrict__ tile_ctr,
    u32 epoch, u32* err) {
  const u32 mask = *mask_ptr;
  if (!((mask >> pass) & 1u) || *(volatile u32*)err != 0u) return;
  const int par = __popc(mask & ((1u << pass) - 1u)) & 1;
  const KeyT* kin = par ? k1 : k0;
  const u32* vin = par ? v1 : v0;
  KeyT* kout = par ? k0 : k1;
  u32* vout = par ? v0 : v1;

  extern __shared__ __align__(16) unsigned char sort_smem_raw[];
  SortSmem<KeyT>& sm = *reinterpret_cast<SortSmem<KeyT>*>(sort_smem_raw);
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

  KeyT key[kSortIpt];
  u32 val[kSortIpt];
  u32 rk[kSortIpt];
#pragma unroll
  for (int k = 0; k < kSortIpt; ++k) {
    const u32 idx = base + k * 32 + lane;
    if (idx < n) {
      key[k] = kin[idx];
      val[k] = vin[idx];
    } else {
      key[k] = 0;
      val[k] = 0;
    }
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
  // thread tid owns digit tid: per-warp offsets, tile total, and (below) the
  // tile-local start of each digit and the global start from the look-back
  const u32 dg = tid;
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
        if (++spins > kLookbackSpinLimit) {
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
  // stage the tile in digit order
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
  // write out: consecutive threads, consecutive positions of one digit's run
  const u32 tile_n = min((u32)kSortTile, n - tile0);
  for (u32 i = tid; i < tile_n; i += kSortThreads) {
    const KeyT kv = sm.keys[i];
    const u32 d = (u32)(kv >> shift) & 255u;
    const u32 pos = sm.base[d] + (i - sm.tile_excl[d]);
    if (pos < n) {
      kout[pos] = kv;
      vout[pos] = sm.vals[i];
    }
  }
}

// Exact order inside runs of equal 32-bit fraction codes (see the file comment).
__global__ void __launch_bounds__(256) k_fixup_runs(const u32* __restrict__ k0, u32* v0,
                                                    const u32* __restrict__ k1, u32* v1,
                                                    const double* __restrict__ delta, Control* ctl,
                                                    u32 n) {
  if (failed(ctl)) return;
  const u32 par = __popc(ctl->mask_f) & 1u;
  const u32* K = par ? k1 : k0;
  u32* U = par ? v1 : v0;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    const u32 kp = K[p];
    const bool cont = p > 0 && K[p - 1] == kp;  // p continues a run
    if (!cont && p + 1 < n && K[p + 1] == kp) {
      // p starts a run: measure it (up to kRunMax + 1) and sort it if short
      u32 len = 1;
      while (len <= (u32)kRunMax && p + len < n && K[p + len] == kp) ++len;
      if (len <= (u32)kRunMax) {
        double f[kRunMax];
        u32 u[kRunMax];
        for (u32 i = 0; i < len; ++i) {
          u[i] = U[p + i];
          f[i] = frac_of(delta[u[i]]);
        }
        for (u32 i = 1; i < len; ++i) {  // insertion sort: f descending, id ascending
          const double fi = f[i];
          const u32 ui = u[i];
          u32 j = i;
          while (j > 0 && (f[j - 1] < fi || (f[j - 1] == fi && u[j - 1] > ui))) {
            f[j] = f[j - 1];
            u[j] = u[j - 1];
            --j;
          }
          f[j] = fi;
          u[j] = ui;
        }
        for (u32 i = 0; i < len; ++i) U[p + i] = u[i];
      }
    } else if (cont) {
      // Inside a run.  Adjacent fractions that differ need sorting; if the run
      // is longer than kRunMax nobody sorts it here, so ask for the exact path.
      // (A short run may be being sorted concurrently; that only affects which
      // threads get here, never the length test.)
      if (frac_of(delta[U[p]]) != frac_of(delta[U[p - 1]])) {
        u32 lo = p, hi = p;
        while (hi - lo <= (u32)kRunMax && lo > 0 && K[lo - 1] == kp) --lo;
        while (hi - lo <= (u32)kRunMax && hi + 1 < n && K[hi + 1] == kp) ++hi;
        if (hi - lo + 1 > (u32)kRunMax) atomicOr(&ctl->err, kErrRankRetry);
      }
    }
  }
}

// rank -> key, and the start-round sort input (R_u, u) in rank order.
__global__ void __launch_bounds__(256) k_rank_keys(const u32* __restrict__ v0,
                                                   const u32* __restrict__ v1,
                                                   const int* __restrict__ a,
                                                   const u32* __restrict__ excl, Control* ctl,
                                                   u32 n, u32* __restrict__ order,
                                                   u64* __restrict__ key, u32* kR, u32* vR) {
  __shared__ u32 sh[kRoundDigits][256];
  const u32 tid = threadIdx.x, lane = tid & 31;
  for (u32 i = tid; i < kRoundDigits * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  if (failed(ctl)) return;
  const u32 par = __popc(ctl->mask_f) & 1u;
  const u32* vals = par ? v1 : v0;
  const int A = ctl->A;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 base = blockIdx.x * blockDim.x + (tid & ~31u); base < n; base += stride) {
    const u32 p = base + lane;
    const bool valid = p < n;
    u32 R = 0;
    if (valid) {
      u32 u = vals[p];
      if (u >= n) {  // cannot happen for a permutation; never index with it
        atomicOr(&ctl->err, kErrInternal);
        u = 0;
      }
      order[p] = u;
      R = (u32)(A - a[u]);
      key[u] = ((u64)R << 32) | p;
      if (excl[u >> 5] >> (u & 31) & 1u) R = (u32)A + 1u;
      kR[p] = R;
      vR[p] = u;
    }
#pragma unroll
    for (int dg = 0; dg < kRoundDigits; ++dg) hist_add(sh[dg], (R >> (8 * dg)) & 255u, valid, lane);
  }
  __syncthreads();
  for (u32 i = tid; i < kRoundDigits * 256; i += blockDim.x) {
    const u32 c = (&sh[0][0])[i];
    if (c) atomicAdd(&(&ctl->hist_r[0][0])[i], c);
  }
}

// bptr[r] = first position of the round-sorted list with R >= r, r = 0..A+1.
__global__ void __launch_bounds__(256) k_bucket_ptr(const u32* __restrict__ k0,
                                                    const u32* __restrict__ k1, Control* ctl, u32 n,
                                                    int* __restrict__ bptr, u32 cap) {
  if (failed(ctl)) return;
  const int A = ctl->A;
  if ((u64)A + 2 > cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->err, kErrBucketCap);
    return;
  }
  const u32* keys = (__popc(ctl->mask_r) & 1) ? k1 : k0;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int R = (int)keys[i];
    const int prev = (i == 0) ? -1 : (int)keys[i - 1];
    for (int r = prev + 1; r <= R; ++r) bptr[r] = (int)i;
    if (i == n - 1)
      for (int r = R + 1; r <= A + 1; ++r) bptr[r] = (int)n;
  }
}

u32 grid_stride_blocks(u32 n, int num_sms) {
  return (u32)max(1ll, min((long long)(n + 255) / 256, (long long)num_sms * 8));
}

// Shared memory of a onesweep pass beyond the default 48 KiB (64-bit keys):
// set once per device.
template <typename KeyT>
void allow_sort_smem() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  if (!done[dev]) {
    cudaFuncSetAttribute(k_onesweep<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(SortSmem<KeyT>));
    done[dev] = true;
  }
}

template <typename KeyT>
int launch_sort_passes(KeyT* k0, u32* v0, KeyT* k1, u32* v1, u32 n, int first_tile_ctr,
                       const u32* hist, u32* off, u32* mask, int ndig, u64* status, u32* epoch,
                       Control* ctl, cudaStream_t s) {
  allow_sort_smem<KeyT>();
  const u32 ntiles = (n + kSortTile - 1) / kSortTile;
  int launches = 0;
  k_scan_digits<<<1, 256, 0, s>>>(hist, off, mask, ndig, n);
  ++launches;
  for (int d = 0; d < ndig; ++d) {
    const u32 ep = ++(*epoch);
    k_onesweep<KeyT><<<ntiles, kSortThreads, sizeof(SortSmem<KeyT>), s>>>(k0, v0, k1, v1, n, d, 8 * d, mask,
                                                     off + 256 * d, status,
                                                     &ctl->tile_ctr[first_tile_ctr + d], ep,
                                                     &ctl->err);
    ++launches;
  }
  return launches;
}

}  // namespace

int launch_rank_and_buckets(const double* d_shift, u32 n, int* d_a, u64* k0, u32* v0, u64* k1,
                            u32* v1, u64* status, u32* epoch, u32* order, u64* key, int* bptr,
                            u32 bptr_cap, const u32* excl, bool exact64, Control* ctl,
                            int num_sms, cudaStream_t s) {
  const u32 gs = grid_stride_blocks(n, num_sms);
  int launches = 0;
  u32* k0w = reinterpret_cast<u32*>(k0);
  u32* k1w = reinterpret_cast<u32*>(k1);
  if (!exact64) {
    k_split<u32><<<gs, 256, 0, s>>>(d_shift, n, d_a, k0w, v0, ctl);
    ++launches;
    launches += launch_sort_passes<u32>(k0w, v0, k1w, v1, n, 0, &ctl->hist_f[0][0],
                                        &ctl->off_f[0][0], &ctl->mask_f, 4, status, epoch, ctl, s);
    k_fixup_runs<<<gs, 256, 0, s>>>(k0w, v0, k1w, v1, d_shift, ctl, n);
    ++launches;
  } else {
    k_split<u64><<<gs, 256, 0, s>>>(d_shift, n, d_a, k0, v0, ctl);
    ++launches;
    launches += launch_sort_passes<u64>(k0, v0, k1, v1, n, 0, &ctl->hist_f[0][0],
                                        &ctl->off_f[0][0], &ctl->mask_f, kFracDigits, status,
                                        epoch, ctl, s);
  }
  k_rank_keys<<<gs, 256, 0, s>>>(v0, v1, d_a, excl, ctl, n, order, key, k0w, v0);
  ++launches;
  launches += launch_sort_passes<u32>(k0w, v0, k1w, v1, n, kFracDigits, &ctl->hist_r[0][0],
                                      &ctl->off_r[0][0], &ctl->mask_r, kRoundDigits, status,
                                      epoch, ctl, s);
  launches += launch_bucket_ptr(k0, k1, ctl, n, bptr, bptr_cap, num_sms, s);
  return launches;
}

int launch_bucket_ptr(const u64* k0, const u64* k1, Control* ctl, u32 n, int* bptr, u32 cap,
                      int num_sms, cudaStream_t s) {
  k_bucket_ptr<<<grid_stride_blocks(n, num_sms), 256, 0, s>>>(
      reinterpret_cast<const u32*>(k0), reinterpret_cast<const u32*>(k1), ctl, n, bptr, cap);
  return 1;
}

}  // namespace ldd

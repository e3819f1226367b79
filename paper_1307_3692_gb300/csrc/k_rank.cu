// Start keys of the delayed-start BFS (Section 4 of Miller, Peng, Xu 2013).
//
//  1. split (Algorithm 1 step 2, Section 4): a_u = floor(delta_u),
//     f_u = delta_u - a_u (exact in FP64), A = max a_u = floor(delta_max).
//  2. fraction rank (Section 4: "these tie breakers can also be replaced by a
//     random permutation"): stable LSD radix sort of ~bits(f_u) (f descending,
//     u ascending on equal f) gives order[rank] = u.
//  3. keys: key_u = ((A - a_u) << 32) | rank_u, i.e. u's own start label at
//     round R_u = A - a_u.
//  4. start buckets (Section 4: the super-source edge of length L is looked at
//     when the frontier reaches distance L): stable sort of the vertices by
//     R_u, and bptr[r] = first position with R >= r, for r = 0 .. A + 1.
//     Vertices the BFS does not handle (no arcs, or a component small enough
//     for the warp solver) sort with R = A + 1, after every real bucket.
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

__device__ __forceinline__ void warp_hist_add(u32* sh, u32 digit, bool valid, u32 lane) {
  const u32 d = valid ? digit : 256u + lane;  // invalid lanes never match anyone
  const u32 peers = __match_any_sync(kFull, d);
  if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&sh[digit], (u32)__popc(peers));
}

__global__ void __launch_bounds__(256) k_split_hist(const double* __restrict__ delta, u32 n,
                                                    int* __restrict__ a_out,
                                                    u64* __restrict__ kout,
                                                    u32* __restrict__ vout, Control* ctl) {
  __shared__ u32 sh[kFracDigits][256];
  __shared__ int s_amax;
  __shared__ u32 s_err;
  const u32 tid = threadIdx.x, lane = tid & 31;
  for (u32 i = tid; i < kFracDigits * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
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
    u64 key = 0;
    if (valid) {
      const double d = delta[idx];
      int a = 0;
      u64 fb = 0;
      if (!(d >= 0.0)) {
        err |= kErrShiftArg;
      } else if (!(d < 2147483648.0)) {
        err |= kErrShiftRange;
      } else {
        const double fl = floor(d);
        a = (int)fl;
        const double f = d - fl;  // exact: fl <= d < 2 fl or fl = 0
        fb = (f == 0.0) ? 0ull : (u64)__double_as_longlong(f);
      }
      key = ~fb;  // ascending key <=> descending fraction
      a_out[idx] = a;
      kout[idx] = key;
      vout[idx] = idx;
      amax = max(amax, a);
    }
#pragma unroll
    for (int dg = 0; dg < kFracDigits; ++dg)
      warp_hist_add(sh[dg], (u32)(key >> (8 * dg)) & 255u, valid, lane);
  }
  if (err) atomicOr(&s_err, err);
  atomicMax(&s_amax, amax);
  __syncthreads();
  if (tid == 0) {
    if (s_err) atomicOr(&ctl->err, s_err);
    atomicMax(&ctl->A, s_amax);
  }
  for (u32 i = tid; i < kFracDigits * 256; i += blockDim.x) {
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

// One stable LSD pass on digit `pass` (bits shift..shift+7).  Buffers are a
// ping-pong pair; the input side is the parity of the passes run before.
__global__ void __launch_bounds__(kSortThreads) k_onesweep(
    u64* __restrict__ k0, u32* __restrict__ v0, u64* __restrict__ k1, u32* __restrict__ v1, u32 n,
    int pass, int shift, const u32* __restrict__ mask_ptr, const u32* __restrict__ digit_off,
    u64* __restrict__ status, u32* __restrict__ tile_ctr, u32 epoch, u32* err) {
  const u32 mask = *mask_ptr;
  if (!((mask >> pass) & 1u) || *(volatile u32*)err != 0u) return;
  const int par = __popc(mask & ((1u << pass) - 1u)) & 1;
  const u64* kin = par ? k1 : k0;
  const u32* vin = par ? v1 : v0;
  u64* kout = par ? k0 : k1;
  u32* vout = par ? v0 : v1;

  constexpr int kWarps = kSortThreads / 32;
  __shared__ u32 s_tile;
  __shared__ u32 s_bad;
  __shared__ u32 s_whist[kWarps][256];
  __shared__ u32 s_base[256];
  const u32 tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(tile_ctr, 1u);
    s_bad = 0;
  }
  for (u32 i = tid; i < kWarps * 256; i += kSortThreads) (&s_whist[0][0])[i] = 0;
  __syncthreads();
  const u32 tile = s_tile;
  const u32 base = tile * kSortTile + warp * (32 * kSortIpt);

  u64 key[kSortIpt];
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
    const u32 cnt = valid ? s_whist[warp][dg] : 0u;
    rk[k] = cnt + __popc(peers & lt);
    __syncwarp();
    if (valid && (peers & lt) == 0) s_whist[warp][dg] = cnt + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    // thread tid owns digit tid: offsets of each warp, tile total, look-back
    const u32 dg = tid;
    u32 run = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const u32 c = s_whist[w][dg];
      s_whist[w][dg] = run;
      run += c;
    }
    u64* mine = status + (u64)tile * 256 + dg;
    const u64 tag = (u64)epoch << 32;
    u32 excl = 0;
    if (tile == 0) {
      st_volatile_u64(mine, tag | (2ull << 30) | run);
    } else {
      st_volatile_u64(mine, tag | (1ull << 30) | run);
      int p = (int)tile - 1;
      u32 spins = 0;
      while (p >= 0) {
        const u64 s = ld_volatile_u64(status + (u64)p * 256 + dg);
        if ((u32)(s >> 32) != epoch) {
          if (++spins > kLookbackSpinLimit) {
            atomicOr(err, kErrTimeout);
            s_bad = 1;
            break;
          }
          if (spins > 16) __nanosleep(64);
          continue;
        }
        excl += (u32)s & 0x3fffffffu;
        if ((((u32)s) >> 30) == 2u) break;
        --p;
      }
      st_volatile_u64(mine, tag | (2ull << 30) | (excl + run));
    }
    s_base[dg] = digit_off[dg] + excl;
  }
  __syncthreads();
  if (s_bad) return;  // offsets unknown: write nothing
#pragma unroll
  for (int k = 0; k < kSortIpt; ++k) {
    const u32 idx = base + k * 32 + lane;
    if (idx < n) {
      const u32 dg = (u32)(key[k] >> shift) & 255u;
      const u32 pos = s_base[dg] + s_whist[warp][dg] + rk[k];
      if (pos < n) {
        kout[pos] = key[k];
        vout[pos] = val[k];
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
                                                   u64* __restrict__ key, u64* kR, u32* vR) {
  __shared__ u32 sh[kRoundDigits][256];
  const u32 tid = threadIdx.x, lane = tid & 31;
  for (u32 i = tid; i < kRoundDigits * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  if (*(volatile u32*)&ctl->err != 0u) return;
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
    for (int dg = 0; dg < kRoundDigits; ++dg) warp_hist_add(sh[dg], (R >> (8 * dg)) & 255u, valid, lane);
  }
  __syncthreads();
  for (u32 i = tid; i < kRoundDigits * 256; i += blockDim.x) {
    const u32 c = (&sh[0][0])[i];
    if (c) atomicAdd(&(&ctl->hist_r[0][0])[i], c);
  }
}

// bptr[r] = first position of the round-sorted list with R >= r, r = 0..A+1.
__global__ void __launch_bounds__(256) k_bucket_ptr(const u64* __restrict__ k0,
                                                    const u64* __restrict__ k1, Control* ctl, u32 n,
                                                    int* __restrict__ bptr, u32 cap) {
  if (*(volatile u32*)&ctl->err != 0u) return;
  const int A = ctl->A;
  if ((u64)A + 2 > cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ctl->err, kErrBucketCap);
    return;
  }
  const u64* keys = (__popc(ctl->mask_r) & 1) ? k1 : k0;
  const u32 stride = gridDim.x * blockDim.x;
  for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int R = (int)keys[i];
    const int prev = (i == 0) ? -1 : (int)keys[i - 1];
    for (int r = prev + 1; r <= R; ++r) bptr[r] = (int)i;
    if (i == n - 1)
      for (int r = R + 1; r <= A + 1; ++r) bptr[r] = (int)n;
  }
}

}  // namespace

int launch_rank_and_buckets(const double* d_shift, u32 n, int* d_a, u64* k0, u32* v0, u64* k1,
                            u32* v1, u64* status, u32* epoch, u32* order, u64* key, int* bptr,
                            u32 bptr_cap, const u32* excl, Control* ctl, int num_sms,
                            cudaStream_t s) {
  const u32 gs = (u32)min((long long)(n + 255) / 256, (long long)num_sms * 8);
  const u32 ntiles = (n + kSortTile - 1) / kSortTile;
  int launches = 0;
  k_split_hist<<<gs, 256, 0, s>>>(d_shift, n, d_a, k0, v0, ctl);
  ++launches;
  k_scan_digits<<<1, 256, 0, s>>>(&ctl->hist_f[0][0], &ctl->off_f[0][0], &ctl->mask_f,
                                  kFracDigits, n);
  ++launches;
  for (int d = 0; d < kFracDigits; ++d) {
    const u32 ep = ++(*epoch);
    k_onesweep<<<ntiles, kSortThreads, 0, s>>>(k0, v0, k1, v1, n, d, 8 * d, &ctl->mask_f,
                                               ctl->off_f[d], status, &ctl->tile_ctr[d], ep,
                                               &ctl->err);
    ++launches;
  }
  k_rank_keys<<<gs, 256, 0, s>>>(v0, v1, d_a, excl, ctl, n, order, key, k0, v0);
  ++launches;
  k_scan_digits<<<1, 256, 0, s>>>(&ctl->hist_r[0][0], &ctl->off_r[0][0], &ctl->mask_r,
                                  kRoundDigits, n);
  ++launches;
  for (int d = 0; d < kRoundDigits; ++d) {
    const u32 ep = ++(*epoch);
    k_onesweep<<<ntiles, kSortThreads, 0, s>>>(k0, v0, k1, v1, n, d, 8 * d, &ctl->mask_r,
                                               ctl->off_r[d], status,
                                               &ctl->tile_ctr[kFracDigits + d], ep, &ctl->err);
    ++launches;
  }
  launches += launch_bucket_ptr(k0, k1, ctl, n, bptr, bptr_cap, num_sms, s);
  return launches;
}

int launch_bucket_ptr(const u64* k0, const u64* k1, Control* ctl, u32 n, int* bptr, u32 cap,
                      int num_sms, cudaStream_t s) {
  const u32 gs = (u32)min((long long)(n + 255) / 256, (long long)num_sms * 8);
  k_bucket_ptr<<<gs, 256, 0, s>>>(k0, k1, ctl, n, bptr, cap);
  return 1;
}

}  // namespace ldd

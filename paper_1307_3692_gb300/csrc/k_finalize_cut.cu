// Assignment and verification kernels (Miller, Peng, Xu 2013).
//
// finalize (Algorithm 1 step 4, Algorithm 2 step 2): a settled key
// (level << 32) | rank names the center order[rank]; the hop distance is the
// key's level minus the center's own start level, which is the level of the
// center's key (a center is its own center, so its key is its start key).
//
// cut (Definition 1.1, second condition; Section 4 notes the check costs
// O(m) work): arcs (v, w) with v < w whose endpoints have different centers.
// Edge-balanced like the BFS: every CTA takes a fixed span of arcs; the rows
// that cover the span (a precomputed first-row table over the vertices with
// arcs) are located with a block max-scan in shared memory, so high-degree
// rows are split across CTAs and reads of col are coalesced.
#include "ldd_internal.cuh"

namespace ldd {

namespace {

constexpr u32 kFull = 0xffffffffu;

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

struct CutSmem {
  int owner[kCutSpan];
  u32 v[kCutSpan + 1];
  int cv[kCutSpan + 1];
  int wtot[kCutThreads / 32];
  unsigned long long wsum[kCutThreads / 32];
};

__global__ void __launch_bounds__(kCutThreads) k_cut(const int* __restrict__ row_ptr,
                                                     const int* __restrict__ col,
                                                     const u32* __restrict__ nzv,
                                                     const u32* __restrict__ first, u32 n_items,
                                                     u32 nnz, u32 n_vert,
                                                     const int* __restrict__ center, u64* out) {
  __shared__ CutSmem s;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const u32 nch = (nnz + kCutSpan - 1) / kCutSpan;
  const u32 c = blockIdx.x;
  const u32 e0 = c * kCutSpan, e1 = min(e0 + kCutSpan, nnz);
  const int len = (int)(e1 - e0);
  const u32 i0 = first[c];
  const u32 ilast = (c + 1 < nch) ? first[c + 1] : n_items - 1;
  const int nwin = (int)(ilast - i0) + 1;
  if (nwin < 1 || nwin > kCutSpan + 1 || ilast >= n_items) return;  // table inconsistent
  for (int j = t; j < len; j += kCutThreads) s.owner[j] = 0;
  __syncthreads();
  for (int j = t; j < nwin; j += kCutThreads) {
    const u32 v = nzv[i0 + j];
    const u32 off = (u32)row_ptr[v];
    if (off < e1) {
      s.v[j] = v;
      s.cv[j] = center[v];
      atomicMax(&s.owner[off > e0 ? off - e0 : 0u], j);
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
  unsigned long long cnt = 0;
  for (int kk = t; kk < len; kk += kCutThreads) {
    const int j = s.owner[kk];
    const u32 wv = (u32)col[e0 + kk];
    if (s.v[j] < wv && wv < n_vert && s.cv[j] != center[wv]) ++cnt;
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

}  // namespace

int launch_finalize(const u64* key, const u32* order, u32 n, int* center, int* dist,
                    const u32* err, int num_sms, cudaStream_t s) {
  const u32 g = (u32)min((long long)(n + 255) / 256, (long long)num_sms * 8);
  k_finalize<<<g, 256, 0, s>>>(key, order, n, center, dist, err);
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

}  // namespace ldd

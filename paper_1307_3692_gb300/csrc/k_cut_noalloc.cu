// ldd_cut_edges_noalloc: the cut-edge count without any device allocation.
//
// Who needs this: code that may not call cudaMalloc at the moment it wants
// the count.  Examples are a process whose framework allocator owns the whole
// device memory pool (a foreign cudaMalloc can fail, or break the pool's
// accounting), and a latency-critical loop where cudaMalloc/cudaFree would
// block on device-wide synchronisation.  Such callers hold the graph and the
// labels in device memory already; this entry point reads them in place.
//
// The scratch it needs -- a 64-bit accumulator and, for every 2048-arc span,
// the row that holds the span's first arc -- lives in the file-scope array
// g_cut_scratch below, sized for spans up to kMaxSpans (nnz <= 2^27 arcs).
// Every GPU that loads this library keeps that array (about 256 KiB) until
// the process exits.  The array's host-side name is only a stand-in, so the
// host fetches its device address with cudaGetSymbolAddress once per device
// and CUDA context (a cudaDeviceReset gives the device a new context, in
// which the array may sit elsewhere) and passes that pointer to the kernels.
//
// The paper has no counterpart to this entry point; it computes the same
// count as ldd_cut_edges (Definition 1.1, second condition).
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/ldd.h"
#include "ldd_internal.cuh"

namespace ldd {

void record_error(const char* msg);  // ldd_api.cu: text for ldd_last_error()

namespace {

constexpr u32 kSpan = 2048;                          // arcs per CTA
constexpr u32 kThreads = 256;
constexpr u32 kMaxSpans = 1u << 16;                  // first-row table entries
constexpr long long kMaxArcs = (long long)kMaxSpans * kSpan;  // 2^27
constexpr u32 kAccWords = 64;                        // accumulator + padding (256 B)
constexpr u32 kScratchWords = kAccWords + kMaxSpans;
constexpr int kMaxDevices = 64;

// Words [0, 2): the accumulator; words [64, 64 + kMaxSpans): first-row table.
static __device__ __align__(256) u32 g_cut_scratch[kScratchWords];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};  // the context each address was looked up in

__global__ void k_na_first_rows(const int* __restrict__ row_ptr, u32 n, u32 nspans,
                                u32* __restrict__ first) {
  const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nspans) return;
  const long long e = (long long)c * kSpan;
  u32 lo = 0, hi = n - 1;  // largest r with row_ptr[r] <= e
  while (lo < hi) {
    const u32 mid = lo + (hi - lo + 1) / 2;
    if ((long long)row_ptr[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  first[c] = lo;
}

__global__ void __launch_bounds__(kThreads) k_na_cut(const int* __restrict__ row_ptr,
                                                     const int* __restrict__ col,
                                                     const int* __restrict__ center, u32 n,
                                                     u32 nnz, u32 nspans,
                                                     const u32* __restrict__ first,
                                                     unsigned long long* acc) {
  __shared__ unsigned long long wsum[kThreads / 32];
  const u32 c = blockIdx.x;
  const u32 e0 = c * kSpan, e1 = min(e0 + kSpan, nnz);
  const u32 r0 = first[c];
  const u32 r1 = (c + 1 < nspans) ? first[c + 1] : n - 1;
  unsigned long long cnt = 0;
  for (u32 e = e0 + threadIdx.x; e < e1; e += kThreads) {
    u32 lo = r0, hi = r1;  // the row holding arc e
    while (lo < hi) {
      const u32 mid = lo + (hi - lo + 1) / 2;
      if ((u32)row_ptr[mid] <= e) lo = mid;
      else hi = mid - 1;
    }
    const u32 w = (u32)col[e];
    if (lo < w && w < n && center[lo] != center[w]) ++cnt;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0;
    for (u32 i = 0; i < kThreads / 32; ++i) tot += wsum[i];
    if (tot) atomicAdd(acc, tot);
  }
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// True for device memory of device `dev` (or managed memory, which every
// device can read).  Memory of another GPU is refused: reading it would be a
// fault without peer access and a slow cross-GPU read with it.
bool on_this_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// The driver's cuCtxGetCurrent, fetched through the runtime (the library does
// not link the driver API); null if unavailable.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<CtxGetCurrentFn>(f);
  }();
  return fn;
}

int fail(int status, const char* msg) {
  record_error(msg);
  return status;
}

// Device address of g_cut_scratch on the current device (dev), looked up on
// the first call in the device's current CUDA context.  Without the driver's
// context query the address is looked up on every call.
int scratch_address(int dev, u32** out) {
  CUcontext ctx = nullptr;
  const CtxGetCurrentFn get_ctx = ctx_get_current();
  const bool keyed = get_ctx && get_ctx(&ctx) == CUDA_SUCCESS && ctx != nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!keyed || !g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_cut_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      g_scratch_addr[dev] = nullptr;
      return fail(LDD_ERR_CUDA, "ldd_cut_edges_noalloc: cudaGetSymbolAddress of the scratch failed");
    }
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = keyed ? ctx : nullptr;
  }
  *out = static_cast<u32*>(g_scratch_addr[dev]);
  return LDD_OK;
}

}  // namespace
}  // namespace ldd

extern "C" int ldd_cut_edges_noalloc(int32_t n, int64_t nnz, const int32_t* row_ptr,
                                     const int32_t* col_idx, const int32_t* center,
                                     int64_t* out_cut, void* cuda_stream) {
  using namespace ldd;
  record_error("");
  if (!out_cut) return fail(LDD_ERR_ARG, "ldd_cut_edges_noalloc: out_cut is NULL");
  if (n < 0 || nnz < 0) return fail(LDD_ERR_ARG, "ldd_cut_edges_noalloc: negative size");
  if (nnz > kMaxArcs)
    return fail(LDD_ERR_RANGE, "ldd_cut_edges_noalloc: nnz exceeds its scratch limit of 2^27 arcs");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(LDD_ERR_CUDA, "ldd_cut_edges_noalloc: no usable current CUDA device");
  }
  const bool out_dev = on_device(out_cut);
  if (out_dev && !on_this_device(out_cut, dev))
    return fail(LDD_ERR_ARG, "ldd_cut_edges_noalloc: out_cut is memory of another device");
  if (n == 0 || nnz == 0) {
    if (!out_dev) {
      *out_cut = 0;
      return LDD_OK;
    }
    if (cudaMemsetAsync(out_cut, 0, sizeof(int64_t), s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      return fail(LDD_ERR_CUDA, "ldd_cut_edges_noalloc: clearing out_cut failed");
    }
    return LDD_OK;
  }
  if (!row_ptr || !col_idx || !center)
    return fail(LDD_ERR_ARG, "ldd_cut_edges_noalloc: NULL input");
  if (!on_this_device(row_ptr, dev) || !on_this_device(col_idx, dev) ||
      !on_this_device(center, dev))
    return fail(LDD_ERR_ARG,
                "ldd_cut_edges_noalloc: row_ptr, col_idx and center must be device memory of "
                "the current device");
  u32* scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc != LDD_OK) return rc;
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(scratch);
  u32* first = scratch + kAccWords;
  const u32 nspans = (u32)((nnz + kSpan - 1) / kSpan);
  if (cudaMemsetAsync(acc, 0, sizeof(*acc), s) != cudaSuccess) {
    cudaGetLastError();
    return fail(LDD_ERR_CUDA, "ldd_cut_edges_noalloc: clearing the accumulator failed");
  }
  k_na_first_rows<<<(nspans + kThreads - 1) / kThreads, kThreads, 0, s>>>(row_ptr, (u32)n, nspans,
                                                                           first);
  k_na_cut<<<nspans, kThreads, 0, s>>>(row_ptr, col_idx, center, (u32)n, (u32)nnz, nspans, first,
                                       acc);
  const cudaError_t e1 = cudaGetLastError();
  const cudaError_t e2 = cudaMemcpyAsync(out_cut, acc, sizeof(int64_t),
                                         out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                         s);
  const cudaError_t e3 = cudaStreamSynchronize(s);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    cudaGetLastError();
    return fail(LDD_ERR_CUDA, "ldd_cut_edges_noalloc: kernel launch or copy failed");
  }
  return LDD_OK;
}

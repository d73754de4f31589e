// compact_static.cu -- valid-row compaction whose scratch lives in static device memory,
// for callers that cannot allocate device memory; its scan also serves other
// flag compactions (compact_flags) with caller-provided scratch.
//
// Some callers cannot call cudaMalloc: code that runs while another framework owns the
// device memory pool (an embedding host that forbids foreign allocations), callers
// on a latency budget where an allocation may block on the driver, and code issued
// between other work that must not trigger an implicit device synchronisation.  For
// them this entry point takes the block sums of its scan from a file-scope static
// array instead of the context's plan, so it needs no context and allocates nothing.
// The array is sized for kStaticMaxRows flags; every GPU that loads the library holds
// it (16 KB) until the process exits.
#include <cuda.h>  // driver types only: the two driver calls are fetched through the runtime

#include <map>
#include <mutex>

#include "links_internal.cuh"

namespace links {
namespace {

constexpr int kBlockRows = 1024;
constexpr int kStaticBlocks = 4096;
constexpr int64_t kStaticMaxRows = (int64_t)kStaticBlocks * kBlockRows;  // 4,194,304 flags

// Block sums of the scan.  Host code must not pass this name to a kernel: it only
// stands for the symbol; the device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) int32_t g_block_sums[kStaticBlocks];

std::mutex g_mu;
// Device address of g_block_sums per CUDA context, keyed by the context's unique id (a
// device reset makes a new context with a new id, so its address is looked up again).
std::map<unsigned long long, int32_t*> g_sums_addr;

__device__ int static_block_scan(int v, int* total) {
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  int excl = x - v + (w ? ws[w - 1] : 0);
  if (total) *total = ws[31];
  __syncthreads();
  return excl;
}

// Entry b counts when valid[b] & mask is nonzero.
__global__ void __launch_bounds__(kBlockRows) static_scan_count(int64_t B, const uint8_t* valid, uint8_t mask,
                                                                int32_t* sums) {
  int64_t b = (int64_t)blockIdx.x * kBlockRows + threadIdx.x;
  int v = (b < B && (valid[b] & mask)) ? 1 : 0;
  int tot;
  static_block_scan(v, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Exclusive offsets of the nblk block sums (every entry read here was written by
// static_scan_count of the same call, so nothing needs clearing between calls).
__global__ void __launch_bounds__(kBlockRows) static_scan_top(int nblk, int32_t* sums, int32_t* n_out) {
  int carry = 0;
  for (int base = 0; base < nblk; base += kBlockRows) {
    int i = base + threadIdx.x;
    int v = i < nblk ? sums[i] : 0;
    int tot;
    int ex = static_block_scan(v, &tot);
    if (i < nblk) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && n_out) *n_out = carry;
}

__global__ void __launch_bounds__(kBlockRows) static_scan_write(int64_t B, const uint8_t* valid, uint8_t mask,
                                                                const int32_t* sums, int32_t* out_index, int64_t cap) {
  int64_t b = (int64_t)blockIdx.x * kBlockRows + threadIdx.x;
  int v = (b < B && (valid[b] & mask)) ? 1 : 0;
  int ex = static_block_scan(v, nullptr) + sums[blockIdx.x];
  if (v && ex < cap && out_index) out_index[ex] = (int32_t)b;
}

// Unique id of the calling thread's current CUDA context (cuCtxGetCurrent + cuCtxGetId,
// fetched through the runtime so the library needs no driver link); false if either
// call is unavailable or fails.
bool current_ctx_id(unsigned long long* id) {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  CUcontext c = nullptr;
  return get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, id) == CUDA_SUCCESS;
}

// Device address of g_block_sums in the current context: looked up once per context
// (cudaGetSymbolAddress with the device current), then cached.  Where the context id
// cannot be read (no context current yet on this thread, before the runtime's first
// call makes the primary context current), it is looked up on that call.
int static_sums(int32_t** out) {
  unsigned long long id = 0;
  const bool keyed = current_ctx_id(&id);
  std::lock_guard<std::mutex> lk(g_mu);
  if (keyed) {
    auto it = g_sums_addr.find(id);
    if (it != g_sums_addr.end()) {
      *out = it->second;
      return LINKS_OK;
    }
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_block_sums);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_block_sums)");
  if (keyed) g_sums_addr[id] = static_cast<int32_t*>(p);
  *out = static_cast<int32_t*>(p);
  return LINKS_OK;
}

}  // namespace

int64_t compact_sums_count(int64_t n) { return (n + kBlockRows - 1) / kBlockRows; }

int compact_flags(cudaStream_t s, const uint8_t* flags, uint8_t mask, int64_t n, int32_t* sums, int32_t* out_index,
                  int64_t cap, int32_t* n_out) {
  const int nblk = (int)compact_sums_count(n);
  if (nblk > 0) static_scan_count<<<nblk, kBlockRows, 0, s>>>(n, flags, mask, sums);
  LINKS_CUDA(cudaGetLastError());
  static_scan_top<<<1, kBlockRows, 0, s>>>(nblk, sums, n_out);
  LINKS_CUDA(cudaGetLastError());
  if (nblk > 0) static_scan_write<<<nblk, kBlockRows, 0, s>>>(n, flags, mask, sums, out_index, cap);
  LINKS_CUDA(cudaGetLastError());
  return LINKS_OK;
}

}  // namespace links

using namespace links;

extern "C" int links_compact_valid_static(const uint8_t* valid, int64_t B, int32_t* out_index,
                                          int64_t out_capacity, int32_t* n_out, void* cuda_stream) {
  if (B < 0 || out_capacity < 0) return set_error(LINKS_EINVAL, "links_compact_valid_static: negative size");
  if (B > kStaticMaxRows)
    return set_error(LINKS_EINVAL, "links_compact_valid_static: B exceeds the static maximum of 4194304 flags");
  if ((B > 0 && !valid) || !n_out || (out_capacity > 0 && !out_index))
    return set_error(LINKS_EINVAL, "links_compact_valid_static: NULL pointer");
  int32_t* sums = nullptr;
  int st = static_sums(&sums);
  if (st) return st;
  return compact_flags((cudaStream_t)cuda_stream, valid, 0xff, B, sums, out_index, out_capacity, n_out);
}

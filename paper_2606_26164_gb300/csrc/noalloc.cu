// chisao_dedup_noalloc: the L-infinity deduplication of Phase 3 for callers
// that cannot allocate device memory.
//
// The context-based path keeps the compacted list of stuck samples in memory
// that chisao_create carves out.  Some callers cannot create a context: hosts
// whose own memory pool has reserved the whole device and forbids side
// allocations, plug-ins that are handed only their input and output buffers,
// and latency-critical loops where a cudaMalloc/cudaFree pair would
// synchronize the device.  This entry point takes only caller buffers; its
// scratch (the stuck list and two counters) is a file-scope __device__ array
// that exists once per GPU for as long as the library stays loaded.  Its
// pairwise scan is O(S^2 d) in the stuck count S (the context path's spatial
// hash is near-linear), which the header states next to the size limit.
#include <mutex>

#include "../../include/chisao.h"
#include "dev_common.cuh"

namespace chisao {
namespace {

constexpr int NA_HEAD = 64;   // counters live in the first 64 ints (keeps the list 256-byte aligned)
constexpr int NA_NT = 1024;

// [0] stuck count, [1] removed count, [NA_HEAD ..] stuck sample indices
static __device__ __align__(256) int g_dedup_scratch[NA_HEAD + CHISAO_DEDUP_NOALLOC_MAX_N];

__global__ void k_na_clear(int* scratch, uint32_t* removed, int nwords) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) removed[w] = 0u;
  if (blockIdx.x == 0 && threadIdx.x < 2) scratch[threadIdx.x] = 0;
}

// Stuck samples in increasing index order (one block: per-thread runs of mask
// words, block scan of their counts, ordered writes).
__global__ void __launch_bounds__(NA_NT) k_na_compact(const uint32_t* __restrict__ stuck, int nwords, int n,
                                                      int* scratch) {
  __shared__ int scan[NA_NT];
  const int t = threadIdx.x;
  const int per = (nwords + NA_NT - 1) / NA_NT;
  const int w0 = min(nwords, t * per), w1 = min(nwords, w0 + per);
  auto word = [&](int w) {
    const int rem = n - w * 32;
    return stuck[w] & (rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u));
  };
  int c = 0;
  for (int w = w0; w < w1; ++w) c += __popc(word(w));
  scan[t] = c;
  __syncthreads();
  for (int off = 1; off < NA_NT; off <<= 1) {
    const int v = t >= off ? scan[t - off] : 0;
    __syncthreads();
    scan[t] += v;
    __syncthreads();
  }
  int base = scan[t] - c;
  int* list = scratch + NA_HEAD;
  for (int w = w0; w < w1; ++w) {
    unsigned m = word(w);
    while (m) {
      const int b = __ffs(m) - 1;
      list[base++] = w * 32 + b;
      m &= m - 1u;
    }
  }
  if (t == NA_NT - 1) scratch[0] = scan[NA_NT - 1];
}

// One warp per stuck x_j, lanes over coordinates (row stride d, caller layout):
// removed iff some other stuck x_i ranks above it (f desc, index asc) and
// max_k |x_ik - x_jk| < eps in binary32 -- the same decision as Phase 3.
__global__ void __launch_bounds__(256) k_na_dedup(const float* __restrict__ x, int d,
                                                  const float* __restrict__ f, float eps, int* scratch,
                                                  uint32_t* removed, int* k_lost_out) {
  const int lane = threadIdx.x & 31;
  const int jj = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int S = scratch[0];
  if (jj >= S) return;
  const int* list = scratch + NA_HEAD;
  const int j = list[jj];
  const float fj = f[j];
  const float xa = lane < d ? x[(size_t)j * d + lane] : 0.f;
  const float xb = lane + 32 < d ? x[(size_t)j * d + lane + 32] : 0.f;
  bool rem = false;
  for (int ii = 0; ii < S; ++ii) {
    const int i = list[ii];
    if (i == j) continue;
    const float fi = f[i];
    if (!(fi > fj || (fi == fj && i < j))) continue;
    const float ya = lane < d ? x[(size_t)i * d + lane] : 0.f;
    const float yb = lane + 32 < d ? x[(size_t)i * d + lane + 32] : 0.f;
    if (__all_sync(0xffffffffu, fabsf(ya - xa) < eps && fabsf(yb - xb) < eps)) {
      rem = true;
      break;
    }
  }
  if (rem && lane == 0) {
    atomicOr(&removed[j >> 5], 1u << (j & 31));
    atomicAdd(&scratch[1], 1);
    if (k_lost_out) atomicAdd(k_lost_out, 1);
  }
}

__global__ void k_na_zero(int* p) {
  if (threadIdx.x == 0) *p = 0;
}

// Device address of the scratch array, looked up once per device.
std::mutex g_mu;
void* g_addr[256] = {};

}  // namespace
}  // namespace chisao

using namespace chisao;

extern "C" chisao_status chisao_dedup_noalloc(const float* x_dev, int32_t d, int64_t n, const float* f_dev,
                                              const uint32_t* stuck_dev, double eps_dup, uint32_t* removed_dev,
                                              int32_t* k_lost_dev, void* cuda_stream) {
  if (d < 1 || d > CHISAO_MAX_DIM || n < 0 || !(eps_dup > 0)) return CHISAO_ERR_ARG;
  if (n > CHISAO_DEDUP_NOALLOC_MAX_N) return CHISAO_ERR_CAPACITY;
  if (n > 0 && (!x_dev || !f_dev || !stuck_dev || !removed_dev)) return CHISAO_ERR_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return CHISAO_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_dedup_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return CHISAO_ERR_CUDA;
      }
      g_addr[dev] = p;
    }
    scratch = g_addr[dev];
  }
  int* sc = static_cast<int*>(scratch);
  const int nwords = (int)((n + 31) / 32);
  k_na_clear<<<nwords > 0 ? (nwords + 255) / 256 : 1, 256, 0, st>>>(sc, removed_dev, nwords);
  if (k_lost_dev) k_na_zero<<<1, 32, 0, st>>>(k_lost_dev);
  if (n > 0) {
    k_na_compact<<<1, NA_NT, 0, st>>>(stuck_dev, nwords, (int)n, sc);
    const long long threads = 32ll * n;
    k_na_dedup<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(x_dev, d, f_dev, (float)eps_dup, sc,
                                                                  removed_dev, k_lost_dev);
  }
  return cudaGetLastError() == cudaSuccess ? CHISAO_OK : CHISAO_ERR_CUDA;
}

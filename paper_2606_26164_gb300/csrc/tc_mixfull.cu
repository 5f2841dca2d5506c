// Full-covariance Gaussian-mixture objective on the 5th-generation tensor cores
// (tcgen05, BF16 operands, FP32 accumulators in tensor memory).
//
// For a tile of 128 points x (one CTA, one point per TMEM lane / thread):
//   Z = X W^T, W = [L_1^-1; ...; L_K^-1] rounded to BF16, as an M=128 x N=256
//   GEMM per group of four components (N = 4 x 64), K = 128 with the input split
//   x = x_hi + x_lo into two BF16 terms (relative residual ~2^-17);
//   z_k = Z_k - b_k with b_k = W_k mu_k formed from the *rounded* W_k, so each
//   component's density peaks exactly at mu_k;
//   lc_k = c_k - |z_k|^2 / 2 with c_k = log w_k + log|det W_k| - (d/2) log 2 pi,
//   f = log sum_k exp(lc_k) as an online log-sum-exp in the epilogue.
// The result is exactly the log-density of the mixture whose precision factors
// are the BF16-rounded L_k^-1 (evaluated at the split input) up to FP32
// accumulation.  The gradient is grad f = -sum_k r_k W_k^T z_k, r = softmax(lc):
// a second pass recomputes Z, writes Y = r_k z_k (BF16) to shared memory and
// accumulates G = Y V on the tensor cores (V = the same rows of W, laid out with
// the output coordinate as the N dimension).
//
// Operand tiles are stored in global memory already in the canonical K-major,
// non-swizzled shared-memory layout (8 x 16-byte core matrices), so each one
// arrives with a single cp.async.bulk.  Every mbarrier wait is bounded by a
// clock budget; on timeout the kernel raises the device error flag, stops
// issuing work and still releases its tensor memory.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/chisao.h"
#include "host.h"
#include "dev_common.cuh"

namespace chisao {
namespace tc {

constexpr int TM = 128;                    // points per CTA (MMA M)
constexpr int TN = 256;                    // columns per component group (4 x 64)
constexpr int DK = 64;                     // padded dimension (MMA K per half of the split input)
constexpr int A_BYTES = TM * DK * 2;       // 16 KB per BF16 input half
constexpr int W_BYTES = TN * DK * 2;       // 32 KB
constexpr int BIAS_BYTES = 4 * DK * 4;     // 1 KB
constexpr int C_BYTES = 16;                // 4 floats
constexpr int WBLK_BYTES = W_BYTES + BIAS_BYTES + C_BYTES;   // one bulk copy per group
constexpr int VT_BYTES = DK * TN * 2;      // 32 KB
constexpr int Y_BYTES = TM * TN * 2;       // 64 KB
constexpr int SMEM_BYTES = 2 * A_BYTES + WBLK_BYTES + VT_BYTES + Y_BYTES + 64;
constexpr uint32_t TMEM_COLS = 512;
constexpr long long WAIT_CYCLES = 2000000000ll;   // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the error flag raised) when the budget runs out.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
  const long long t0 = clock64();
  while (!mbar_try(b, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(err, 2);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets of the 8-row core matrices, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// Byte offset of element (row, k) in a canonical K-major non-swizzled tile
// whose rows hold `kdim` elements: core matrix (row/8, k/8), 16 bytes per row.
__host__ __device__ constexpr uint32_t canon_off(uint32_t row, uint32_t k, uint32_t kdim) {
  return (row >> 3) * (kdim / 8) * 128u + (k >> 3) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

__device__ __forceinline__ uint16_t f2bf(float f) {  // round to nearest even
  const uint32_t u = __float_as_uint(f);
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

struct TcArgs {
  const float* x;         // [.][ldx] points (FP32, first d columns used)
  int ldx;
  int n;                  // rows when count is null
  const int* idx;         // optional row list: launch row i is x row idx[i] (outputs too)
  const int* count;       // optional device row count (overrides n; CTAs past it exit)
  int d;
  int ngroups;            // component groups of 4
  const uint8_t* wblk;    // [ngroups][WBLK_BYTES]  W tile (canonical), bias [4][64] f32, c [4] f32
  const uint8_t* vt;      // [ngroups][VT_BYTES]    V tile (canonical, N = 64 output coordinates)
  float* f;               // [n] or null
  float* g;               // [n][ldg] or null
  int ldg;
  int* err;               // device error flag
};

template <bool GRAD>
__global__ void __launch_bounds__(TM, 1) k_tc_mixfull(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sA = sm;                                   // x_hi, then x_lo
  uint8_t* sW = sm + 2 * A_BYTES;                     // W tile | bias | c
  uint8_t* sV = sW + WBLK_BYTES;                      // V tile
  uint8_t* sY = sV + VT_BYTES;                        // Y tile
  uint64_t* bars = reinterpret_cast<uint64_t*>(sY + Y_BYTES);   // [0] loads, [1] mma
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;
  const int t = threadIdx.x, warp = t >> 5;
  const int nrows = a.count ? *a.count : a.n;
  if ((int)blockIdx.x * TM >= nrows) return;          // whole CTA past the rows: nothing to do
  const int lrow = blockIdx.x * TM + t;
  const bool live = lrow < nrows;
  const int row = live ? (a.idx ? a.idx[lrow] : lrow) : 0;

  // ---- set-up: barriers, tensor memory, the split BF16 input tile
  if (t == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  {
    const float* xr = a.x + (size_t)row * a.ldx;
    for (int k8 = 0; k8 < DK / 8; ++k8) {
      uint16_t hi[8], lo[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int j = k8 * 8 + e;
        const float v = (live && j < a.d) ? xr[j] : 0.f;
        hi[e] = f2bf(v);
        lo[e] = f2bf(v - bf2f(hi[e]));
      }
      uint4 ph, pl;
      ph.x = hi[0] | ((uint32_t)hi[1] << 16); ph.y = hi[2] | ((uint32_t)hi[3] << 16);
      ph.z = hi[4] | ((uint32_t)hi[5] << 16); ph.w = hi[6] | ((uint32_t)hi[7] << 16);
      pl.x = lo[0] | ((uint32_t)lo[1] << 16); pl.y = lo[2] | ((uint32_t)lo[3] << 16);
      pl.z = lo[4] | ((uint32_t)lo[5] << 16); pl.w = lo[6] | ((uint32_t)lo[7] << 16);
      *reinterpret_cast<uint4*>(sA + canon_off(t, k8 * 8, DK)) = ph;
      *reinterpret_cast<uint4*>(sA + A_BYTES + canon_off(t, k8 * 8, DK)) = pl;
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t idF = idesc_bf16(TM, TN), idB = idesc_bf16(TM, DK);
  uint32_t ph_ld = 0, ph_mma = 0;

  // one component group: load its operands, Z = X W^T into TMEM columns [0, 256)
  auto forward = [&](int grp, bool with_v) -> bool {
    if (t == 0) {
      mbar_expect_tx(&bars[0], (uint32_t)(WBLK_BYTES + (with_v ? VT_BYTES : 0)));
      bulk_g2s(sW, a.wblk + (size_t)grp * WBLK_BYTES, WBLK_BYTES, &bars[0]);
      if (with_v) bulk_g2s(sV, a.vt + (size_t)grp * VT_BYTES, VT_BYTES, &bars[0]);
    }
    if (!mbar_wait(&bars[0], ph_ld, a.err)) s_fail = 1;
    ph_ld ^= 1u;
    __syncthreads();
    if (s_fail) return false;
    if (t == 0) {
      tc_fence_after();
      const uint32_t aH = smem_u32(sA), aL = aH + A_BYTES, bW = smem_u32(sW);
#pragma unroll
      for (int s = 0; s < DK / 16; ++s)
        mma_bf16(tmem, sdesc(aH + s * 256, 128, 1024), sdesc(bW + s * 256, 128, 1024), idF, s > 0);
#pragma unroll
      for (int s = 0; s < DK / 16; ++s)
        mma_bf16(tmem, sdesc(aL + s * 256, 128, 1024), sdesc(bW + s * 256, 128, 1024), idF, 1u);
      mma_commit(&bars[1]);
    }
    if (!mbar_wait(&bars[1], ph_mma, a.err)) s_fail = 1;
    ph_mma ^= 1u;
    __syncthreads();
    tc_fence_after();
    return !s_fail;
  };

  // q_k of component kl of the current group for this thread's point
  auto comp_q = [&](int kl, float (&z)[64]) -> float {
    const float* bias = reinterpret_cast<const float*>(sW + W_BYTES) + kl * DK;
    float v[32];
    float q = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      tmem_ld32(tlane + (uint32_t)(kl * DK + h * 32), v);
#pragma unroll
      for (int e = 0; e < 32; ++e) {
        z[h * 32 + e] = v[e] - bias[h * 32 + e];
        q = fmaf(z[h * 32 + e], z[h * 32 + e], q);
      }
    }
    return q;
  };

  // ---- pass 1: f = log sum_k exp(lc_k)
  float m = -CUDART_INF_F, s = 0.f;
  for (int grp = 0; grp < a.ngroups; ++grp) {
    if (!forward(grp, false)) break;
    const float* cst = reinterpret_cast<const float*>(sW + W_BYTES + BIAS_BYTES);
    for (int kl = 0; kl < 4; ++kl) {
      float z[64];
      const float lc = cst[kl] - 0.5f * comp_q(kl, z);
      if (lc > m) {
        s = s * expf(m - lc) + 1.f;
        m = lc;
      } else {
        s += expf(lc - m);
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  const float fval = m + logf(s);

  // ---- pass 2: G = sum_k (r_k z_k)^T W_k on the tensor cores (TMEM columns [256, 320))
  if (GRAD && !s_fail) {
    for (int grp = 0; grp < a.ngroups; ++grp) {
      if (!forward(grp, true)) break;
      const float* cst = reinterpret_cast<const float*>(sW + W_BYTES + BIAS_BYTES);
      for (int kl = 0; kl < 4; ++kl) {
        float z[64];
        const float lc = cst[kl] - 0.5f * comp_q(kl, z);
        const float r = expf(lc - fval);
#pragma unroll
        for (int k8 = 0; k8 < 8; ++k8) {
          uint4 p;
          p.x = f2bf(r * z[k8 * 8 + 0]) | ((uint32_t)f2bf(r * z[k8 * 8 + 1]) << 16);
          p.y = f2bf(r * z[k8 * 8 + 2]) | ((uint32_t)f2bf(r * z[k8 * 8 + 3]) << 16);
          p.z = f2bf(r * z[k8 * 8 + 4]) | ((uint32_t)f2bf(r * z[k8 * 8 + 5]) << 16);
          p.w = f2bf(r * z[k8 * 8 + 6]) | ((uint32_t)f2bf(r * z[k8 * 8 + 7]) << 16);
          *reinterpret_cast<uint4*>(sY + canon_off(t, kl * DK + k8 * 8, TN)) = p;
        }
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (t == 0) {
        tc_fence_after();
        const uint32_t aY = smem_u32(sY), bV = smem_u32(sV);
#pragma unroll
        for (int s2 = 0; s2 < TN / 16; ++s2)
          mma_bf16(tmem + TN, sdesc(aY + s2 * 256, 128, 4096), sdesc(bV + s2 * 256, 128, 4096), idB,
                   (grp > 0 || s2 > 0) ? 1u : 0u);
        mma_commit(&bars[1]);
      }
      if (!mbar_wait(&bars[1], ph_mma, a.err)) s_fail = 1;
      ph_mma ^= 1u;
      __syncthreads();
      tc_fence_after();
      if (s_fail) break;
    }
  }

  // ---- outputs
  if (live && !s_fail) {
    if (a.f) a.f[row] = fval;
  }
  if (GRAD && !s_fail) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[32];
      tmem_ld32(tlane + (uint32_t)(TN + h * 32), v);
      if (live)
        for (int e = 0; e < 32; ++e)
          if (h * 32 + e < a.d) a.g[(size_t)row * a.ldg + h * 32 + e] = -v[e];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

}  // namespace tc

// ------------------------------------------------------------------ host side
cudaError_t tc_prepare_attributes() {
  cudaError_t e = cudaFuncSetAttribute(tc::k_tc_mixfull<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       tc::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc::k_tc_mixfull<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
}

size_t tc_weight_bytes(int K) {
  const size_t ng = (size_t)(K + 3) / 4;
  return ng * (tc::WBLK_BYTES + tc::VT_BYTES);
}
size_t tc_vt_offset(int K) { return (size_t)((K + 3) / 4) * tc::WBLK_BYTES; }

static uint16_t host_f2bf(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
static double host_bf2d(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

// Operand tiles of the tensor-core objective from the FP64 inverse Cholesky
// factors linv[K][d][d] (lower-triangular), means mu[K][d] and log-weights.
void tc_build_weights(int K, int d, const double* linv, const double* mu, const double* logw,
                      std::vector<uint8_t>& out) {
  using namespace tc;
  const int ng = (K + 3) / 4;
  out.assign(tc_weight_bytes(K), 0);
  const double half_log2pi = 0.5 * std::log(2.0 * M_PI);
  for (int grp = 0; grp < ng; ++grp) {
    uint8_t* W = out.data() + (size_t)grp * WBLK_BYTES;
    float* bias = reinterpret_cast<float*>(W + W_BYTES);
    float* cst = reinterpret_cast<float*>(W + W_BYTES + BIAS_BYTES);
    uint8_t* Vt = out.data() + tc_vt_offset(K) + (size_t)grp * VT_BYTES;
    for (int kl = 0; kl < 4; ++kl) {
      const int k = grp * 4 + kl;
      if (k >= K) {
        cst[kl] = -INFINITY;
        continue;
      }
      const double* Li = linv + (size_t)k * d * d;
      double ldet = 0.0;
      for (int i = 0; i < d; ++i) {
        double b = 0.0;
        for (int j = 0; j < d; ++j) {
          const uint16_t h = host_f2bf((float)Li[(size_t)i * d + j]);
          const int n = kl * DK + i;
          *reinterpret_cast<uint16_t*>(W + canon_off(n, j, DK)) = h;
          *reinterpret_cast<uint16_t*>(Vt + canon_off(j, n, TN)) = h;
          b += host_bf2d(h) * mu[(size_t)k * d + j];
          if (i == j) ldet += std::log(host_bf2d(h));
        }
        bias[kl * DK + i] = (float)b;
      }
      cst[kl] = (float)(logw[k] + ldet - d * half_log2pi);
    }
  }
}

cudaError_t tc_launch_mixfull(const float* x, int ldx, int n, int d, int K, const uint8_t* weights, float* f,
                              float* g, int ldg, int* err, cudaStream_t st, const int* idx, const int* count) {
  if (n <= 0) return cudaSuccess;
  tc::TcArgs a{x, ldx, n, idx, count, d, (K + 3) / 4, weights, weights + tc_vt_offset(K), f, g, ldg, err};
  const unsigned grid = (unsigned)((n + tc::TM - 1) / tc::TM);
  if (g)
    tc::k_tc_mixfull<true><<<grid, tc::TM, tc::SMEM_BYTES, st>>>(a);
  else
    tc::k_tc_mixfull<false><<<grid, tc::TM, tc::SMEM_BYTES, st>>>(a);
  return cudaGetLastError();
}

}  // namespace chisao

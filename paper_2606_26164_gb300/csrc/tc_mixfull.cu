// Full-covariance Gaussian-mixture objective on the 5th-generation tensor cores
// (tcgen05, BF16 operands, FP32 accumulators in tensor memory).
//
// For a tile of 128 points (one CTA, one point per TMEM lane), per group of two
// components (MMA N = 2 x 64 = 128):
//   Z = [x_hi | x_lo | 1] [W | W | -b]^T, W = the two components' L_k^-1 rounded to
//   BF16, the input split into two BF16 terms x = x_hi + x_lo (relative residual
//   ~2^-17) and b_k = W_k mu_k formed from the *rounded* W_k and entered as three
//   BF16 terms against a K block of ones, so z_k = W_k (x - mu_k) leaves the tensor
//   cores centred and each component's density peaks exactly at mu_k;
//   lc_k = c_k - |z_k|^2 / 2 with c_k = log w_k + log|det W_k| - (d/2) log 2 pi,
//   f = log sum_k exp(lc_k).
// The result is exactly the log-density of the mixture whose precision factors
// are the BF16-rounded L_k^-1 (evaluated at the split input) up to FP32
// accumulation.  The gradient is grad f = -sum_k r_k W_k^T z_k, r = softmax(lc),
// formed in the same pass: the weights y = e^(lc_k - m_ref) z_k go to tensor memory
// as BF16 (Y, two buffers) and G += Y V accumulates on the tensor cores (V = the same
// rows of W with the output coordinate as the N dimension); G is rescaled when the
// reference m_ref rises, and normalised by the final sum.
//
// The factors are lower-triangular, so only the blocks on or below the diagonal
// are multiplied: the output rows of a group's factor tile are ordered by 16-row
// slab, the last slab first, so the input K-chunk c (coordinates 16c .. 16c+15)
// meets exactly the first (4 - c) x 32 rows (N = 128, 96, 64, 32), and in G += Y V
// the K-chunk c of y meets the first 16 (c + 1) output coordinates (N = 64, 48,
// 32, 16): 10 of the 16 16x16 blocks of each factor, in both contractions.
//
// Operand tiles are stored in global memory already in the canonical K-major,
// non-swizzled shared-memory layout (8 x 16-byte core matrices), so each one
// arrives with a single cp.async.bulk; each group's log-constants are read by the
// epilogue straight from global memory, one group ahead.  Every mbarrier wait is
// bounded by a clock budget; on timeout the kernel raises the device error flag,
// every role stops issuing work, waits for its copies and MMAs in flight, and the
// tensor memory is still released.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/chisao.h"
#include "host.h"
#include "dev_common.cuh"

namespace chisao {
namespace tc {

constexpr int TM = 128;                    // points per CTA (MMA M)
constexpr int CG = 2;                      // components per group
constexpr int TN = CG * 64;                // GEMM1 columns per group (MMA N)
constexpr int DK = 64;                     // padded dimension (MMA K per half of the split input)
constexpr int W_BYTES = TN * DK * 2;       // 16 KB factor tile of a group
constexpr int BT_BYTES = TN * 16 * 2;      // 4 KB bias tile: K block [-b_hi, -b_mid, -b_lo, 0 ...] per output row
constexpr int C_BYTES = 1024;              // c [CG] f32, zero padding
constexpr int WC_BYTES = W_BYTES + BT_BYTES + C_BYTES;     // one stage of the factor-tile ring
constexpr int VT_BYTES = DK * TN * 2;      // 16 KB V tile of a group
constexpr int GBLK_BYTES = WC_BYTES + VT_BYTES;            // one group in global memory
constexpr int NSLAB = DK / 16;              // 16-row slabs of a factor (and K-chunks of the input)
constexpr uint32_t TMEM_COLS = 512;
// Row of a group's factor tile (and Z column) holding output coordinate i of component kl:
// slab-major, the last slab first, the two components interleaved per slab.
__host__ __device__ constexpr int zrow(int kl, int i) { return (NSLAB - 1 - i / 16) * (16 * CG) + 16 * kl + (i % 16); }
// MMA N of the input K-chunk c in Z (the rows whose slab is >= c) and of the y K-chunk c
// in G (the output coordinates j <= 16 c + 15)
__host__ __device__ constexpr int zn_of_chunk(int c) { return (NSLAB - c) * 16 * CG; }
__host__ __device__ constexpr int gn_of_chunk(int c) { return 16 * (c + 1); }
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
// The same MMA with the A operand read from tensor memory (M rows = lanes, two BF16
// K-elements per 32-bit column, K ascending along the columns).
__device__ __forceinline__ void mma_bf16_ts(uint32_t dtmem, uint32_t atmem, uint64_t bd, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(dtmem),
      "r"(atmem), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// Byte offset of element (row, k) in a canonical K-major non-swizzled tile
// whose rows hold `kdim` elements: core matrix (row/8, k/8), 16 bytes per row.
__host__ __device__ constexpr uint32_t canon_off(uint32_t row, uint32_t k, uint32_t kdim) {
  return (row >> 3) * (kdim / 8) * 128u + (k >> 3) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

struct TcArgs {
  const float* x;         // [.][ldx] points (FP32, first d columns used)
  int ldx;
  int n;                  // rows when count is null
  const int* idx;         // optional row list: launch row i is x row idx[i] (outputs too)
  const int* count;       // optional device row count (overrides n; CTAs past it exit)
  int d;
  int ngroups;            // component groups of CG
  const uint8_t* gblk;    // [ngroups][GBLK_BYTES]: W tile | bias tile | c | V tile (canonical layouts)
  float* f;               // [n] or null
  float* g;               // [n][ldg] or null
  int ldg;
  int* err;               // device error flag
  float* part;            // [SPLIT_UNITS_MAX][PART_FIELDS][TM] partial results, or null (no split)
  int* ticket;            // [SPLIT_UNITS_MAX] arrivals per tile, zero between launches
  int nsm;                // multiprocessors of the device
};

// Component split: a launch of fewer tiles than half the multiprocessors (the later
// line-search rounds, small evaluations) would leave most of them idle for a whole tile's
// time, so the component groups of each tile are divided among nsplit CTAs, as many as
// still fit one wave.  Each writes its partial log-sum-exp (reference m, sum relative to m)
// and unnormalised gradient, and the last of a tile's CTAs to finish merges them.  Longer
// launches keep whole tiles: measured on 152 multiprocessors, splitting them into more
// waves cost more in per-CTA set-up and pipeline fill than it saved in the last wave.
constexpr int SPLIT_MAX = 16;
constexpr int SPLIT_UNITS_MAX = 256;       // CTAs of a split launch (one wave)
constexpr int PART_FIELDS = 2 + 64;        // m, sum, gradient coordinates
__host__ __device__ inline int split_of(int tiles, int ngroups, int grid, int nsm) {
  if (tiles <= 0 || nsm <= 0) return 1;
  int sp = nsm / tiles;
  if (grid / tiles < sp) sp = grid / tiles;
  if (SPLIT_UNITS_MAX / tiles < sp) sp = SPLIT_UNITS_MAX / tiles;
  if (ngroups < sp) sp = ngroups;
  if (SPLIT_MAX < sp) sp = SPLIT_MAX;
  return sp < 2 ? 1 : sp;
}

constexpr int NW = 4;                      // stages of the factor-tile ring (W, bias tile, constants)
constexpr int NV = 3;                      // stages of the V-tile ring
// Barriers in shared memory (index into the array after the tiles).
enum : int {
  B_WFULL = 0,                 // [NW] factor tile, bias tile and constants of a group landed
  B_WEMPTY = B_WFULL + NW,     // [NW] read by the Z MMAs
  B_VFULL = B_WEMPTY + NW,     // [NV] V tile of a group landed
  B_VEMPTY = B_VFULL + NV,     // [NV] read by the gradient MMAs of both components (two commits)
  B_ZFULL = B_VEMPTY + NV,     // [2] Z buffer b holds its group (groups of parity b)
  B_ZEMPTY = B_ZFULL + 2,      // [2] Z buffer b read into registers by all eight epilogue warps
  B_YFULL = B_ZEMPTY + 2,      // [2 h + b] component h's half of Y buffer b written (warpgroup h)
  B_GDONE = B_YFULL + 4,       // [2 h + b] gradient MMAs of component h for a group of parity b finished
  B_XREADY = B_GDONE + 4,      // split input tile written (eight warps)
  B_DRAIN = B_XREADY + 1,      // [4] every MMA of issuer i finished
  NBARS = B_DRAIN + 4
};
// warp 0 copies, warps 1-2 issue Z (groups of parity 0 / 1), warps 3 and 12 issue the
// gradient MMAs of component 0 / 1, warps 4-11 are the epilogue
constexpr int NTHREADS = 416;
constexpr int A_BYTES = TM * DK * 2;                      // 16 KB per BF16 input half
constexpr int ONES_BYTES = TM * 16 * 2;                   // 4 KB: the K block [1, 1, 1, 0 ...] of every point
constexpr int OFF_ONES = 2 * A_BYTES;
constexpr int OFF_W = OFF_ONES + ONES_BYTES;              // [NW] factor tile | bias tile | constants
constexpr int OFF_V = OFF_W + NW * WC_BYTES;              // [NV] V tiles
constexpr int OFF_XCH = OFF_V + NV * VT_BYTES;            // exchange of the two warpgroups at the end
constexpr int XCH_BYTES = TM * 64 * 4 + 8 * TM * 4;       // [64][TM] gradient half, [2][2][TM] max, [2][2][TM] sum
constexpr int OFF_BAR = OFF_XCH + XCH_BYTES;
constexpr int SMEM2_BYTES = OFF_BAR + NBARS * 8 + 16;     // + TMEM address, abort flag, merge flag
static_assert(WC_BYTES % 1024 == 0 && VT_BYTES % 1024 == 0 && OFF_W % 1024 == 0, "1024-byte aligned tiles");
static_assert(SMEM2_BYTES <= 232448, "shared memory per block");
// TMEM columns: Z buffer b at COL_Z + 128 b, the gradient accumulator of component h at
// COL_G + 64 h, and Y buffer b (BF16 weights, two K-elements per column) at COL_Y + 64 b,
// component h's half at + 32 h
constexpr uint32_t COL_Z = 0, COL_G = 2 * TN, COL_Y = 2 * TN + 128;
static_assert(COL_Y + 2 * 64 <= TMEM_COLS, "tensor memory columns");
// Z column of component h's slab s of z
__host__ __device__ constexpr uint32_t zcol(int h, int s) { return (uint32_t)zrow(h, 16 * s); }
constexpr float TAU = 16.f;                // lazy rescale: Y weights stay below e^TAU

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// Bounded wait that also gives up as soon as another role has aborted.
// A failed try sleeps NAP_NS before the next one: the single-thread roles (producer,
// MMA issuers) nap ROLE_NAP_NS and so leave their sub-partition's issue slots to the
// epilogue warps that share it (measured: 0.446 -> 0.418 ms per launch at N = 65536);
// the epilogue's own waits nap EPI_NAP_NS.
#ifndef CHISAO_TC_ROLE_NAP_NS
#define CHISAO_TC_ROLE_NAP_NS 64
#endif
#ifndef CHISAO_TC_EPI_NAP_NS
#define CHISAO_TC_EPI_NAP_NS 0
#endif
constexpr unsigned ROLE_NAP_NS = CHISAO_TC_ROLE_NAP_NS, EPI_NAP_NS = CHISAO_TC_EPI_NAP_NS;
template <unsigned NAP_NS = 0>
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* b, uint32_t parity, int* err, volatile int* abort_flag) {
  const long long t0 = clock64();
  while (!mbar_try(b, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(err, 2);
      *abort_flag = 1;
      return false;
    }
    if (NAP_NS) __nanosleep(NAP_NS);
  }
  return true;
}
// Every lane waits; the warp proceeds only if all of them saw the phase complete.
__device__ __forceinline__ bool warp_wait(uint64_t* b, uint32_t parity, int* err, volatile int* abort_flag) {
  const bool w = mbar_wait_ab<EPI_NAP_NS>(b, parity, err, abort_flag);
  return __all_sync(0xffffffffu, w);
}
// 32 consecutive FP32 columns of this thread's TMEM lane, without the completion wait.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// Makes the registers of an asynchronous TMEM load depend on the completion wait.
__device__ __forceinline__ void tmem_pin32(uint32_t (&r)[32]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 16 consecutive FP32 columns of this thread's TMEM lane, without the completion wait.
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_pin16(uint32_t (&r)[16]) {
  asm volatile(""
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]),
      "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]),
      "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // a in the low half
  return *reinterpret_cast<const uint32_t*>(&h);
}
// 64 accumulator columns of this thread's lane, multiplied in place by s.
__device__ __forceinline__ void tmem_scale64(uint32_t taddr, float s) {
#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    uint32_t r[32];
    tmem_ld32_async(taddr + 32u * half, r);
    tmem_wait_ld();
    tmem_pin32(r);
#pragma unroll
    for (int e = 0; e < 32; ++e) r[e] = __float_as_uint(__uint_as_float(r[e]) * s);
    tmem_st32(taddr + 32u * half, r);
  }
}

// One CTA = one tile of 128 points; the components go in groups of two (parity b = g & 1):
//   warp 0 (one thread) bulk-copies each group's factor tile, bias tile and constants
//   into a ring of NW stages and its V tile into a ring of NV stages;
//   warps 1 and 2 (one thread each, the groups of parity 0 and 1) issue
//   Z = [x_hi|x_lo|1] [W|W|-b]^T into Z buffer b, only the nonzero triangle of each
//   K-chunk (the bias enters the contraction through a K block of ones against the
//   exact three-term BF16 split of -b, so z leaves the tensor cores centred);
//   warps 3 and 12 (one thread each, components 0 and 1 of every group) issue
//   G_h += Y_h V_h, Y read from TMEM buffer b.
//   A thread's tcgen05.mma issues are serial: each takes about 117 clocks whatever N
//   (measured for N = 16 ... 128, A from shared or tensor memory), while MMAs issued by
//   different threads into different accumulators overlap.  The nine dependent MMAs of
//   a group's Z therefore run about 1050 clocks: two Z buffers with one issuer each let
//   the next group's Z run while the epilogue reads this one, and one gradient issuer per
//   component keeps each accumulator's MMAs in group order (deterministic sums);
//   warps 4-11 are two warpgroups, one per component of the group, each covering the
//   four TMEM lane quadrants (one point per thread): they read z, fold the component
//   into a log-sum-exp and write the gradient weights e^(lc - m_ref) z as BF16 into
//   TMEM.  Each warpgroup keeps one reference m_ref and sum per point: m_ref is raised
//   only when a component exceeds it by TAU, its accumulator's rows then being rescaled
//   in place once the gradient MMAs of the previous group have finished with it.  The
//   two partial results are combined at the end.
template <bool GRAD>
__global__ void __launch_bounds__(NTHREADS, 1) k_tc_mixfull(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
  uint32_t& s_tmem = *reinterpret_cast<uint32_t*>(sm + OFF_BAR + NBARS * 8);
  int& s_abort = *reinterpret_cast<int*>(sm + OFF_BAR + NBARS * 8 + 4);
  volatile int* abort_flag = &s_abort;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nrows = a.count ? *a.count : a.n;
  const int tiles = (nrows + TM - 1) / TM;
  const int nsplit = a.part ? split_of(tiles, a.ngroups, (int)gridDim.x, a.nsm) : 1;
  const int tile = (int)blockIdx.x / nsplit;
  if (tile >= tiles) return;                            // whole CTA past the rows: nothing to do
  // this CTA's component groups [g0, g0 + ng)
  const int sp = (int)blockIdx.x - tile * nsplit;
  const int g0 = (int)((long long)sp * a.ngroups / nsplit);
  const int ng = (int)((long long)(sp + 1) * a.ngroups / nsplit) - g0;
  const uint8_t* gblk = a.gblk + (size_t)g0 * GBLK_BYTES;

  if (t == 0) {
    for (int i = 0; i < NW; ++i) {
      mbar_init(&bars[B_WFULL + i], 1);
      mbar_init(&bars[B_WEMPTY + i], 1);
    }
    for (int i = 0; i < NV; ++i) {
      mbar_init(&bars[B_VFULL + i], 1);
      mbar_init(&bars[B_VEMPTY + i], 2);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars[B_ZFULL + b], 1);
      mbar_init(&bars[B_ZEMPTY + b], 8);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&bars[B_YFULL + i], 4);
      mbar_init(&bars[B_GDONE + i], 1);
      mbar_init(&bars[B_DRAIN + i], 1);
    }
    mbar_init(&bars[B_XREADY], 8);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int lastW[NW], lastV[NV];
      for (int s = 0; s < NW; ++s) lastW[s] = -1;
      for (int s = 0; s < NV; ++s) lastV[s] = -1;
      // the V tile of a group is needed one group after its factor tile: it trails by two
      for (int g = 0; g < ng + (GRAD ? 2 : 0); ++g) {
        if (g < ng) {
          const int s = g % NW, u = g / NW;
          if (u > 0 && !mbar_wait_ab<ROLE_NAP_NS>(&bars[B_WEMPTY + s], (u - 1) & 1, a.err, abort_flag)) break;
          mbar_expect_tx(&bars[B_WFULL + s], (uint32_t)WC_BYTES);
          bulk_g2s(sm + OFF_W + s * WC_BYTES, gblk + (size_t)g * GBLK_BYTES, WC_BYTES, &bars[B_WFULL + s]);
          lastW[s] = u;
        }
        const int gv = g - 2;
        if (GRAD && gv >= 0) {
          const int s = gv % NV, u = gv / NV;
          if (u > 0 && !mbar_wait_ab<ROLE_NAP_NS>(&bars[B_VEMPTY + s], (u - 1) & 1, a.err, abort_flag)) break;
          mbar_expect_tx(&bars[B_VFULL + s], (uint32_t)VT_BYTES);
          bulk_g2s(sm + OFF_V + s * VT_BYTES, gblk + (size_t)gv * GBLK_BYTES + WC_BYTES, VT_BYTES,
                   &bars[B_VFULL + s]);
          lastV[s] = u;
        }
      }
      // copies still in flight land before the CTA may exit (bounded)
      for (int s = 0; s < NW; ++s)
        if (lastW[s] >= 0) mbar_wait(&bars[B_WFULL + s], lastW[s] & 1, a.err);
      for (int s = 0; s < NV; ++s)
        if (lastV[s] >= 0) mbar_wait(&bars[B_VFULL + s], lastV[s] & 1, a.err);
    }
  } else if (warp == 1 || warp == 2) {
    // ------------------------------------------------------------ Z issuer of the groups of parity j
    if (lane == 0) {
      const int j = warp - 1;
      const uint32_t idF = idesc_bf16(TM, TN);
      const uint32_t aX = smem_u32(sm), aOnes = smem_u32(sm + OFF_ONES);
      const uint32_t dz = tmem + COL_Z + (uint32_t)(TN * j);
      bool issued = false;
      if (mbar_wait_ab<ROLE_NAP_NS>(&bars[B_XREADY], 0, a.err, abort_flag)) {
        for (int g = j; g < ng; g += 2) {
          const int s = g % NW;                        // NW is even: stage s always holds groups of parity j
          if (!mbar_wait_ab<ROLE_NAP_NS>(&bars[B_WFULL + s], (g / NW) & 1, a.err, abort_flag)) break;
          if (g >= 2 && !mbar_wait_ab<ROLE_NAP_NS>(&bars[B_ZEMPTY + j], ((g - 2) >> 1) & 1, a.err, abort_flag)) break;
          tc_fence_after();
          const uint32_t bW = smem_u32(sm + OFF_W + s * WC_BYTES);
#pragma unroll
          for (int hl = 0; hl < 2; ++hl)               // x_hi then x_lo against the same factor tile
#pragma unroll
            for (int c = 0; c < NSLAB; ++c)            // K-chunk c meets the rows of slabs >= c
              mma_bf16(dz, sdesc(aX + hl * A_BYTES + c * 256, 128, 1024), sdesc(bW + c * 256, 128, 1024),
                       idesc_bf16(TM, zn_of_chunk(c)), (hl | c) ? 1u : 0u);
          mma_bf16(dz, sdesc(aOnes, 128, 256), sdesc(bW + W_BYTES, 128, 256), idF, 1u);   // - b
          mma_commit(&bars[B_ZFULL + j]);
          mma_commit(&bars[B_WEMPTY + s]);
          issued = true;
        }
      }
      if (issued) {                                     // every issued MMA completes before exit
        mma_commit(&bars[B_DRAIN + j]);
        mbar_wait(&bars[B_DRAIN + j], 0, a.err);
      }
    }
  } else if (warp == 3 || warp == 12) {
    // ------------------------------------------------------------ gradient issuer of component h
    if (GRAD && lane == 0) {
      const int h = warp == 3 ? 0 : 1;
      const uint32_t dg = tmem + COL_G + 64u * (uint32_t)h;
      bool issued = false;
      for (int g = 0; g < ng; ++g) {
        const int b = g & 1, s = g % NV;
        if (!mbar_wait_ab<ROLE_NAP_NS>(&bars[B_YFULL + 2 * h + b], (g >> 1) & 1, a.err, abort_flag)) break;
        if (!mbar_wait_ab<ROLE_NAP_NS>(&bars[B_VFULL + s], (g / NV) & 1, a.err, abort_flag)) break;
        tc_fence_after();
        const uint32_t bV = smem_u32(sm + OFF_V + s * VT_BYTES);
        const uint32_t aY = tmem + COL_Y + 64u * (uint32_t)b + 32u * (uint32_t)h;
#pragma unroll
        for (int c = NSLAB - 1; c >= 0; --c)           // y K-chunk c meets outputs j <= 16 c + 15
          mma_bf16_ts(dg, aY + 8u * c, sdesc(bV + (h * NSLAB + c) * 256, 128, 2048), idesc_bf16(TM, gn_of_chunk(c)),
                      (g > 0 || c < NSLAB - 1) ? 1u : 0u);
        mma_commit(&bars[B_GDONE + 2 * h + b]);
        mma_commit(&bars[B_VEMPTY + s]);
        issued = true;
      }
      if (issued) {
        mma_commit(&bars[B_DRAIN + 2 + h]);
        mbar_wait(&bars[B_DRAIN + 2 + h], 0, a.err);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 4-11)
    const int h = (warp - 4) >> 2;                      // component of the group
    const int quad = warp & 3;                          // TMEM lane quadrant of this warp
    const int p = quad * 32 + lane;                     // point of the tile
    const int lrow = tile * TM + p;
    const bool live = lrow < nrows;
    const int row = live ? (a.idx ? a.idx[lrow] : lrow) : 0;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    const uint32_t gcol = tl + COL_G + 64u * (uint32_t)h;

    // split input: this thread converts columns [32h, 32h + 32) of its point; the first
    // warpgroup also writes the point's ones block
    {
      const float* xr = a.x + (size_t)row * a.ldx;
#pragma unroll
      for (int k8 = 0; k8 < 4; ++k8) {
        const int j0 = 32 * h + 8 * k8;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = j0 + 2 * e;
          const float v0 = (live && j < a.d) ? xr[j] : 0.f;
          const float v1 = (live && j + 1 < a.d) ? xr[j + 1] : 0.f;
          const __nv_bfloat162 hh = __floats2bfloat162_rn(v0, v1);
          const float2 hf = __bfloat1622float2(hh);
          hi[e] = *reinterpret_cast<const uint32_t*>(&hh);
          lo[e] = pack_bf16x2(v0 - hf.x, v1 - hf.y);
        }
        *reinterpret_cast<uint4*>(sm + canon_off(p, j0, DK)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(sm + A_BYTES + canon_off(p, j0, DK)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      if (h == 0) {
        const uint32_t one = 0x3F80u;                   // BF16 1.0
        *reinterpret_cast<uint4*>(sm + OFF_ONES + canon_off(p, 0, 16)) = make_uint4(one | (one << 16), one, 0u, 0u);
        *reinterpret_cast<uint4*>(sm + OFF_ONES + canon_off(p, 8, 16)) = make_uint4(0u, 0u, 0u, 0u);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[B_XREADY]);
    }

    const float* cst_ptr = reinterpret_cast<const float*>(gblk + W_BYTES + BT_BYTES) + h;
    float cst_next = __ldg(cst_ptr);
    float mref = -CUDART_INF_F, ssum = 0.f;
    bool ok = true;
    for (int g = 0; g < ng; ++g) {
      const int b = g & 1;
      if (!warp_wait(&bars[B_ZFULL + b], (g >> 1) & 1, a.err, abort_flag)) { ok = false; break; }
      tc_fence_after();
      float z[64];
      {
        uint32_t r[NSLAB][16];
#pragma unroll
        for (int c = 0; c < NSLAB; ++c) tmem_ld16_async(tl + COL_Z + (uint32_t)(TN * b) + zcol(h, c), r[c]);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < NSLAB; ++c) {
          tmem_pin16(r[c]);
#pragma unroll
          for (int e = 0; e < 16; ++e) z[16 * c + e] = __uint_as_float(r[c][e]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[B_ZEMPTY + b]);   // Z buffer b may take group g + 2

      // the log-constant of this group, read from global memory one group ahead (the factor
      // ring then depends on the Z MMAs alone)
      const float cst = cst_next;
      if (g + 1 < ng) cst_next = __ldg(cst_ptr + (size_t)(g + 1) * (GBLK_BYTES / 4));
      float2 qa = make_float2(0.f, 0.f), qb = qa, qc = qa, qd = qa;   // four packed chains
#pragma unroll
      for (int e = 0; e < 64; e += 8) {
        const float2 z0 = make_float2(z[e], z[e + 1]), z1 = make_float2(z[e + 2], z[e + 3]);
        const float2 z2 = make_float2(z[e + 4], z[e + 5]), z3 = make_float2(z[e + 6], z[e + 7]);
        qa = __ffma2_rn(z0, z0, qa);
        qb = __ffma2_rn(z1, z1, qb);
        qc = __ffma2_rn(z2, z2, qc);
        qd = __ffma2_rn(z3, z3, qd);
      }
      const float lc = cst - 0.5f * (((qa.x + qa.y) + (qb.x + qb.y)) + ((qc.x + qc.y) + (qd.x + qd.y)));

      if (!GRAD) {
        if (lc > mref) {
          ssum = ssum * expf(mref - lc) + 1.f;
          mref = lc;
        } else if (lc > -CUDART_INF_F) {
          ssum += expf(lc - mref);
        }
        continue;
      }
      float scale = 1.f;
      bool resc = false;
      if (lc > mref + TAU) {
        if (mref > -CUDART_INF_F) {
          scale = expf(mref - lc);
          resc = true;
          ssum *= scale;
        }
        mref = lc;
      }
      // this component's half of Y buffer b is free once its gradient MMAs of group g - 2
      // finished
      if (g >= 2 && !warp_wait(&bars[B_GDONE + 2 * h + b], ((g - 2) >> 1) & 1, a.err, abort_flag)) { ok = false; break; }
      tc_fence_after();
      const float r = lc > -CUDART_INF_F ? expf(lc - mref) : 0.f;
      ssum += r;
      {
        uint32_t y[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const float2 w = __fmul2_rn(make_float2(z[2 * e], z[2 * e + 1]), make_float2(r, r));
          y[e] = pack_bf16x2(w.x, w.y);
        }
        tmem_st32(tl + COL_Y + 64u * (uint32_t)b + 32u * h, y);
      }
      // a raised reference rescales the accumulator, once the gradient MMAs of group g - 1
      // have finished with it (waited for last: they ran while this group's weights were
      // formed); group g's MMAs are issued only after the arrival below
      if (__any_sync(0xffffffffu, resc)) {
        if (g >= 1 && !warp_wait(&bars[B_GDONE + 2 * h + (b ^ 1)], ((g - 1) >> 1) & 1, a.err, abort_flag)) {
          tmem_wait_st();
          ok = false;
          break;
        }
        tc_fence_after();
        tmem_scale64(gcol, scale);
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars[B_YFULL + 2 * h + b]);
    }

    // ---- combine the two warpgroups, write f and g
    float gacc[64];
    if (GRAD && ok) {
      // the gradient MMAs of the last group complete this component's accumulator (the
      // issuer's earlier MMAs were issued before them)
      ok = warp_wait(&bars[B_GDONE + 2 * h + ((ng - 1) & 1)], ((ng - 1) >> 1) & 1, a.err, abort_flag);
    }
    float* xch = reinterpret_cast<float*>(sm + OFF_XCH);            // [64][TM]
    float* s_m = xch + 64 * TM;                                     // [h][TM]
    float* s_s = s_m + 2 * TM;                                      // [h][TM]
    s_m[h * TM + p] = mref;
    s_s[h * TM + p] = ssum;
    epi_sync();
    const float m = fmaxf(s_m[p], s_m[TM + p]);
    float stot = 0.f, eb = 0.f;                         // eb: weight of this warpgroup's partial
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const float mi = s_m[i * TM + p];
      const float ei = mi > -CUDART_INF_F ? expf(mi - m) : 0.f;
      stot += s_s[i * TM + p] * ei;
      if (i == h) eb = ei;
    }
    const bool fine = ok && !*abort_flag;
    // a split CTA's partial, field-major: [0] m, [1] the sum relative to m, [2 + e] the
    // unnormalised gradient sum_h e^(m_h - m) G_h
    float* part = nsplit > 1 ? a.part + (size_t)blockIdx.x * PART_FIELDS * TM : nullptr;
    if (h == 0 && part) {
      part[p] = m;
      part[TM + p] = stot;
    }
    if (h == 0 && !part && live && fine && a.f) a.f[row] = m + logf(stot);
    if (GRAD) {
      if (fine) {
        tc_fence_after();
        const float sc = part ? eb : -eb / stot;
        uint32_t r0[32], r1[32];
        tmem_ld32_async(gcol, r0);
        tmem_ld32_async(gcol + 32, r1);
        tmem_wait_ld();
        tmem_pin32(r0);
        tmem_pin32(r1);
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          gacc[e] = __uint_as_float(r0[e]) * sc;
          gacc[32 + e] = __uint_as_float(r1[e]) * sc;
        }
        if (h == 1) {
#pragma unroll
          for (int e = 0; e < 64; ++e) xch[e * TM + p] = gacc[e];
        }
      }
      epi_sync();
      if (h == 0 && part && fine) {
#pragma unroll
        for (int e = 0; e < 64; ++e) part[(2 + e) * TM + p] = gacc[e] + xch[e * TM + p];
      } else if (h == 0 && live && fine) {
        float* gr = a.g + (size_t)row * a.ldg;
#pragma unroll
        for (int e = 0; e < 64; ++e)                    // the row's padding (d <= e < ldg) gets zeros
          if (e < a.ldg) gr[e] = e < a.d ? gacc[e] + xch[e * TM + p] : 0.f;
      }
    }
    if (part) {
      // the last of the tile's nsplit CTAs to arrive merges their partials (every CTA arrives,
      // also after an abort, so the tickets return to zero)
      int* s_last = reinterpret_cast<int*>(sm + OFF_BAR + NBARS * 8 + 8);
      __threadfence();
      epi_sync();
      if (t == 128) {
        const int prev = atomicAdd(&a.ticket[tile], 1);
        const int last = prev == nsplit - 1;
        if (last) a.ticket[tile] = 0;
        __threadfence();
        *s_last = last;
      }
      epi_sync();
      if (*s_last && live && fine) {
        const float* pt = a.part + (size_t)tile * nsplit * PART_FIELDS * TM + p;
        float mm = -CUDART_INF_F;
        for (int q = 0; q < nsplit; ++q) mm = fmaxf(mm, __ldcg(pt + (size_t)q * PART_FIELDS * TM));
        float st = 0.f;
        for (int q = 0; q < nsplit; ++q) {
          const float mq = __ldcg(pt + (size_t)q * PART_FIELDS * TM);
          if (mq > -CUDART_INF_F) st += __ldcg(pt + (size_t)q * PART_FIELDS * TM + TM) * expf(mq - mm);
        }
        if (h == 0 && a.f) a.f[row] = mm + logf(st);
        if (GRAD) {
          float acc[32];
#pragma unroll
          for (int e = 0; e < 32; ++e) acc[e] = 0.f;
          for (int q = 0; q < nsplit; ++q) {
            const float* pq = pt + (size_t)q * PART_FIELDS * TM;
            const float mq = __ldcg(pq);
            const float wq = mq > -CUDART_INF_F ? expf(mq - mm) : 0.f;
#pragma unroll
            for (int e = 0; e < 32; ++e) acc[e] = fmaf(__ldcg(pq + (size_t)(2 + 32 * h + e) * TM), wq, acc[e]);
          }
          float* gr = a.g + (size_t)row * a.ldg;
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const int j = 32 * h + e;
            if (j < a.ldg) gr[j] = j < a.d ? -acc[e] / st : 0.f;
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// The failure path of the bounded waits, on its own: thread 0 waits on a barrier that
// expects one arrival nobody makes, gives up after budget_ns of the global timer, raises
// the error flag and returns (no trap), as every barrier wait of k_tc_mixfull does.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__global__ void k_wait_selftest(long long budget_ns, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long t0 = global_ns();
    while (!mbar_try(&bar, 0)) {
      if ((long long)(global_ns() - t0) > budget_ns) {
        atomicExch(err, 2);
        break;
      }
    }
  }
  __syncthreads();
}

// Instruction rate of the tensor core for the MMA shape this kernel issues: lane 0 of
// warps 0 .. threads - 1 each issues `reps` MMAs (kind::f16, M = 128, K = 16, width n)
// into its own accumulator (columns 128 i for up to two issuers, 64 i for more; n fits
// that width), the last tmem_a of them with A read from tensor memory (columns 256 ..),
// the others from shared memory (zero operands: the rate, not the values, is measured).  clk[i] receives issuer i's clocks from its first issue until
// its MMAs completed (a bounded wait; *err = 2 when it runs out).
constexpr int RATE_SMEM = 65536 + 128;
__global__ void __launch_bounds__(128, 1) k_mma_rate(int n, int reps, int threads, int tmem_a, long long* clk,
                                                     int* err) {
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 65536);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + 65536 + 64);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int i = t; i < 65536 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(sm)[i] = 0u;
  if (t == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_async_smem();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  if (lane == 0 && warp < threads) {
    const uint32_t wide = threads <= 2 ? 2u : 1u;      // accumulator and B stride in units of 64 rows
    const uint32_t d = tmem + 64u * wide * (uint32_t)warp;
    const uint64_t ad = sdesc(smem_u32(sm), 128, 1024);
    const uint64_t bd = sdesc(smem_u32(sm + 16384 + (int)(8192u * wide) * warp), 128, 1024);
    const uint32_t aT = tmem + 256u + 32u * (uint32_t)(warp & 1);
    const uint32_t id = idesc_bf16(TM, n);
    const bool ts = warp >= threads - tmem_a;
    const long long t0 = clock64();
    for (int r = 0; r < reps; ++r) {
      if (ts)
        mma_bf16_ts(d, aT, bd, id, r > 0 ? 1u : 0u);
      else
        mma_bf16(d, ad, bd, id, r > 0 ? 1u : 0u);
    }
    mma_commit(&bars[warp]);
    mbar_wait(&bars[warp], 0, err);
    clk[warp] = clock64() - t0;
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
static int g_tc_nsm = 0;   // multiprocessors of the device, read once with the attributes
cudaError_t tc_prepare_attributes() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_tc_nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(tc::k_tc_mixfull<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       tc::SMEM2_BYTES);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(tc::k_tc_mixfull<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM2_BYTES);
}

size_t tc_weight_bytes(int K) { return (size_t)((K + tc::CG - 1) / tc::CG) * tc::GBLK_BYTES; }
size_t tc_split_floats() { return (size_t)tc::SPLIT_UNITS_MAX * tc::PART_FIELDS * tc::TM; }
size_t tc_split_tickets() { return (size_t)tc::SPLIT_UNITS_MAX; }

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

// Operand blocks of the tensor-core objective from the FP64 inverse Cholesky
// factors linv[K][d][d] (lower-triangular), means mu[K][d] and log-weights: per
// group of CG components the BF16 factor tile (rows = component-major output
// coordinates, K = input coordinate), the bias tile holding -W mu (from the rounded W,
// in binary32) as three BF16 terms whose sum is exact, the log-constants, and the V
// tile (rows = input coordinate, K = component-major output coordinate).
void tc_build_weights(int K, int d, const double* linv, const double* mu, const double* logw,
                      std::vector<uint8_t>& out) {
  using namespace tc;
  const int ng = (K + CG - 1) / CG;
  out.assign(tc_weight_bytes(K), 0);
  const double half_log2pi = 0.5 * std::log(2.0 * M_PI);
  for (int grp = 0; grp < ng; ++grp) {
    uint8_t* W = out.data() + (size_t)grp * GBLK_BYTES;
    uint8_t* Bt = W + W_BYTES;
    float* cst = reinterpret_cast<float*>(W + W_BYTES + BT_BYTES);
    uint8_t* Vt = W + WC_BYTES;
    for (int kl = 0; kl < CG; ++kl) {
      const int k = grp * CG + kl;
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
          *reinterpret_cast<uint16_t*>(W + canon_off(zrow(kl, i), j, DK)) = h;
          *reinterpret_cast<uint16_t*>(Vt + canon_off(j, kl * DK + i, TN)) = h;
          b += host_bf2d(h) * mu[(size_t)k * d + j];
          if (i == j) ldet += std::log(host_bf2d(h));
        }
        // -b in binary32 = t0 + t1 + t2 exactly, each term a BF16 value
        float r = (float)(-b);
        for (int e = 0; e < 3; ++e) {
          const uint16_t te = host_f2bf(r);
          *reinterpret_cast<uint16_t*>(Bt + canon_off(zrow(kl, i), e, 16)) = te;
          r -= (float)host_bf2d(te);
        }
      }
      cst[kl] = (float)(logw[k] + ldet - d * half_log2pi);
    }
  }
}

// Clocks per MMA of the tensor core, all issuers together (the slowest issuer's clocks
// over all MMAs), after one untimed run; synchronizes the stream.
cudaError_t tc_measure_mma_rate(int n, int threads, int tmem_a, double* clk_per_mma, cudaStream_t st) {
  constexpr int reps = 2048;
  long long* clk = nullptr;
  int* err = nullptr;
  cudaError_t e = cudaFuncSetAttribute(tc::k_mma_rate, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::RATE_SMEM);
  if (e == cudaSuccess) e = cudaMalloc(&clk, 4 * sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    tc::k_mma_rate<<<1, 128, tc::RATE_SMEM, st>>>(n, reps, threads, tmem_a, clk, err);
    e = cudaGetLastError();
  }
  long long h[4] = {0, 0, 0, 0};
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, clk, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(clk);
  cudaFree(err);
  if (e != cudaSuccess) return e;
  if (herr) return cudaErrorTimeout;
  long long mx = 0;
  for (int i = 0; i < threads; ++i) mx = h[i] > mx ? h[i] : mx;
  *clk_per_mma = (double)mx / ((double)reps * threads);
  return cudaSuccess;
}

cudaError_t tc_wait_selftest(long long budget_ns, int* err, cudaStream_t st) {
  tc::k_wait_selftest<<<1, 32, 0, st>>>(budget_ns, err);
  return cudaGetLastError();
}

cudaError_t tc_launch_mixfull(const float* x, int ldx, int n, int d, int K, const uint8_t* weights, float* f,
                              float* g, int ldg, int* err, cudaStream_t st, float* part, int* ticket,
                              const int* idx, const int* count) {
  if (n <= 0) return cudaSuccess;
  const bool split = part && ticket && g_tc_nsm > 0;
  tc::TcArgs a{x,    ldx, n,    idx, count, d, (K + tc::CG - 1) / tc::CG, weights, f, g, ldg, err,
               split ? part : nullptr, split ? ticket : nullptr, g_tc_nsm};
  // a row count known here gets exactly its CTAs; one known only on the device (count) gets
  // the tiles of the capacity, or the one wave a split of fewer tiles may fill
  const long long tiles = (n + tc::TM - 1) / tc::TM;
  const int ngroups = (K + tc::CG - 1) / tc::CG;
  long long grid = tiles;
  if (split && !count) grid = tiles * tc::split_of((int)std::min<long long>(tiles, 1 << 30), ngroups, 1 << 30, g_tc_nsm);
  else if (split) grid = std::max<long long>(tiles, std::min<long long>(tc::SPLIT_MAX * tiles, g_tc_nsm));
  if (g)
    tc::k_tc_mixfull<true><<<(unsigned)grid, tc::NTHREADS, tc::SMEM2_BYTES, st>>>(a);
  else
    tc::k_tc_mixfull<false><<<(unsigned)grid, tc::NTHREADS, tc::SMEM2_BYTES, st>>>(a);
  return cudaGetLastError();
}

}  // namespace chisao

// Device-side building blocks shared by every kernel of the ChiSao step.
//
// Layout (sample-major SoA, one problem):
//   x, g      float [n][dp]          dp = padded dimension (power of two >= 4)
//   f         float [n]
//   hs, hy    float [n][MMAX][dp]    L-BFGS pairs, slot 0 = newest
//   hrho      float [n][MMAX]        1 / s^T y (s^T y accumulated in double-single)
//   hlen      int [n]
//   stuck, removed   uint32 bit masks [ceil(n/32)]
// Padded coordinates are zero in x, g, the history and every objective
// parameter, so they never contribute to a dot product or a norm.
//
// A sample is processed by a "group" of LPS = dp/4 consecutive lanes of one
// warp; lane l of the group owns the four coordinates 4l .. 4l+3 (a float4),
// so a warp carries 32/LPS samples (two at d = 64, one per lane at d <= 4).
// Group reductions are xor-butterflies restricted to the group's lane mask, so
// every lane of the group ends with the bitwise-identical result and all
// control decisions stay group-uniform.
#pragma once
#include <cfloat>
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>
#include <math_constants.h>

namespace chisao {

constexpr int MMAX = 10;                 // register-resident L-BFGS memory
constexpr int GRAD_FD64 = 0, GRAD_FD32 = 1, GRAD_ADJOINT = 2;
constexpr int OBJ_MIXTURE_DIAG = 1, OBJ_MIXTURE_FULL = 2, OBJ_QUADRATIC = 3;
// the diagonal mixture evaluated with 2 or 8 components per step instead of 4 (grouped
// launches only: tile shapes the batched contexts' tuner can choose, same results)
constexpr int OBJ_MIXDIAG_C2 = 21, OBJ_MIXDIAG_C8 = 22;
// the Appendix D benchmark functions share one kind; ObjParams::fn selects the function
constexpr int OBJ_BENCH = 10;
constexpr int FN_RASTRIGIN = 0, FN_ACKLEY = 1, FN_SCHWEFEL = 2, FN_STYBLINSKI_TANG = 3, FN_MICHALEWICZ = 4,
              FN_TRID = 5, FN_BUKIN6 = 6;
constexpr int RESEED_NONE = 0, RESEED_RM = 1, RESEED_GR = 2, RESEED_UNIFORM = 3;
// Philox stream tags (same layout as the paper-side definition of the method's
// random draws; see the stream description in the library documentation).
constexpr unsigned TAG_RM = 1, TAG_RM_DIR = 2, TAG_GR_MAT = 3, TAG_GR_T = 4,
                   TAG_UNIFORM = 5, TAG_HLC = 6, TAG_NOISE = 7;

// Objective parameters in one precision.  Interpretation by kind:
//   MIXTURE_DIAG: p0 = mu [K][dp], p1 = 1/sigma^2 [K][dp], p2 = c [K]
//   MIXTURE_FULL: p0 = mu [K][dp], p1 = L^-1 [K][dp][dp] row-major,
//                 p3 = (L^-1)^T [K][dp][dp], p2 = c [K]
//   QUADRATIC:    p0 = center [dp], p1 = A = Q^T diag(lam) Q [dp][dp],
//                 p2 = A's blocks packed for the symmetric product [(dp/8 + 1) * 4 * dp]
// with c_k = log w_k - log|L_k| - (d/2) log(2 pi).
template <typename T>
struct ObjParams {
  int K, d, dp;
  int fn;                       // benchmark function (OBJ_BENCH)
  const T* p0;
  const T* p1;
  const T* p2;
  const T* p3;
};

struct ObjDev {
  int kind;
  int prob_index;
  float noise_sigma;            // additive evaluation noise (0: none)
  ObjParams<float> f32;
  ObjParams<double> f64;
};

// Device counters of one problem (one 256-byte block).
struct Counters {
  unsigned int fmax_key;        // order-preserving key of max f (0: no finite f)
  int n_stuck0;                 // stuck after Phase 2
  int n_removed;                // K_lost of the last Phase 3
  int n_stuck;                  // stuck after Phase 3
  int n_unfrozen;               // unfrozen when Phase 4 chose its strategy
  int n_surv;                   // survivors (stuck after Phase 3)
  int reseed_mode;
  int gr_enabled;
  int gr_noprog;
  int gr_prev_surv;
  int cycle;                    // completed cycles
  int n_free;                   // free slots (== n_removed)
  unsigned long long evals, grads, ls_trials, ls_fail;
  float fmax;
  float sigma;                  // scales of the last Phase 5 / 6 start
  float alpha_hlc;
  float alpha_anti;
  float sc_sigma;               // scales computed by the last finalize
  float sc_alpha;
  int sc_count;
  int err;                      // device-side error flag (0 ok)
};

struct ProbDev {
  int d, dp, n, nwords, prob_index, m;
  float* x;
  float* g;
  float* f;
  float* hs;
  float* hy;
  float* hrho;                  // 1 / s^T y per slot
  int* hlen;
  uint32_t* stuck;
  uint32_t* removed;
  int* l_stuck;                 // stuck samples, index order
  int* l_free;                  // removed samples (free slots), index order
  int* l_unf;                   // unfrozen samples, index order
  int* l_surv;                  // survivors, index order
  int* l_rank;                  // survivors ranked by (f desc, index asc)
  const float* lo;              // [dp] box, padded with 0
  const float* hi;
  Counters* cnt;
  float2* partials;             // [max_part_blocks][2 dp + 2] double-single sums
  int max_part_blocks;
  double* grq;                  // Golden Rooster Q [d][d], column-major
  // Phase 3 spatial hash: open addressing over 2^k >= 2 n slots, one list of stuck
  // samples per cell key (head per slot, next per stuck-list position)
  unsigned long long* hkey;
  unsigned long long* hbest;    // per slot: the cell's top-ranked member, (f bits << 32) | ~index
  int* hhead;
  int* hnext;
  int hmask;
  unsigned* hspread;            // [2][dp] ordered-key min and max of each coordinate over the stuck set
  int* haxes;                   // [4] the hashed coordinates (-1 unused) and their count
  ObjDev obj;
};

struct StepParams {
  int n_conv, n_anti, n_cloud, M, m, T_ls, grad_mode, rm_min, gr_patience, n_refine, hlc_value_only;
  float eps_grad, eps_dup, log_delta, mu, alpha_fixed, sigma_fixed, c_sigma, alpha_scale;
  double h, h_rel, c1, curv_eps;
  unsigned seed_lo, seed_hi;
};

// A grouped launch over several problems: block b belongs to problem q = blk_prob[b]
// and is block b - blk_first[q] of that problem (its blocks are consecutive).
struct GroupTab {
  const ProbDev* probs;
  const StepParams* sps;
  const int* blk_prob;
  const int* blk_first;
  const int* blk_count;         // blocks of problem q in this launch
};

// One launch over several problems for the objective-independent kernels: entry j of
// the launch's problem list (problem qidx[j], or j itself when qidx is null) owns blocks
// first[j] .. first[j + 1] - 1; each per-problem body gets its block index and block
// count within its problem, so it computes exactly what its own launch would.
struct AllTab {
  const ProbDev* probs;          // [problems]
  const StepParams* sps;         // [problems]
  const int* first;              // [n + 1] prefix sums of the entries' block counts
  const int* qidx;               // [n] or null
  int n;
};
struct BlkPos {
  int q;
  unsigned b, nb;
};
__device__ __forceinline__ BlkPos all_pos(const AllTab& T) {
  const int bx = (int)blockIdx.x;
  int lo = 0, hi = T.n - 1;                  // the last entry whose first block is <= bx
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (T.first[mid] <= bx) lo = mid;
    else hi = mid - 1;
  }
  return {T.qidx ? T.qidx[lo] : lo, (unsigned)(bx - T.first[lo]), (unsigned)(T.first[lo + 1] - T.first[lo])};
}

enum ObjKernelId { OKID_PHASE1 = 0, OKID_DIRECTION = 1, OKID_SCALES = 2, OKID_HLC = 3, OKID_ANTI = 4, OKID_EVAL = 5,
                   OKID_REFINE = 6 };

// Gradient mode of the scale pass when the gradient was computed by a batched
// evaluator and is already in g.
constexpr int GRAD_GIVEN = 9;

// Buffers of the batched-evaluator (tensor-core) path.
// Trial steps evaluated per sample in each line-search round after the first (the
// batched-evaluator Phase 1): round r >= 1 evaluates alpha0 2^-t for the next LS_BATCH
// values of t at once, and the first passing one wins.
constexpr int LS_BATCH = 4;
__host__ __device__ constexpr int ls_rounds(int T_ls) { return 1 + (T_ls - 1 + LS_BATCH - 1) / LS_BATCH; }

struct ExtBuf {
  float* p;        // [n][dp] search directions
  float* xt;       // [n][dp] first trial points (round 0)
  float* ft;       // [n] their values
  float* gt;       // [n][dp] their gradients
  float* a0;       // [n] initial steps
  int* list0;      // samples pending in round 0
  int* mlist[2];   // samples pending in a later round (double-buffered by round parity)
  int* cnt;        // [ls_rounds + 1] pending samples of each round, then [ls_rounds + 1] trial rows
  int* iota;       // [2 LS_BATCH n] 0, 1, 2, ...: the row list of a later round's trial points
  float* fm;       // [2 LS_BATCH n] values of the later rounds' trial points
  float* xp;       // [max(M, 2 LS_BATCH) n][dp] HLC perturbed points; the later line-search
                   //   rounds' trial points (buffer b at rows b LS_BATCH n, LS_BATCH rows per sample)
  float* gp;       // the same shape: their gradients
  float* vel;      // [n][dp] anti-convergence velocity
  int* head;       // [n] physical slot of the newest history pair during Phase 1 (the pairs form
                   //   a ring of m slots: logical slot k at (head + k) mod m); 0 between phases,
                   //   where slot 0 is the newest as everywhere else
};
enum ExtKernelId { EXT_DIR = 0, EXT_ACCEPT = 1, EXT_HLC_POINTS = 2, EXT_HLC_STEP = 3, EXT_ANTI_STEP = 4,
                   EXT_SCALES = 5, EXT_ACCEPT_MULTI = 6, EXT_IOTA = 7, EXT_HIST_ROTATE = 8 };

// Caller points for plain objective evaluation.
struct EvalArgs {
  const float* x;   // [n][d] device
  int n;
  float* f;         // [n] device or null
  float* g;         // [n][d] device or null
};

// ------------------------------------------------------------------ double-single sums
// s^T y of the L-BFGS update is accumulated beyond binary32: every product
// s_j y_j is split exactly into hi + lo with one FMA, and the terms are summed
// with Knuth's TwoSum, so the result carries ~48 significant bits (as accurate
// as an FP64 accumulation of the same binary32 products) while running on the
// FP32 pipe -- GB300's FP64 rate is a small fraction of its FP32 rate.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  float s, t;
  two_sum(h, bh, s, t);
  t += l + bl;
  h = s + t;
  l = t - (h - s);
}
// exact s0*y0 + s1*y1 as a double-single pair
__device__ __forceinline__ void ff_dot2(float s0, float y0, float s1, float y1, float& h, float& l) {
  const float p0 = s0 * y0, e0 = fmaf(s0, y0, -p0);
  const float p1 = s1 * y1, e1 = fmaf(s1, y1, -p1);
  h = p0;
  l = e0;
  ff_add(h, l, p1, e1);
}

// ------------------------------------------------------------------ groups
template <int LPS>
struct Grp {
  unsigned mask;
  int l;
  __device__ __forceinline__ Grp() {
    const int lane = threadIdx.x & 31;
    l = lane & (LPS - 1);
    mask = (LPS == 32) ? 0xffffffffu : (((1u << LPS) - 1u) << (lane & ~(LPS - 1)));
  }
  template <typename T>
  __device__ __forceinline__ T sum(T v) const {
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, LPS);
    return v;
  }
  __device__ __forceinline__ float maxf(float v) const {
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, o, LPS));
    return v;
  }
  template <typename T>
  __device__ __forceinline__ T bcast(T v, int src) const {
    return __shfl_sync(mask, v, src, LPS);
  }
  // the value held by the previous / next lane of the group (the first / last lane gets its own)
  template <typename T>
  __device__ __forceinline__ T from_prev(T v) const {
    return __shfl_up_sync(mask, v, 1, LPS);
  }
  template <typename T>
  __device__ __forceinline__ T from_next(T v) const {
    return __shfl_down_sync(mask, v, 1, LPS);
  }
  __device__ __forceinline__ bool all(bool p) const { return __all_sync(mask, p); }
  __device__ __forceinline__ unsigned xor_all(unsigned v) const {
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) v ^= __shfl_xor_sync(mask, v, o, LPS);
    return v;
  }
  // double-single sum over the group (bitwise identical in every lane: TwoSum
  // is exact, so swapping the operands of each butterfly step changes nothing)
  __device__ __forceinline__ void ff_sum(float& h, float& l) const {
#pragma unroll
    for (int o = LPS / 2; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(mask, h, o, LPS), ol = __shfl_xor_sync(mask, l, o, LPS);
      ff_add(h, l, oh, ol);
    }
  }
};

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

template <typename T>
__device__ __forceinline__ typename Vec2<T>::type ldg2(const T* p) {
  return __ldg(reinterpret_cast<const typename Vec2<T>::type*>(p));
}

// V consecutive values (V = 1, 2 or 4) through the read-only path / plain loads / stores.
template <typename T, int V>
__device__ __forceinline__ void ldg_vec(const T* p, T (&a)[V]) {
  if constexpr (V == 1) {
    a[0] = __ldg(p);
  } else if constexpr (V == 2) {
    const auto t = ldg2(p);
    a[0] = t.x; a[1] = t.y;
  } else if constexpr (std::is_same<T, float>::value) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
  } else {
    const auto t0 = ldg2(p), t1 = ldg2(p + 2);
    a[0] = t0.x; a[1] = t0.y; a[2] = t1.x; a[3] = t1.y;
  }
}

template <int V>
__device__ __forceinline__ void ld_vec(const float* p, float (&a)[V]) {
  if constexpr (V == 1) {
    a[0] = *p;
  } else if constexpr (V == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    a[0] = t.x; a[1] = t.y;
  } else {
    const float4 t = *reinterpret_cast<const float4*>(p);
    a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
  }
}

template <int V>
__device__ __forceinline__ void st_vec(float* p, const float (&a)[V]) {
  if constexpr (V == 1) {
    *p = a[0];
  } else if constexpr (V == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(a[0], a[1]);
  } else {
    *reinterpret_cast<float4*>(p) = make_float4(a[0], a[1], a[2], a[3]);
  }
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of the two multiply-hi/lo
// S-boxes with the Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 rng_words(const StepParams& S, unsigned c0, unsigned c1, unsigned tag,
                                           unsigned cycle, unsigned step, unsigned prob, unsigned k) {
  const uint4 c = make_uint4(c0, c1, (tag << 24) | ((cycle & 0xffffu) << 8) | (step & 0xffu),
                             ((prob & 0xffffu) << 16) | (k & 0xffffu));
  return philox4x32_10(c, make_uint2(S.seed_lo, S.seed_hi));
}

// u = (2 (w >> 9) + 1) 2^-24: exact in binary32, strictly inside (0, 1).
__device__ __forceinline__ float u01f(unsigned w) {
  return (float)(2u * (w >> 9) + 1u) * 5.9604644775390625e-8f;
}

// Box-Muller pairs (w0, w1) and (w2, w3) -> four standard normals.
__device__ __forceinline__ float4 normals4f(uint4 w) {
  float s0, c0, s1, c1;
  const float r0 = sqrtf(-2.0f * logf(u01f(w.x)));
  const float r1 = sqrtf(-2.0f * logf(u01f(w.z)));
  sincospif(2.0f * u01f(w.y), &s0, &c0);
  sincospif(2.0f * u01f(w.w), &s1, &c1);
  return make_float4(r0 * c0, r0 * s0, r1 * c1, r1 * s1);
}

__device__ __forceinline__ void normals4d(uint4 w, double out[4]) {
  double s0, c0, s1, c1;
  const double r0 = sqrt(-2.0 * log((double)u01f(w.x)));
  const double r1 = sqrt(-2.0 * log((double)u01f(w.z)));
  sincospi(2.0 * (double)u01f(w.y), &s0, &c0);
  sincospi(2.0 * (double)u01f(w.w), &s1, &c1);
  out[0] = r0 * c0;
  out[1] = r0 * s0;
  out[2] = r1 * c1;
  out[3] = r1 * s1;
}

// The normals of the lane's coordinates V l .. V l + V - 1 (coordinate j is
// normal j mod 4 of stream block j / 4): with V = 4 a lane's block is exactly
// Philox block l; with V = 2 it is half of block l / 2 (one Box-Muller pair).
template <int V>
__device__ __forceinline__ void normals_lane(const StepParams& S, unsigned row, int l, unsigned tag,
                                             unsigned cycle, unsigned step, unsigned prob, unsigned k,
                                             float (&z)[V]) {
  static_assert(V == 2 || V == 4, "lanes hold 2 or 4 coordinates");
  if constexpr (V == 4) {
    const float4 t = normals4f(rng_words(S, row, (unsigned)l, tag, cycle, step, prob, k));
    z[0] = t.x; z[1] = t.y; z[2] = t.z; z[3] = t.w;
  } else {
    const uint4 w = rng_words(S, row, (unsigned)(l >> 1), tag, cycle, step, prob, k);
    const unsigned wa = (l & 1) ? w.z : w.x, wb = (l & 1) ? w.w : w.y;
    float sn, cs;
    const float r = sqrtf(-2.0f * logf(u01f(wa)));
    sincospif(2.0f * u01f(wb), &sn, &cs);
    z[0] = r * cs;
    z[1] = r * sn;
  }
}

// ------------------------------------------------------------------ misc
// order-preserving map float -> uint32 (for atomicMax over floats)
__device__ __forceinline__ unsigned fkey(float v) {
  const unsigned b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__device__ __forceinline__ bool bit_of(const uint32_t* bits, int i) {
  return (bits[i >> 5] >> (i & 31)) & 1u;
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// Block-wide sum of 64-bit counters into device memory: one atomic per block.
template <int NT>
__device__ __forceinline__ void block_add_u64(unsigned long long v, unsigned long long* dst) {
  __shared__ unsigned long long red[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    if (t) atomicAdd(dst, t);
  }
  __syncthreads();
}

template <int NT>
__device__ __forceinline__ void block_max_key(unsigned v, unsigned* dst) {
  __shared__ unsigned red[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < NT / 32; ++w) t = max(t, red[w]);
    if (t) atomicMax(dst, t);
  }
  __syncthreads();
}

}  // namespace chisao

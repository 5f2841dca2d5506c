// Kernels that evaluate the objective: Phase 1 (batched L-BFGS, Sec. 3.2.1),
// the scale estimates at the start of Phases 5 and 6, Hands Like Clouds
// (Eq. 5), anti-convergence (Eq. 6), the L-BFGS direction alone, and plain
// objective evaluation.  Templated on objective kind, padded dimension DP
// (a group of DP/V lanes per sample, V = 4 coordinates per lane) and gradient
// mode.
#pragma once
#include "objectives.cuh"

namespace chisao {

constexpr int VL = 4;              // coordinates per lane
constexpr int NT_OBJ = 128;        // threads per block of the per-sample kernels
constexpr int NT_SCALES = 256;     // threads per block of the scale reduction
constexpr int SCALE_BLOCKS = 608;  // fixed grid of the scale reduction (4 x 152 SMs)
// HLC perturbations evaluated per pass over the objective's matrix (8 measured the same
// as 4 at d = 64 with 34 more registers)
constexpr int HLC_NP = 4;

template <int V>
__device__ __forceinline__ float dotv(const float (&a)[V], const float (&b)[V]) {
  float s = 0.f;
#pragma unroll
  for (int v = 0; v < V; ++v) s = fmaf(a[v], b[v], s);
  return s;
}

// L-BFGS two-loop recursion (Nocedal & Wright, Algorithm 7.4) on F = -f with
// the register-resident history (slot 0 newest), H0 = gam * I, in binary32
// with group-sum dot products.
template <int V, int LPS>
__device__ __forceinline__ void two_loop(const float (&s)[MMAX][V], const float (&y)[MMAX][V],
                                         const float (&rho)[MMAX], int len, float gam, const float (&G)[V],
                                         float (&p)[V], const Grp<LPS>& g) {
  float q[V], al[MMAX];
#pragma unroll
  for (int v = 0; v < V; ++v) q[v] = G[v];
#pragma unroll
  for (int k = 0; k < MMAX; ++k) {
    al[k] = 0.f;
    if (k < len) {
      al[k] = rho[k] * g.sum(dotv<V>(s[k], q));
#pragma unroll
      for (int v = 0; v < V; ++v) q[v] = fmaf(-al[k], y[k][v], q[v]);
    }
  }
  const float gm = len > 0 ? gam : 1.f;
#pragma unroll
  for (int v = 0; v < V; ++v) q[v] *= gm;
#pragma unroll
  for (int k = MMAX - 1; k >= 0; --k) {
    if (k < len) {
      const float be = rho[k] * g.sum(dotv<V>(y[k], q));
#pragma unroll
      for (int v = 0; v < V; ++v) q[v] = fmaf(s[k][v], al[k] - be, q[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) p[v] = -q[v];
}

// The same recursion over a history held in shared memory as a ring: logical slot
// k (0 newest) of this lane is row (head + k) mod MMAX of hs / hy, column t (one float4
// per lane and slot); rho stays in registers in logical order.
template <int LPS, int NC = NT_OBJ>
__device__ __forceinline__ void two_loop_ring(const float4 (*hs)[NC], const float4 (*hy)[NC], int head,
                                              const float (&rho)[MMAX], int len, float gam, const float (&G)[4],
                                              float (&p)[4], const Grp<LPS>& g, int t) {
  float q[4], al[MMAX];
#pragma unroll
  for (int v = 0; v < 4; ++v) q[v] = G[v];
#pragma unroll
  for (int k = 0; k < MMAX; ++k) {
    al[k] = 0.f;
    if (k < len) {
      const int r = head + k < MMAX ? head + k : head + k - MMAX;
      const float4 s4 = hs[r][t], y4 = hy[r][t];
      const float sv[4] = {s4.x, s4.y, s4.z, s4.w}, yv[4] = {y4.x, y4.y, y4.z, y4.w};
      al[k] = rho[k] * g.sum(dotv<4>(sv, q));
#pragma unroll
      for (int v = 0; v < 4; ++v) q[v] = fmaf(-al[k], yv[v], q[v]);
    }
  }
  const float gm = len > 0 ? gam : 1.f;
#pragma unroll
  for (int v = 0; v < 4; ++v) q[v] *= gm;
#pragma unroll
  for (int k = MMAX - 1; k >= 0; --k) {
    if (k < len) {
      const int r = head + k < MMAX ? head + k : head + k - MMAX;
      const float4 s4 = hs[r][t], y4 = hy[r][t];
      const float sv[4] = {s4.x, s4.y, s4.z, s4.w}, yv[4] = {y4.x, y4.y, y4.z, y4.w};
      const float be = rho[k] * g.sum(dotv<4>(yv, q));
#pragma unroll
      for (int v = 0; v < 4; ++v) q[v] = fmaf(sv[v], al[k] - be, q[v]);
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) p[v] = -q[v];
}

// History of sample i into registers; gam = s^T y / y^T y of the newest pair
// (s^T y = 1 / rho).
template <int DP, int V, int LPS>
__device__ __forceinline__ void load_history(const ProbDev& P, int i, int j0, int len, float (&s)[MMAX][V],
                                             float (&y)[MMAX][V], float (&rho)[MMAX], float& gam,
                                             const Grp<LPS>& g) {
#pragma unroll
  for (int k = 0; k < MMAX; ++k) {
    if (k < len) {
      const size_t o = ((size_t)i * MMAX + k) * DP + j0;
      ld_vec<V>(P.hs + o, s[k]);
      ld_vec<V>(P.hy + o, y[k]);
      rho[k] = P.hrho[(size_t)i * MMAX + k];
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) s[k][v] = y[k][v] = 0.f;
      rho[k] = 0.f;
    }
  }
  gam = 1.f;
  if (len > 0) gam = (1.0f / rho[0]) / g.sum(dotv<V>(y[0], y[0]));
}

// ------------------------------------------------------------------ Phase 1
// n_iter iterations of L-BFGS per sample, all in registers:
//   p = -H grad F (two-loop); restart with -grad F when p is an ascent direction
//   or not finite; backtracking Armijo over alpha0 2^-t on the box projection
//   x_t = clip(x + alpha p), F(x_t) <= F(x) + c1 grad F^T (x_t - x), first pass
//   wins (alpha0 = 1, or min(1, 1/|grad F|_inf) on an empty history); new
//   gradient; pair (s, y) kept iff s^T y > curv_eps |s||y| and 1/s^T y is finite
//   (a subnormal s^T y near a mode at the origin would give rho = inf), s^T y summed from
//   exact products in double-single.  A failed search clears the history.
// With a row list (rows, *nrows on the device) only those samples iterate:
// the final FP32 refinement of the survivors.
// Resident blocks per SM the fused Phase 1 asks the compiler for: with the history in
// shared memory (45 KB per block) the binary32 adjoint kernels of the cheaper
// objectives fit five blocks in 96 registers without spilling; the FP64 stencil
// and full-covariance variants keep the compiler's register choice.
template <int KIND, int GM>
constexpr int phase1_min_blocks() {
  return (GM == GRAD_ADJOINT && KIND != OBJ_MIXTURE_FULL) ? 5 : 1;
}

// The body takes the problem, its parameters and the block's index within the
// problem, so one problem's launch and a grouped launch over many problems share it.
template <int KIND, int DP, int GM>
__device__ __forceinline__ void phase1_body(const ProbDev& P, const StepParams& S, int n_iter, int fresh,
                                            const int* __restrict__ rows, const int* __restrict__ nrows,
                                            unsigned blk) {
  constexpr int V = VL, LPS = DP / V;
  static_assert(V == 4, "one float4 of history per lane and slot");
  using TE = EvalT<GM>;
  __shared__ float4 hist_s[MMAX][NT_OBJ], hist_y[MMAX][NT_OBJ];
  const Grp<LPS> g;
  const int gi = (int)(((size_t)blk * NT_OBJ + threadIdx.x) / LPS);
  const bool act = rows ? gi < *nrows : gi < P.n;
  const int i = rows ? (act ? rows[gi] : 0) : gi;
  EvalCount ec;
  unsigned long long trials = 0, fails = 0;
  if (act) {
    const int j0 = V * g.l;
    float x[V], lo[V], hi[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    ld_vec<V>(P.lo + j0, lo);
    ld_vec<V>(P.hi + j0, hi);
    int len = P.hlen[i];
    float rho[MMAX], gam = 1.f;
    const float curv_eps = (float)S.curv_eps;
    // the (s, y) history lives in shared memory (a ring per lane, logical slot k at row
    // head + k mod MMAX): registers hold only rho, which keeps more samples resident
    int head = 0;
#pragma unroll
    for (int k = 0; k < MMAX; ++k) {
      if (k < len) {
        const size_t o = ((size_t)i * MMAX + k) * DP + j0;
        hist_s[k][threadIdx.x] = *reinterpret_cast<const float4*>(P.hs + o);
        hist_y[k][threadIdx.x] = *reinterpret_cast<const float4*>(P.hy + o);
        rho[k] = P.hrho[(size_t)i * MMAX + k];
      } else {
        rho[k] = 0.f;
      }
    }
    if (len > 0) {                                 // gam = s^T y / y^T y of the newest pair
      const float4 y4 = hist_y[0][threadIdx.x];
      const float y0[V] = {y4.x, y4.y, y4.z, y4.w};
      gam = (1.0f / rho[0]) / g.sum(dotv<V>(y0, y0));
    }
    TE F;
    float G[V];
    if (fresh) {
      float a[V];
      F = -value_and_gradient<KIND, GM, V, LPS>(P.obj, S, P.d, x, a, g, ec);
#pragma unroll
      for (int v = 0; v < V; ++v) G[v] = -a[v];
    } else {
      F = -(TE)P.f[i];
      ld_vec<V>(P.g + (size_t)i * DP + j0, G);
#pragma unroll
      for (int v = 0; v < V; ++v) G[v] = -G[v];
    }
    for (int it = 0; it < n_iter; ++it) {
      float gl = 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v) gl = fmaxf(gl, fabsf(G[v]));
      const float gn = g.maxf(gl);
      if (!(gn > 0.f)) break;                      // exactly stationary (or invalid): stays put
      float p[V];
      two_loop_ring<LPS>(hist_s, hist_y, head, rho, len, gam, G, p, g, (int)threadIdx.x);
      float a0 = len > 0 ? 1.f : fminf(1.f, 1.f / gn);
      const float gp = g.sum(dotv<V>(G, p));
      // restart when p is an ascent direction or not finite; g^T p = 0 (the product
      // underflows next to a stationary point) keeps the history, the mode's curvature
      if (!(gp <= 0.f)) {
        len = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) p[v] = -G[v];
        a0 = fminf(1.f, 1.f / gn);
      }
      bool acc = false;
      float xt[V], Gt[V];
      TE Ft = F;
      for (int t = 0; t < S.T_ls; ++t) {
        const float a = ldexpf(a0, -t);
        float c[V], ga[V];
        TE dl = TE(0);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          c[v] = clampf(fmaf(a, p[v], x[v]), lo[v], hi[v]);
          dl += (TE)G[v] * ((TE)c[v] - (TE)x[v]);
          ga[v] = 0.f;
        }
        TE ft;
        if constexpr (GM == GRAD_ADJOINT) {
          ft = value_grad_noisy<KIND, V, LPS>(P.obj, S, c, ga, g);
          ec.evals += 1;
          ec.grads += 1;
        } else {
          TE ce[V];
#pragma unroll
          for (int v = 0; v < V; ++v) ce[v] = (TE)c[v];
          ft = value_noisy<KIND, TE, V, LPS>(P.obj, params_of<GM>(P.obj), S, ce, g);
          ec.evals += 1;
        }
        ++trials;
        const TE dec = g.sum(dl);
        if (-ft <= F + (TE)S.c1 * dec) {
          acc = true;
          Ft = -ft;
#pragma unroll
          for (int v = 0; v < V; ++v) {
            xt[v] = c[v];
            Gt[v] = -ga[v];
          }
          break;
        }
      }
      if (!acc) {
        len = 0;
        ++fails;
        continue;
      }
      if constexpr (GM != GRAD_ADJOINT) {
        float ag[V];
        gradient_only<KIND, GM, V, LPS>(P.obj, S, P.d, xt, ag, g, ec);
#pragma unroll
        for (int v = 0; v < V; ++v) Gt[v] = -ag[v];
      }
      float sv[V], yv[V];
      float syh = 0.f, syl = 0.f, ss = 0.f, yy = 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        sv[v] = xt[v] - x[v];
        yv[v] = Gt[v] - G[v];
        const float pr = sv[v] * yv[v];             // exact product as pr + err
        ff_add(syh, syl, pr, fmaf(sv[v], yv[v], -pr));
        ss = fmaf(sv[v], sv[v], ss);
        yy = fmaf(yv[v], yv[v], yy);
      }
      g.ff_sum(syh, syl);                            // s^T y, compensated
      const float sy = syh + syl;
      ss = g.sum(ss);                                // sums of squares: no cancellation
      yy = g.sum(yy);
      const float rsy = 1.0f / sy;
      if (sy > curv_eps * sqrtf(ss) * sqrtf(yy) && rsy <= FLT_MAX) {   // rho = 1/s^T y finite
#pragma unroll
        for (int k = MMAX - 1; k > 0; --k) rho[k] = rho[k - 1];
        head = head == 0 ? MMAX - 1 : head - 1;      // the oldest row takes the newest pair
        hist_s[head][threadIdx.x] = make_float4(sv[0], sv[1], sv[2], sv[3]);
        hist_y[head][threadIdx.x] = make_float4(yv[0], yv[1], yv[2], yv[3]);
        rho[0] = rsy;
        len = min(len + 1, S.m);
        gam = sy / yy;
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        x[v] = xt[v];
        G[v] = Gt[v];
      }
      F = Ft;
    }
    float gout[V];
#pragma unroll
    for (int v = 0; v < V; ++v) gout[v] = -G[v];
    st_vec<V>(P.x + (size_t)i * DP + j0, x);
    st_vec<V>(P.g + (size_t)i * DP + j0, gout);
#pragma unroll
    for (int k = 0; k < MMAX; ++k) {
      if (k < len) {
        const size_t o = ((size_t)i * MMAX + k) * DP + j0;
        const int r = head + k < MMAX ? head + k : head + k - MMAX;
        *reinterpret_cast<float4*>(P.hs + o) = hist_s[r][threadIdx.x];
        *reinterpret_cast<float4*>(P.hy + o) = hist_y[r][threadIdx.x];
        if (g.l == 0) P.hrho[(size_t)i * MMAX + k] = rho[k];
      }
    }
    if (g.l == 0) {
      P.f[i] = (float)(-F);
      P.hlen[i] = len;
    } else {
      ec.evals = ec.grads = 0;
      trials = fails = 0;
    }
  }
  block_add_u64<NT_OBJ>(ec.evals, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ec.grads, &P.cnt->grads);
  block_add_u64<NT_OBJ>(trials, &P.cnt->ls_trials);
  block_add_u64<NT_OBJ>(fails, &P.cnt->ls_fail);
}

template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ, phase1_min_blocks<KIND, GM>()) k_phase1(ProbDev P, StepParams S, int n_iter, int fresh,
                                                   const int* __restrict__ rows, const int* __restrict__ nrows) {
  phase1_body<KIND, DP, GM>(P, S, n_iter, fresh, rows, nrows, blockIdx.x);
}

// Phase 1 for samples of at most sixteen coordinates (a group of DP / 4 lanes each) with
// finite-difference gradients.  There a sample's iteration is a serial chain of evaluations:
// up to T_ls Armijo trials (all of them at a mode, where no step decreases F) and the 2d
// stencil points of the new gradient.  Here P1_W groups share a sample and keep identical
// copies of its state: a batch of P1_W trials is evaluated side by side (group q trial t0 + q)
// and the first that passes is taken, which is the step sequential backtracking takes, and the
// stencil points are spread over the groups (fd_gradient_wide).  Every value is the one
// phase1_body computes, so the results (and the counters, which count the trials and
// evaluations of the sequential search) are the same bit for bit.
constexpr int P1_W = 8;

// The lanes of one sample: P1_W groups of LPS lanes, aligned in the warp.
template <int LPS>
__device__ __forceinline__ unsigned wide_mask() {
  constexpr int SL = P1_W * LPS;
  const int lane = threadIdx.x & 31;
  return SL == 32 ? 0xffffffffu : ((1u << SL) - 1u) << (lane & ~(SL - 1));
}

// Central differences with the 2d stencil values spread over the P1_W groups of a sample
// (group q evaluates the points s = 8 r + q, r < LPS: coordinate s / 2, plus for even s,
// minus for odd s), combined on every group exactly as fd_gradient combines them.  Lane l's
// coordinates 4 l + v take their two values from round l of groups 2 v and 2 v + 1.
template <int KIND, int GM, int LPS>
__device__ __forceinline__ void fd_gradient_wide(const ObjDev& O, const StepParams& S, int d, const float (&xf)[4],
                                                 float (&gr)[4], const Grp<LPS>& g, int q, unsigned smask) {
  using TE = EvalT<GM>;
  constexpr int SL = P1_W * LPS;
  const auto& o = params_of<GM>(O);
  TE x[4], hs[4], fr[LPS];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    x[v] = (TE)xf[v];
    gr[v] = 0.f;
    hs[v] = (GM == GRAD_FD32) ? (TE)S.h_rel * fmax((TE)1, fabs(x[v])) : (TE)S.h;
  }
#pragma unroll
  for (int r = 0; r < LPS; ++r) {
    const int sp = P1_W * r + q, js = sp >> 1;
    fr[r] = TE(0);
    if (js < d) {
      TE y[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        y[v] = x[v];
        if (g.l == (js >> 2) && v == (js & 3)) y[v] = (sp & 1) ? stencil_sub(x[v], hs[v]) : stencil_add(x[v], hs[v]);
      }
      fr[r] = value_noisy<KIND, TE, 4, LPS>(O, o, S, y, g);
    }
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    TE fp = TE(0), fm = TE(0);
#pragma unroll
    for (int r = 0; r < LPS; ++r) {
      const TE a = __shfl_sync(smask, fr[r], (2 * v) * LPS + g.l, SL);
      const TE b = __shfl_sync(smask, fr[r], (2 * v + 1) * LPS + g.l, SL);
      if (r == g.l) {
        fp = a;
        fm = b;
      }
    }
    if (4 * g.l + v < d) {
      const TE xp = stencil_add(x[v], hs[v]), xm = stencil_sub(x[v], hs[v]);
      gr[v] = (float)((fp - fm) / (xp - xm));
    }
  }
}

template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_phase1_wide(ProbDev P, StepParams S, int n_iter, int fresh,
                                                        const int* __restrict__ rows, const int* __restrict__ nrows) {
  constexpr int V = VL, LPS = DP / V, SL = P1_W * LPS, NC = NT_OBJ / P1_W;   // ring columns per block
  static_assert(GM != GRAD_ADJOINT, "finite-difference gradients");
  static_assert(SL <= 32, "a sample within one warp");
  using TE = EvalT<GM>;
  __shared__ float4 hist_s[MMAX][NC], hist_y[MMAX][NC];        // one ring per sample, shared by its groups
  const Grp<LPS> g;
  const int lane = threadIdx.x & 31, q = (lane / LPS) & (P1_W - 1);
  const int col = (int)(threadIdx.x / SL) * LPS + g.l;
  const unsigned smask = wide_mask<LPS>();
  const int gi = (int)(((size_t)blockIdx.x * NT_OBJ + threadIdx.x) / SL);
  const bool act = rows ? gi < *nrows : gi < P.n;
  const int i = rows ? (act ? rows[gi] : 0) : gi;
  unsigned long long evals = 0, grads = 0, trials = 0, fails = 0;
  if (act) {
    const int j0 = V * g.l;
    float x[V], lo[V], hi[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    ld_vec<V>(P.lo + j0, lo);
    ld_vec<V>(P.hi + j0, hi);
    int len = P.hlen[i];
    float rho[MMAX], gam = 1.f;
    int head = 0;
#pragma unroll
    for (int k = 0; k < MMAX; ++k) {
      rho[k] = 0.f;
      if (k < len) {
        const size_t o = ((size_t)i * MMAX + k) * DP + j0;
        if (q == 0) {
          hist_s[k][col] = *reinterpret_cast<const float4*>(P.hs + o);
          hist_y[k][col] = *reinterpret_cast<const float4*>(P.hy + o);
        }
        rho[k] = P.hrho[(size_t)i * MMAX + k];
      }
    }
    __syncwarp(smask);
    if (len > 0) {
      const float4 y4 = hist_y[0][col];
      const float y0[V] = {y4.x, y4.y, y4.z, y4.w};
      gam = (1.0f / rho[0]) / g.sum(dotv<V>(y0, y0));
    }
    TE F;
    float G[V];
    if (fresh) {
      TE xe[V];
#pragma unroll
      for (int v = 0; v < V; ++v) xe[v] = (TE)x[v];
      F = -value_noisy<KIND, TE, V, LPS>(P.obj, params_of<GM>(P.obj), S, xe, g);
      float a[V];
      fd_gradient_wide<KIND, GM, LPS>(P.obj, S, P.d, x, a, g, q, smask);
      evals += 1 + 2ull * P.d;
      grads += 1;
#pragma unroll
      for (int v = 0; v < V; ++v) G[v] = -a[v];
    } else {
      F = -(TE)P.f[i];
      ld_vec<V>(P.g + (size_t)i * DP + j0, G);
#pragma unroll
      for (int v = 0; v < V; ++v) G[v] = -G[v];
    }
    for (int it = 0; it < n_iter; ++it) {
      float gl = 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v) gl = fmaxf(gl, fabsf(G[v]));
      const float gn = g.maxf(gl);
      if (!(gn > 0.f)) break;                        // exactly stationary (or invalid): stays put
      float p[V];
      two_loop_ring<LPS, NC>(hist_s, hist_y, head, rho, len, gam, G, p, g, col);
      float a0 = len > 0 ? 1.f : fminf(1.f, 1.f / gn);
      const float gp = g.sum(dotv<V>(G, p));
      if (!(gp <= 0.f)) {
        len = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) p[v] = -G[v];
        a0 = fminf(1.f, 1.f / gn);
      }
      // the trials in batches of P1_W: the first that passes wins
      int tacc = -1;
      TE Ft = F;
      for (int t0 = 0; t0 < S.T_ls && tacc < 0; t0 += P1_W) {
        const int t = t0 + q;
        bool pass = false;
        TE ft = TE(0);
        if (t < S.T_ls) {
          const float a = ldexpf(a0, -t);
          float c[V];
          TE ce[V];
          TE dl = TE(0);
#pragma unroll
          for (int v = 0; v < V; ++v) {
            c[v] = clampf(fmaf(a, p[v], x[v]), lo[v], hi[v]);
            dl += (TE)G[v] * ((TE)c[v] - (TE)x[v]);
            ce[v] = (TE)c[v];
          }
          ft = value_noisy<KIND, TE, V, LPS>(P.obj, params_of<GM>(P.obj), S, ce, g);
          const TE dec = g.sum(dl);
          pass = -ft <= F + (TE)S.c1 * dec;
        }
        const unsigned b = (__ballot_sync(smask, pass) & smask) >> (lane & ~(SL - 1));
        unsigned gb = 0;                              // one bit per group (its lanes agree)
#pragma unroll
        for (int w = 0; w < P1_W; ++w) gb |= ((b >> (w * LPS)) & 1u) << w;
        const int nt = min(P1_W, S.T_ls - t0);
        if (gb) {
          const int w = __ffs(gb) - 1;
          tacc = t0 + w;
          Ft = -__shfl_sync(smask, ft, w * LPS + g.l, SL);
          trials += w + 1;
          evals += w + 1;
        } else {
          trials += nt;
          evals += nt;
        }
      }
      if (tacc < 0) {
        len = 0;
        ++fails;
        continue;
      }
      float xt[V], Gt[V];
      {
        const float a = ldexpf(a0, -tacc);
#pragma unroll
        for (int v = 0; v < V; ++v) xt[v] = clampf(fmaf(a, p[v], x[v]), lo[v], hi[v]);
      }
      {
        float ag[V];
        fd_gradient_wide<KIND, GM, LPS>(P.obj, S, P.d, xt, ag, g, q, smask);
        evals += 2ull * P.d;
        grads += 1;
#pragma unroll
        for (int v = 0; v < V; ++v) Gt[v] = -ag[v];
      }
      float sv[V], yv[V];
      float syh = 0.f, syl = 0.f, ss = 0.f, yy = 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        sv[v] = xt[v] - x[v];
        yv[v] = Gt[v] - G[v];
        const float pr = sv[v] * yv[v];
        ff_add(syh, syl, pr, fmaf(sv[v], yv[v], -pr));
        ss = fmaf(sv[v], sv[v], ss);
        yy = fmaf(yv[v], yv[v], yy);
      }
      g.ff_sum(syh, syl);
      const float sy = syh + syl;
      ss = g.sum(ss);
      yy = g.sum(yy);
      const float rsy = 1.0f / sy;
      if (sy > (float)S.curv_eps * sqrtf(ss) * sqrtf(yy) && rsy <= FLT_MAX) {
#pragma unroll
        for (int k = MMAX - 1; k > 0; --k) rho[k] = rho[k - 1];
        head = head == 0 ? MMAX - 1 : head - 1;
        __syncwarp(smask);                           // every lane has read the row it replaces
        if (q == 0) {
          hist_s[head][col] = make_float4(sv[0], sv[1], sv[2], sv[3]);
          hist_y[head][col] = make_float4(yv[0], yv[1], yv[2], yv[3]);
        }
        __syncwarp(smask);
        rho[0] = rsy;
        len = min(len + 1, S.m);
        gam = sy / yy;
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        x[v] = xt[v];
        G[v] = Gt[v];
      }
      F = Ft;
    }
    if (q == 0) {
      float gout[V];
#pragma unroll
      for (int v = 0; v < V; ++v) gout[v] = -G[v];
      st_vec<V>(P.x + (size_t)i * DP + j0, x);
      st_vec<V>(P.g + (size_t)i * DP + j0, gout);
#pragma unroll
      for (int k = 0; k < MMAX; ++k) {
        if (k < len) {
          const size_t o = ((size_t)i * MMAX + k) * DP + j0;
          const int r = head + k < MMAX ? head + k : head + k - MMAX;
          *reinterpret_cast<float4*>(P.hs + o) = hist_s[r][col];
          *reinterpret_cast<float4*>(P.hy + o) = hist_y[r][col];
          if (g.l == 0) P.hrho[(size_t)i * MMAX + k] = rho[k];
        }
      }
      if (g.l == 0) {
        P.f[i] = (float)(-F);
        P.hlen[i] = len;
      }
    }
    if (q != 0 || g.l != 0) evals = grads = trials = fails = 0;
  }
  block_add_u64<NT_OBJ>(evals, &P.cnt->evals);
  block_add_u64<NT_OBJ>(grads, &P.cnt->grads);
  block_add_u64<NT_OBJ>(trials, &P.cnt->ls_trials);
  block_add_u64<NT_OBJ>(fails, &P.cnt->ls_fail);
}

// The gradients a scale pass needs, for samples of at most sixteen coordinates with finite
// differences, on P1_W groups per sample (fd_gradient_wide): every unfrozen sample, or with
// removed_only those Phase 4 reseeded (the others keep Phase 1's).  The scale pass then reads
// them (reuse = 2) and sums in its own fixed order, so sigma and alpha are the one-group
// pass's bit for bit.
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_grad_wide(ProbDev P, StepParams S, int removed_only) {
  constexpr int V = VL, LPS = DP / V, SL = P1_W * LPS;
  static_assert(GM != GRAD_ADJOINT, "finite-difference gradients");
  const Grp<LPS> g;
  const int lane = threadIdx.x & 31, q = (lane / LPS) & (P1_W - 1);
  const unsigned smask = wide_mask<LPS>();
  const int i = (int)(((size_t)blockIdx.x * NT_OBJ + threadIdx.x) / SL);
  unsigned long long evals = 0, grads = 0;
  if (i < P.n && !bit_of(P.stuck, i) && (!removed_only || bit_of(P.removed, i))) {
    const int j0 = V * g.l;
    float x[V], a[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    fd_gradient_wide<KIND, GM, LPS>(P.obj, S, P.d, x, a, g, q, smask);
    if (q == 0) {
      st_vec<V>(P.g + (size_t)i * DP + j0, a);
      if (g.l == 0) {
        evals = 2ull * P.d;
        grads = 1;
      }
    }
  }
  block_add_u64<NT_OBJ>(evals, &P.cnt->evals);
  block_add_u64<NT_OBJ>(grads, &P.cnt->grads);
}

// Anti-convergence (Eq. 6) for samples of at most sixteen coordinates with finite
// differences: anti_body's steps with each step's gradient evaluated on P1_W groups
// (fd_gradient_wide); the groups keep identical copies of the sample's position and velocity.
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_anti_wide(ProbDev P, StepParams S) {
  constexpr int V = VL, LPS = DP / V, SL = P1_W * LPS;
  static_assert(GM != GRAD_ADJOINT, "finite-difference gradients");
  const Grp<LPS> g;
  const int lane = threadIdx.x & 31, q = (lane / LPS) & (P1_W - 1);
  const unsigned smask = wide_mask<LPS>();
  const int i = (int)(((size_t)blockIdx.x * NT_OBJ + threadIdx.x) / SL);
  unsigned long long evals = 0, grads = 0;
  if (i < P.n && !bit_of(P.stuck, i) && P.cnt->sc_count > 0) {
    const int j0 = V * g.l;
    const float alpha = P.cnt->sc_alpha, mu = S.mu;
    float x[V], gr[V], vel[V], lo[V], hi[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    ld_vec<V>(P.g + (size_t)i * DP + j0, gr);
    ld_vec<V>(P.lo + j0, lo);
    ld_vec<V>(P.hi + j0, hi);
#pragma unroll
    for (int v = 0; v < V; ++v) vel[v] = 0.f;
    for (int t = 0; t < S.n_anti; ++t) {
      if (t > 0) {
        fd_gradient_wide<KIND, GM, LPS>(P.obj, S, P.d, x, gr, g, q, smask);
        evals += 2ull * P.d;
        grads += 1;
      }
#pragma unroll
      for (int v = 0; v < V; ++v) {
        vel[v] = mu * vel[v] - alpha * gr[v];
        const float nx = x[v] + vel[v];
        const float cx = clampf(nx, lo[v], hi[v]);
        if (cx != nx) vel[v] = 0.f;
        x[v] = cx;
      }
    }
    if (q == 0) {
      st_vec<V>(P.x + (size_t)i * DP + j0, x);
      if (g.l == 0) P.hlen[i] = 0;
    }
    if (q != 0 || g.l != 0) evals = grads = 0;
  }
  block_add_u64<NT_OBJ>(evals, &P.cnt->evals);
  block_add_u64<NT_OBJ>(grads, &P.cnt->grads);
}

// Phase 1 of every problem of a group in one launch (n_conv iterations each, fresh gradient).
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ, phase1_min_blocks<KIND, GM>()) k_phase1_grp(GroupTab T) {
  const int q = T.blk_prob[blockIdx.x];
  const StepParams& S = T.sps[q];
  phase1_body<KIND, DP, GM>(T.probs[q], S, S.n_conv, 1, nullptr, nullptr, blockIdx.x - (unsigned)T.blk_first[q]);
}

// Direction only (test hook): p = -H grad F written into g.
template <int DP>
__global__ void __launch_bounds__(NT_OBJ) k_direction(ProbDev P) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  if (i >= P.n) return;
  const int j0 = V * g.l;
  const int len = P.hlen[i];
  float s[MMAX][V], y[MMAX][V], rho[MMAX], gam, G[V], p[V];
  load_history<DP, V, LPS>(P, i, j0, len, s, y, rho, gam, g);
  ld_vec<V>(P.g + (size_t)i * DP + j0, G);
#pragma unroll
  for (int v = 0; v < V; ++v) G[v] = -G[v];
  two_loop<V, LPS>(s, y, rho, len, gam, G, p, g);
  st_vec<V>(P.g + (size_t)i * DP + j0, p);
}

// ------------------------------------------------------------------ scales (Phase 5/6 start)
// Gradient at every unfrozen sample (stored in g) and per-block partial sums
// (sum x_j, sum x_j^2 per coordinate, sum |g|^2, count), accumulated in
// double-single and reduced in a fixed order so the result is deterministic.
template <int KIND, int DP, int GM>
__device__ __forceinline__ void scales_body(const ProbDev& P, const StepParams& S, unsigned blk, unsigned nblk,
                                            int reuse) {
  constexpr int V = VL, LPS = DP / V;
  constexpr int GPB = NT_SCALES / LPS;             // groups per block
  constexpr int W = 2 * DP + 2;
  __shared__ float2 buf[GPB][W];
  const Grp<LPS> g;
  const int grp = threadIdx.x / LPS;
  const int j0 = V * g.l;
  EvalCount ec;
  float sxh[V], sxl[V], sqh[V], sql[V], sgh = 0.f, sgl = 0.f;
#pragma unroll
  for (int v = 0; v < V; ++v) sxh[v] = sxl[v] = sqh[v] = sql[v] = 0.f;
  int cnt = 0;
  auto add = [&](const float (&x)[V], const float (&a)[V]) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      ff_add(sxh[v], sxl[v], x[v], 0.f);
      const float p2 = x[v] * x[v];
      ff_add(sqh[v], sql[v], p2, fmaf(x[v], x[v], -p2));
    }
    ff_add(sgh, sgl, g.sum(dotv<V>(a, a)), 0.f);    // sum of squares: no cancellation
    ++cnt;
  };
  for (int i = (int)blk * GPB + grp; i < P.n; i += (int)nblk * GPB) {
    if (bit_of(P.stuck, i)) continue;
    float x[V], a[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    if constexpr (GM == GRAD_GIVEN) {
      ld_vec<V>(P.g + (size_t)i * DP + j0, a);          // computed by the batched evaluator
      ec.evals += 1;
      ec.grads += 1;
    } else if (reuse == 2 || (reuse && !bit_of(P.removed, i))) {
      // Phase 1 left the gradient at this point in g and nothing has moved the sample
      // since (only the reseeded slots, the removed ones, have): the same bits.  With
      // reuse = 2 a wide pre-pass (k_grad_wide) has just stored every gradient needed.
      ld_vec<V>(P.g + (size_t)i * DP + j0, a);
    } else {
      gradient_only<KIND, GM, V, LPS>(P.obj, S, P.d, x, a, g, ec);
      st_vec<V>(P.g + (size_t)i * DP + j0, a);
    }
    add(x, a);
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    buf[grp][j0 + v] = make_float2(sxh[v], sxl[v]);
    buf[grp][DP + j0 + v] = make_float2(sqh[v], sql[v]);
  }
  if (g.l == 0) {
    buf[grp][2 * DP] = make_float2(sgh, sgl);
    buf[grp][2 * DP + 1] = make_float2((float)cnt, 0.f);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < W; t += blockDim.x) {
    float h = 0.f, l = 0.f;
    for (int q = 0; q < GPB; ++q) ff_add(h, l, buf[q][t].x, buf[q][t].y);
    P.partials[(size_t)blk * W + t] = make_float2(h, l);
  }
  if (g.l != 0) ec.evals = ec.grads = 0;
  block_add_u64<NT_SCALES>(ec.evals, &P.cnt->evals);
  block_add_u64<NT_SCALES>(ec.grads, &P.cnt->grads);
}

// reuse = 1 at the start of Phase 5: the gradients Phase 1 stored are still those of the
// current points except at the reseeded slots
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_SCALES) k_scales(ProbDev P, StepParams S, int reuse) {
  scales_body<KIND, DP, GM>(P, S, blockIdx.x, gridDim.x, reuse);
}

// The scale pass of every problem of a group (its own partial-sum grid each).
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_SCALES) k_scales_grp(GroupTab T, int reuse) {
  const int q = T.blk_prob[blockIdx.x];
  scales_body<KIND, DP, GM>(T.probs[q], T.sps[q], blockIdx.x - (unsigned)T.blk_first[q], (unsigned)T.blk_count[q],
                            reuse);
}

// ------------------------------------------------------------------ Phase 5
// n_cloud steps x <- clip(x + alpha (1/M) sum_k grad f(x + sigma z_k)) on the
// unfrozen samples; z_k from the HLC Philox stream (row = sample, step = cloud
// step, k = perturbation).  History is cleared (the sample moved).
template <int KIND, int DP, int GM>
__device__ __forceinline__ void hlc_body(const ProbDev& P, const StepParams& S, unsigned blk) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blk * NT_OBJ + threadIdx.x) / LPS);
  EvalCount ec;
  if (i < P.n && !bit_of(P.stuck, i) && P.cnt->sc_count > 0) {
    const int j0 = V * g.l;
    const unsigned cyc = (unsigned)P.cnt->cycle + 1u;
    const float sigma = P.cnt->sc_sigma, alpha = P.cnt->sc_alpha;
    float x[V], lo[V], hi[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    ld_vec<V>(P.lo + j0, lo);
    ld_vec<V>(P.hi + j0, hi);
    const float invM = 1.0f / (float)S.M;
    using TE = EvalT<GM>;
    for (int t = 0; t < S.n_cloud; ++t) {
      float acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = 0.f;
      // value-only variant: f at the centre once per step
      const TE f0 = S.hlc_value_only ? value_at<KIND, GM, V, LPS>(P.obj, S, x, g, ec) : TE(0);
      for (int k = 0; k < S.M; ++k) {
        float z[V], xp[V], a[V];
        normals_lane<V>(S, (unsigned)i, g.l, TAG_HLC, cyc, (unsigned)t, (unsigned)P.obj.prob_index,
                        (unsigned)k, z);
#pragma unroll
        for (int v = 0; v < V; ++v) xp[v] = (j0 + v < P.d) ? fmaf(sigma, z[v], x[v]) : x[v];
        if (S.hlc_value_only) {
          // (f(x + sigma z) - f(x)) z / sigma, the difference formed in the evaluation precision
          const float w = (float)((value_at<KIND, GM, V, LPS>(P.obj, S, xp, g, ec) - f0) / (TE)sigma);
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = fmaf(w, (j0 + v < P.d) ? z[v] : 0.f, acc[v]);
        } else if (GM == GRAD_ADJOINT && HasMulti<KIND>::value && k + HLC_NP - 1 < S.M) {
          // HLC_NP perturbations at once (one pass over the matrix); the sum keeps the
          // order of the one-at-a-time loop
          float zq[HLC_NP][V], xq[HLC_NP][V], aq[HLC_NP][V], fq[HLC_NP];
#pragma unroll
          for (int p = 0; p < HLC_NP; ++p) {
            normals_lane<V>(S, (unsigned)i, g.l, TAG_HLC, cyc, (unsigned)t, (unsigned)P.obj.prob_index,
                            (unsigned)(k + p), zq[p]);
#pragma unroll
            for (int v = 0; v < V; ++v) xq[p][v] = (j0 + v < P.d) ? fmaf(sigma, zq[p][v], x[v]) : x[v];
          }
          if constexpr (HasMulti<KIND>::value)
            Obj<KIND>::template value_grad_multi<HLC_NP, V, LPS>(P.obj.f32, xq, aq, fq, g);
          ec.evals += HLC_NP;
          ec.grads += HLC_NP;
#pragma unroll
          for (int p = 0; p < HLC_NP; ++p)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += aq[p][v];
          k += HLC_NP - 1;
        } else if (GM == GRAD_ADJOINT && HasPair<KIND>::value && k + 1 < S.M) {
          // two perturbations at once, sharing the objective's parameter loads; the sum
          // keeps the order of the one-at-a-time loop
          float z2[V], xp2[V], a2[V], fa, fb;
          normals_lane<V>(S, (unsigned)i, g.l, TAG_HLC, cyc, (unsigned)t, (unsigned)P.obj.prob_index,
                          (unsigned)(k + 1), z2);
#pragma unroll
          for (int v = 0; v < V; ++v) xp2[v] = (j0 + v < P.d) ? fmaf(sigma, z2[v], x[v]) : x[v];
          if constexpr (HasPair<KIND>::value)
            Obj<KIND>::template value_grad_pair<V, LPS>(P.obj.f32, xp, xp2, a, a2, fa, fb, g);
          ec.evals += 2;
          ec.grads += 2;
#pragma unroll
          for (int v = 0; v < V; ++v) {
            acc[v] += a[v];
            acc[v] += a2[v];
          }
          ++k;
        } else {
          gradient_only<KIND, GM, V, LPS>(P.obj, S, P.d, xp, a, g, ec);
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] += a[v];
        }
      }
#pragma unroll
      for (int v = 0; v < V; ++v) x[v] = clampf(fmaf(alpha, acc[v] * invM, x[v]), lo[v], hi[v]);
    }
    st_vec<V>(P.x + (size_t)i * DP + j0, x);
    if (g.l == 0) P.hlen[i] = 0;
    else ec.evals = ec.grads = 0;
  }
  block_add_u64<NT_OBJ>(ec.evals, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ec.grads, &P.cnt->grads);
}

// Hands Like Clouds for samples of at most sixteen coordinates (a group of DP / 4 lanes each)
// with finite-difference gradients: the gradient at each perturbed point is a serial chain of
// 2d evaluations, and one group per sample would run the M chains of a step one after another.
// Here HLC_W groups share a sample: group k draws perturbation k's normals and evaluates its
// gradient (the same calls as the one-group loop), and every group adds the M gradients in the
// order k = 0, 1, ... by shuffles, so the step is the one-group kernel's bit for bit with
// M-fold shorter chains and HLC_W times the warps.  Used when M <= HLC_W and the gradient
// estimator is Eq. 5's (not the value-only variant).
constexpr int HLC_W = 8;
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_hlc_wide(ProbDev P, StepParams S) {
  constexpr int V = VL, LPS = DP / V, SL = HLC_W * LPS;      // lanes per sample
  static_assert(GM != GRAD_ADJOINT, "exact gradients keep the paired and multi-point products of k_hlc");
  static_assert(SL <= 32, "a sample within one warp");
  const Grp<LPS> g;                                         // this group's lanes (one copy of the sample)
  const int lane = threadIdx.x & 31;
  const int k = (lane / LPS) & (HLC_W - 1);                // this group's perturbation
  const unsigned smask = SL == 32 ? 0xffffffffu : ((1u << SL) - 1u) << (lane & ~(SL - 1));
  const int i = (int)(((size_t)blockIdx.x * NT_OBJ + threadIdx.x) / SL);
  EvalCount ec;
  if (i < P.n && !bit_of(P.stuck, i) && P.cnt->sc_count > 0) {
    const int j0 = V * g.l;
    const unsigned cyc = (unsigned)P.cnt->cycle + 1u;
    const float sigma = P.cnt->sc_sigma, alpha = P.cnt->sc_alpha;
    float x[V], lo[V], hi[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    ld_vec<V>(P.lo + j0, lo);
    ld_vec<V>(P.hi + j0, hi);
    const float invM = 1.0f / (float)S.M;
    for (int t = 0; t < S.n_cloud; ++t) {
      float a[V];
#pragma unroll
      for (int v = 0; v < V; ++v) a[v] = 0.f;
      if (k < S.M) {
        float z[V], xp[V];
        normals_lane<V>(S, (unsigned)i, g.l, TAG_HLC, cyc, (unsigned)t, (unsigned)P.obj.prob_index, (unsigned)k,
                        z);
#pragma unroll
        for (int v = 0; v < V; ++v) xp[v] = (j0 + v < P.d) ? fmaf(sigma, z[v], x[v]) : x[v];
        gradient_only<KIND, GM, V, LPS>(P.obj, S, P.d, xp, a, g, ec);
      }
      float acc[V];
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] = 0.f;
#pragma unroll
      for (int q = 0; q < HLC_W; ++q)
        if (q < S.M) {
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] += __shfl_sync(smask, a[v], q * LPS + g.l, SL);
        }
#pragma unroll
      for (int v = 0; v < V; ++v) x[v] = clampf(fmaf(alpha, acc[v] * invM, x[v]), lo[v], hi[v]);
    }
    if (k == 0) {
      st_vec<V>(P.x + (size_t)i * DP + j0, x);
      if (g.l == 0) P.hlen[i] = 0;
    }
    if (g.l != 0) ec.evals = ec.grads = 0;
  }
  block_add_u64<NT_OBJ>(ec.evals, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ec.grads, &P.cnt->grads);
}

template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_hlc(ProbDev P, StepParams S) {
  hlc_body<KIND, DP, GM>(P, S, blockIdx.x);
}

template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_hlc_grp(GroupTab T) {
  const int q = T.blk_prob[blockIdx.x];
  hlc_body<KIND, DP, GM>(T.probs[q], T.sps[q], blockIdx.x - (unsigned)T.blk_first[q]);
}

// ------------------------------------------------------------------ Phase 6
// n_anti momentum steps v <- mu v - alpha grad f(x), x <- clip(x + v), v = 0
// on coordinates the projection moved; v_0 = 0; the first gradient is the one
// the scale pass stored.  History is cleared.
template <int KIND, int DP, int GM>
__device__ __forceinline__ void anti_body(const ProbDev& P, const StepParams& S, unsigned blk) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blk * NT_OBJ + threadIdx.x) / LPS);
  EvalCount ec;
  if (i < P.n && !bit_of(P.stuck, i) && P.cnt->sc_count > 0) {
    const int j0 = V * g.l;
    const float alpha = P.cnt->sc_alpha, mu = S.mu;
    float x[V], gr[V], vel[V], lo[V], hi[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    ld_vec<V>(P.g + (size_t)i * DP + j0, gr);
    ld_vec<V>(P.lo + j0, lo);
    ld_vec<V>(P.hi + j0, hi);
#pragma unroll
    for (int v = 0; v < V; ++v) vel[v] = 0.f;
    for (int t = 0; t < S.n_anti; ++t) {
      if (t > 0) gradient_only<KIND, GM, V, LPS>(P.obj, S, P.d, x, gr, g, ec);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        vel[v] = mu * vel[v] - alpha * gr[v];
        const float nx = x[v] + vel[v];
        const float cx = clampf(nx, lo[v], hi[v]);
        if (cx != nx) vel[v] = 0.f;
        x[v] = cx;
      }
    }
    st_vec<V>(P.x + (size_t)i * DP + j0, x);
    if (g.l == 0) P.hlen[i] = 0;
    else ec.evals = ec.grads = 0;
  }
  block_add_u64<NT_OBJ>(ec.evals, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ec.grads, &P.cnt->grads);
}

template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_anti(ProbDev P, StepParams S) {
  anti_body<KIND, DP, GM>(P, S, blockIdx.x);
}

template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_anti_grp(GroupTab T) {
  const int q = T.blk_prob[blockIdx.x];
  anti_body<KIND, DP, GM>(T.probs[q], T.sps[q], blockIdx.x - (unsigned)T.blk_first[q]);
}

// ------------------------------------------------------------------ plain evaluation
// f and (optionally) grad f at n caller points x[n][d] (unpadded rows).
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_eval(ProbDev P, StepParams S, const float* __restrict__ x,
                                                 int n, float* __restrict__ fout, float* __restrict__ gout) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  if (i >= n) return;
  const int d = P.d, j0 = V * g.l;
  float xv[V];
#pragma unroll
  for (int v = 0; v < V; ++v) xv[v] = (j0 + v < d) ? x[(size_t)i * d + j0 + v] : 0.f;
  EvalCount ec;
  using TE = EvalT<GM>;
  if (gout) {
    float a[V];
    const TE f = value_and_gradient<KIND, GM, V, LPS>(P.obj, S, d, xv, a, g, ec);
#pragma unroll
    for (int v = 0; v < V; ++v)
      if (j0 + v < d) gout[(size_t)i * d + j0 + v] = a[v];
    if (fout && g.l == 0) fout[i] = (float)f;
  } else {
    TE xe[V];
#pragma unroll
    for (int v = 0; v < V; ++v) xe[v] = (TE)xv[v];
    const TE f = value_noisy<KIND, TE, V, LPS>(P.obj, params_of<GM>(P.obj), S, xe, g);
    if (fout && g.l == 0) fout[i] = (float)f;
  }
}

// ------------------------------------------------------------------ launch dispatch
template <int KIND, int DP, int GM>
cudaError_t launch_obj_dp_gm(int which, const ProbDev& P, const StepParams& S, int arg, const EvalArgs* ea,
                             cudaStream_t st) {
  constexpr int LPS = DP / VL;
  const long long rows = (which == OKID_EVAL) ? ea->n : P.n;
  const unsigned blocks = (unsigned)((rows * LPS + NT_OBJ - 1) / NT_OBJ);
  if (rows <= 0) return cudaSuccess;
  switch (which) {
    case OKID_PHASE1:
      if constexpr (DP <= 16 && GM != GRAD_ADJOINT) {
        k_phase1_wide<KIND, DP, GM><<<(unsigned)((rows * P1_W * (DP / VL) + NT_OBJ - 1) / NT_OBJ), NT_OBJ, 0, st>>>(
            P, S, arg < 0 ? -arg : arg, arg >= 0 ? 1 : 0, nullptr, nullptr);
        break;
      }
      k_phase1<KIND, DP, GM><<<blocks, NT_OBJ, 0, st>>>(P, S, arg < 0 ? -arg : arg, arg >= 0 ? 1 : 0, nullptr,
                                                        nullptr);
      break;
    case OKID_REFINE:
      k_phase1<KIND, DP, GM><<<blocks, NT_OBJ, 0, st>>>(P, S, arg, 1, P.l_surv, &P.cnt->n_surv);
      break;
    case OKID_DIRECTION:
      k_direction<DP><<<blocks, NT_OBJ, 0, st>>>(P);
      break;
    case OKID_SCALES:
      if constexpr (DP <= 16 && GM != GRAD_ADJOINT) {
        k_grad_wide<KIND, DP, GM><<<(unsigned)((rows * P1_W * (DP / VL) + NT_OBJ - 1) / NT_OBJ), NT_OBJ, 0, st>>>(
            P, S, arg);
        k_scales<KIND, DP, GM><<<(unsigned)scale_blocks(P), NT_SCALES, 0, st>>>(P, S, 2);
        break;
      }
      k_scales<KIND, DP, GM><<<(unsigned)scale_blocks(P), NT_SCALES, 0, st>>>(P, S, arg);
      break;
    case OKID_HLC:
      if constexpr (DP <= 16 && GM != GRAD_ADJOINT) {
        if (S.M <= HLC_W && !S.hlc_value_only) {
          k_hlc_wide<KIND, DP, GM><<<(unsigned)((rows * HLC_W * (DP / VL) + NT_OBJ - 1) / NT_OBJ), NT_OBJ, 0, st>>>(
              P, S);
          break;
        }
      }
      k_hlc<KIND, DP, GM><<<blocks, NT_OBJ, 0, st>>>(P, S);
      break;
    case OKID_ANTI:
      if constexpr (DP <= 16 && GM != GRAD_ADJOINT) {
        k_anti_wide<KIND, DP, GM><<<(unsigned)((rows * P1_W * (DP / VL) + NT_OBJ - 1) / NT_OBJ), NT_OBJ, 0, st>>>(
            P, S);
        break;
      }
      k_anti<KIND, DP, GM><<<blocks, NT_OBJ, 0, st>>>(P, S);
      break;
    case OKID_EVAL:
      k_eval<KIND, DP, GM><<<blocks, NT_OBJ, 0, st>>>(P, S, ea->x, ea->n, ea->f, ea->g);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int KIND, int DP>
cudaError_t launch_obj_dp(int which, int gm, const ProbDev& P, const StepParams& S, int arg, const EvalArgs* ea,
                          cudaStream_t st) {
  switch (gm) {
    case GRAD_FD64: return launch_obj_dp_gm<KIND, DP, GRAD_FD64>(which, P, S, arg, ea, st);
    case GRAD_FD32: return launch_obj_dp_gm<KIND, DP, GRAD_FD32>(which, P, S, arg, ea, st);
    case GRAD_ADJOINT: return launch_obj_dp_gm<KIND, DP, GRAD_ADJOINT>(which, P, S, arg, ea, st);
  }
  return cudaErrorInvalidValue;
}

template <int KIND>
cudaError_t launch_obj(int which, int gm, const ProbDev& P, const StepParams& S, int arg, const EvalArgs* ea,
                       cudaStream_t st) {
  switch (P.dp) {
    case 4: return launch_obj_dp<KIND, 4>(which, gm, P, S, arg, ea, st);
    case 8: return launch_obj_dp<KIND, 8>(which, gm, P, S, arg, ea, st);
    case 16: return launch_obj_dp<KIND, 16>(which, gm, P, S, arg, ea, st);
    case 32: return launch_obj_dp<KIND, 32>(which, gm, P, S, arg, ea, st);
    case 64: return launch_obj_dp<KIND, 64>(which, gm, P, S, arg, ea, st);
  }
  return cudaErrorInvalidValue;
}

// Grouped launches (exact gradients): one launch runs Phase 1, the scale pass, Phase 5 or
// Phase 6 of every problem of a group that shares the objective kind and padded dimension
// (T maps the launch's blocks to problems: NT_OBJ-thread blocks over the samples, or the
// problems' scale-pass grids for OKID_SCALES).
template <int KIND, int DP>
cudaError_t launch_grp_dp(int which, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0) {
  if (blocks == 0) return cudaSuccess;
  switch (which) {
    case OKID_PHASE1: k_phase1_grp<KIND, DP, GRAD_ADJOINT><<<blocks, NT_OBJ, 0, st>>>(T); break;
    case OKID_HLC: k_hlc_grp<KIND, DP, GRAD_ADJOINT><<<blocks, NT_OBJ, 0, st>>>(T); break;
    case OKID_ANTI: k_anti_grp<KIND, DP, GRAD_ADJOINT><<<blocks, NT_OBJ, 0, st>>>(T); break;
    case OKID_SCALES: k_scales_grp<KIND, DP, GRAD_ADJOINT><<<blocks, NT_SCALES, 0, st>>>(T, arg); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_grp(int which, int dp, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0) {
  switch (dp) {
    case 4: return launch_grp_dp<KIND, 4>(which, T, blocks, st, arg);
    case 8: return launch_grp_dp<KIND, 8>(which, T, blocks, st, arg);
    case 16: return launch_grp_dp<KIND, 16>(which, T, blocks, st, arg);
    case 32: return launch_grp_dp<KIND, 32>(which, T, blocks, st, arg);
    case 64: return launch_grp_dp<KIND, 64>(which, T, blocks, st, arg);
  }
  return cudaErrorInvalidValue;
}

}  // namespace chisao

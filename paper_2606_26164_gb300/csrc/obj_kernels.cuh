// Kernels that evaluate the objective: Phase 1 (batched L-BFGS, Sec. 3.2.1),
// the scale estimates at the start of Phases 5 and 6, Hands Like Clouds
// (Eq. 5), anti-convergence (Eq. 6), the L-BFGS direction alone, and plain
// objective evaluation.  Templated on objective kind, padded dimension DP
// (lane group of DP/2 lanes per sample) and gradient mode.
#pragma once
#include "objectives.cuh"

namespace chisao {

constexpr int NT_OBJ = 128;     // threads per block of the per-sample kernels
constexpr int NT_SCALES = 256;  // threads per block of the scale reduction
constexpr int SCALE_BLOCKS = 608;  // fixed grid of the scale reduction (4 x 152 SMs)

// L-BFGS two-loop recursion (Nocedal & Wright, Algorithm 7.4) on F = -f with
// the register-resident history (slot 0 newest), H0 = gam * I, in binary32
// with group-sum dot products.
template <int LPS>
__device__ __forceinline__ void two_loop(const float (&s0)[MMAX], const float (&s1)[MMAX],
                                         const float (&y0)[MMAX], const float (&y1)[MMAX],
                                         const float (&rho)[MMAX], int len, float gam, float G0,
                                         float G1, float& p0, float& p1, const Grp<LPS>& g) {
  float q0 = G0, q1 = G1;
  float al[MMAX];
#pragma unroll
  for (int k = 0; k < MMAX; ++k) {
    al[k] = 0.f;
    if (k < len) {
      al[k] = rho[k] * g.sum(s0[k] * q0 + s1[k] * q1);
      q0 = fmaf(-al[k], y0[k], q0);
      q1 = fmaf(-al[k], y1[k], q1);
    }
  }
  const float gm = len > 0 ? gam : 1.f;
  float r0 = gm * q0, r1 = gm * q1;
#pragma unroll
  for (int k = MMAX - 1; k >= 0; --k) {
    if (k < len) {
      const float be = rho[k] * g.sum(y0[k] * r0 + y1[k] * r1);
      r0 = fmaf(s0[k], al[k] - be, r0);
      r1 = fmaf(s1[k], al[k] - be, r1);
    }
  }
  p0 = -r0;
  p1 = -r1;
}

// History of sample i into registers; gam = s^T y / y^T y of the newest pair
// (s^T y = 1 / rho).
template <int DP, int LPS>
__device__ __forceinline__ void load_history(const ProbDev& P, int i, int j0, int len, float (&s0)[MMAX],
                                             float (&s1)[MMAX], float (&y0)[MMAX], float (&y1)[MMAX],
                                             float (&rho)[MMAX], float& gam, const Grp<LPS>& g) {
#pragma unroll
  for (int k = 0; k < MMAX; ++k) {
    if (k < len) {
      const size_t o = ((size_t)i * MMAX + k) * DP + j0;
      const float2 sv = *reinterpret_cast<const float2*>(P.hs + o);
      const float2 yv = *reinterpret_cast<const float2*>(P.hy + o);
      s0[k] = sv.x; s1[k] = sv.y; y0[k] = yv.x; y1[k] = yv.y;
      rho[k] = P.hrho[(size_t)i * MMAX + k];
    } else {
      s0[k] = s1[k] = y0[k] = y1[k] = 0.f;
      rho[k] = 0.f;
    }
  }
  gam = 1.f;
  if (len > 0) gam = (1.0f / rho[0]) / g.sum(y0[0] * y0[0] + y1[0] * y1[0]);
}

// ------------------------------------------------------------------ Phase 1
// n_iter iterations of L-BFGS per sample, all in registers:
//   p = -H grad F (two-loop); restart with -grad F when p is not a descent
//   direction; backtracking Armijo over alpha0 2^-t on the box projection
//   x_t = clip(x + alpha p), F(x_t) <= F(x) + c1 grad F^T (x_t - x), first pass
//   wins (alpha0 = 1, or min(1, 1/|grad F|_inf) on an empty history); new
//   gradient; pair (s, y) kept iff s^T y > curv_eps |s||y|, s^T y summed from
//   exact products in double-single.  A failed search clears the history.
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_phase1(ProbDev P, StepParams S, int n_iter, int fresh) {
  constexpr int LPS = DP / 2;
  using TE = EvalT<GM>;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  EvalCount ec;
  unsigned long long trials = 0, fails = 0;
  if (i < P.n) {
    const int j0 = 2 * g.l;
    const float2 xv = *reinterpret_cast<const float2*>(P.x + (size_t)i * DP + j0);
    float x0 = xv.x, x1 = xv.y;
    const float lo0 = P.lo[j0], lo1 = P.lo[j0 + 1], hi0 = P.hi[j0], hi1 = P.hi[j0 + 1];
    int len = P.hlen[i];
    float s0[MMAX], s1[MMAX], y0[MMAX], y1[MMAX], gam;
    float rho[MMAX];
    const float curv_eps = (float)S.curv_eps;
    load_history<DP, LPS>(P, i, j0, len, s0, s1, y0, y1, rho, gam, g);
    TE F;
    float G0, G1;
    if (fresh) {
      float a0, a1;
      const TE f = value_and_gradient<KIND, GM, LPS>(P.obj, S, P.d, x0, x1, a0, a1, g, ec);
      F = -f;
      G0 = -a0;
      G1 = -a1;
    } else {
      F = -(TE)P.f[i];
      const float2 gv = *reinterpret_cast<const float2*>(P.g + (size_t)i * DP + j0);
      G0 = -gv.x;
      G1 = -gv.y;
    }
    for (int it = 0; it < n_iter; ++it) {
      const float gn = g.maxf(fmaxf(fabsf(G0), fabsf(G1)));
      if (!(gn > 0.f)) break;                      // exactly stationary (or invalid): stays put
      float p0, p1;
      two_loop<LPS>(s0, s1, y0, y1, rho, len, gam, G0, G1, p0, p1, g);
      float a0 = len > 0 ? 1.f : fminf(1.f, 1.f / gn);
      const float gp = g.sum(G0 * p0 + G1 * p1);
      if (!(gp < 0.f)) {                           // not a descent direction: restart
        len = 0;
        p0 = -G0;
        p1 = -G1;
        a0 = fminf(1.f, 1.f / gn);
      }
      bool acc = false;
      float xt0 = x0, xt1 = x1, Gt0 = 0.f, Gt1 = 0.f;
      TE Ft = F;
      for (int t = 0; t < S.T_ls; ++t) {
        const float a = ldexpf(a0, -t);
        const float c0 = clampf(fmaf(a, p0, x0), lo0, hi0);
        const float c1 = clampf(fmaf(a, p1, x1), lo1, hi1);
        TE ft;
        float ga0 = 0.f, ga1 = 0.f;
        if constexpr (GM == GRAD_ADJOINT) {
          ft = value_grad_noisy<KIND>(P.obj, S, c0, c1, ga0, ga1, g);
          ec.evals += 1;
          ec.grads += 1;
        } else {
          ft = value_noisy<KIND>(P.obj, params_of<GM>(P.obj), S, (TE)c0, (TE)c1, g);
          ec.evals += 1;
        }
        ++trials;
        const TE dec = g.sum((TE)G0 * ((TE)c0 - (TE)x0) + (TE)G1 * ((TE)c1 - (TE)x1));
        if (-ft <= F + (TE)S.c1 * dec) {
          acc = true;
          xt0 = c0; xt1 = c1; Ft = -ft; Gt0 = -ga0; Gt1 = -ga1;
          break;
        }
      }
      if (!acc) {
        len = 0;
        ++fails;
        continue;
      }
      if constexpr (GM != GRAD_ADJOINT) {
        float a0g, a1g;
        gradient_only<KIND, GM, LPS>(P.obj, S, P.d, xt0, xt1, a0g, a1g, g, ec);
        Gt0 = -a0g;
        Gt1 = -a1g;
      }
      const float sv0 = xt0 - x0, sv1 = xt1 - x1, yv0 = Gt0 - G0, yv1 = Gt1 - G1;
      float syh, syl;                                // s^T y, exact products + compensated sum
      ff_dot2(sv0, yv0, sv1, yv1, syh, syl);
      g.ff_sum(syh, syl);
      const float sy = syh + syl;
      const float ss = g.sum(sv0 * sv0 + sv1 * sv1);  // sums of squares: no cancellation
      const float yy = g.sum(yv0 * yv0 + yv1 * yv1);
      if (sy > curv_eps * sqrtf(ss) * sqrtf(yy)) {
#pragma unroll
        for (int k = MMAX - 1; k > 0; --k) {
          s0[k] = s0[k - 1]; s1[k] = s1[k - 1]; y0[k] = y0[k - 1]; y1[k] = y1[k - 1]; rho[k] = rho[k - 1];
        }
        s0[0] = sv0; s1[0] = sv1; y0[0] = yv0; y1[0] = yv1;
        rho[0] = 1.0f / sy;
        len = min(len + 1, S.m);
        gam = sy / yy;
      }
      x0 = xt0; x1 = xt1; F = Ft; G0 = Gt0; G1 = Gt1;
    }
    *reinterpret_cast<float2*>(P.x + (size_t)i * DP + j0) = make_float2(x0, x1);
    *reinterpret_cast<float2*>(P.g + (size_t)i * DP + j0) = make_float2(-G0, -G1);
#pragma unroll
    for (int k = 0; k < MMAX; ++k) {
      if (k < len) {
        const size_t o = ((size_t)i * MMAX + k) * DP + j0;
        *reinterpret_cast<float2*>(P.hs + o) = make_float2(s0[k], s1[k]);
        *reinterpret_cast<float2*>(P.hy + o) = make_float2(y0[k], y1[k]);
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
  if (i >= P.n) { ec.evals = ec.grads = 0; trials = fails = 0; }
  block_add_u64<NT_OBJ>(ec.evals, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ec.grads, &P.cnt->grads);
  block_add_u64<NT_OBJ>(trials, &P.cnt->ls_trials);
  block_add_u64<NT_OBJ>(fails, &P.cnt->ls_fail);
}

// Direction only (test hook): p = -H grad F written into g.
template <int DP>
__global__ void __launch_bounds__(NT_OBJ) k_direction(ProbDev P) {
  constexpr int LPS = DP / 2;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  if (i >= P.n) return;
  const int j0 = 2 * g.l;
  const int len = P.hlen[i];
  float s0[MMAX], s1[MMAX], y0[MMAX], y1[MMAX], gam;
  float rho[MMAX];
  load_history<DP, LPS>(P, i, j0, len, s0, s1, y0, y1, rho, gam, g);
  const float2 gv = *reinterpret_cast<const float2*>(P.g + (size_t)i * DP + j0);
  float p0, p1;
  two_loop<LPS>(s0, s1, y0, y1, rho, len, gam, -gv.x, -gv.y, p0, p1, g);
  *reinterpret_cast<float2*>(P.g + (size_t)i * DP + j0) = make_float2(p0, p1);
}

// ------------------------------------------------------------------ scales (Phase 5/6 start)
// Gradient at every unfrozen sample (stored in g) and per-block partial sums
// (sum x_j, sum x_j^2 per coordinate, sum |g|^2, count) in FP64, reduced in a
// fixed order so the result is deterministic.
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_SCALES) k_scales(ProbDev P, StepParams S) {
  constexpr int LPS = DP / 2;
  constexpr int GPB = NT_SCALES / LPS;             // groups per block
  constexpr int W = 2 * DP + 2;
  __shared__ double buf[GPB][W];
  const Grp<LPS> g;
  const int grp = threadIdx.x / LPS;
  const int j0 = 2 * g.l;
  EvalCount ec;
  // double-single running sums (exact squares via FMA), converted to FP64 once
  float sx0h = 0.f, sx0l = 0.f, sx1h = 0.f, sx1l = 0.f, sq0h = 0.f, sq0l = 0.f, sq1h = 0.f, sq1l = 0.f;
  float sgh = 0.f, sgl = 0.f;
  int cnt = 0;
  for (int i = blockIdx.x * GPB + grp; i < P.n; i += gridDim.x * GPB) {
    if (bit_of(P.stuck, i)) continue;
    const float2 xv = *reinterpret_cast<const float2*>(P.x + (size_t)i * DP + j0);
    float a0, a1;
    gradient_only<KIND, GM, LPS>(P.obj, S, P.d, xv.x, xv.y, a0, a1, g, ec);
    *reinterpret_cast<float2*>(P.g + (size_t)i * DP + j0) = make_float2(a0, a1);
    ff_add(sx0h, sx0l, xv.x, 0.f);
    ff_add(sx1h, sx1l, xv.y, 0.f);
    const float p0 = xv.x * xv.x, p1 = xv.y * xv.y;
    ff_add(sq0h, sq0l, p0, fmaf(xv.x, xv.x, -p0));
    ff_add(sq1h, sq1l, p1, fmaf(xv.y, xv.y, -p1));
    ff_add(sgh, sgl, g.sum(a0 * a0 + a1 * a1), 0.f);   // sum of squares: no cancellation
    ++cnt;
  }
  buf[grp][j0] = (double)sx0h + (double)sx0l;
  buf[grp][j0 + 1] = (double)sx1h + (double)sx1l;
  buf[grp][DP + j0] = (double)sq0h + (double)sq0l;
  buf[grp][DP + j0 + 1] = (double)sq1h + (double)sq1l;
  if (g.l == 0) {
    buf[grp][2 * DP] = (double)sgh + (double)sgl;
    buf[grp][2 * DP + 1] = (double)cnt;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < W; t += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < GPB; ++q) acc += buf[q][t];
    P.partials[(size_t)blockIdx.x * W + t] = acc;
  }
  if (g.l != 0) ec.evals = ec.grads = 0;
  block_add_u64<NT_SCALES>(ec.evals, &P.cnt->evals);
  block_add_u64<NT_SCALES>(ec.grads, &P.cnt->grads);
}

// ------------------------------------------------------------------ Phase 5
// n_cloud steps x <- clip(x + alpha (1/M) sum_k grad f(x + sigma z_k)) on the
// unfrozen samples; z_k from the HLC Philox stream (row = sample, step = cloud
// step, k = perturbation).  History is cleared (the sample moved).
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_hlc(ProbDev P, StepParams S) {
  constexpr int LPS = DP / 2;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  EvalCount ec;
  if (i < P.n && !bit_of(P.stuck, i) && P.cnt->sc_count > 0) {
    const int j0 = 2 * g.l;
    const unsigned cyc = (unsigned)P.cnt->cycle + 1u;
    const float sigma = P.cnt->sc_sigma, alpha = P.cnt->sc_alpha;
    const float2 xv = *reinterpret_cast<const float2*>(P.x + (size_t)i * DP + j0);
    float x0 = xv.x, x1 = xv.y;
    const float lo0 = P.lo[j0], lo1 = P.lo[j0 + 1], hi0 = P.hi[j0], hi1 = P.hi[j0 + 1];
    const bool v0 = j0 < P.d, v1 = j0 + 1 < P.d;
    const float invM = 1.0f / (float)S.M;
    for (int t = 0; t < S.n_cloud; ++t) {
      float acc0 = 0.f, acc1 = 0.f;
      for (int k = 0; k < S.M; ++k) {
        const float2 z = normals_pair(S, (unsigned)i, g.l, TAG_HLC, cyc, (unsigned)t, (unsigned)P.prob_index,
                                      (unsigned)k);
        const float xp0 = v0 ? fmaf(sigma, z.x, x0) : x0;
        const float xp1 = v1 ? fmaf(sigma, z.y, x1) : x1;
        float a0, a1;
        gradient_only<KIND, GM, LPS>(P.obj, S, P.d, xp0, xp1, a0, a1, g, ec);
        acc0 += a0;
        acc1 += a1;
      }
      x0 = clampf(fmaf(alpha, acc0 * invM, x0), lo0, hi0);
      x1 = clampf(fmaf(alpha, acc1 * invM, x1), lo1, hi1);
    }
    *reinterpret_cast<float2*>(P.x + (size_t)i * DP + j0) = make_float2(x0, x1);
    if (g.l == 0) P.hlen[i] = 0;
    else ec.evals = ec.grads = 0;
  }
  block_add_u64<NT_OBJ>(ec.evals, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ec.grads, &P.cnt->grads);
}

// ------------------------------------------------------------------ Phase 6
// n_anti momentum steps v <- mu v - alpha grad f(x), x <- clip(x + v), v = 0
// on coordinates the projection moved; v_0 = 0; the first gradient is the one
// the scale pass stored.  History is cleared.
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_anti(ProbDev P, StepParams S) {
  constexpr int LPS = DP / 2;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  EvalCount ec;
  if (i < P.n && !bit_of(P.stuck, i) && P.cnt->sc_count > 0) {
    const int j0 = 2 * g.l;
    const float alpha = P.cnt->sc_alpha, mu = S.mu;
    const float2 xv = *reinterpret_cast<const float2*>(P.x + (size_t)i * DP + j0);
    const float2 gv = *reinterpret_cast<const float2*>(P.g + (size_t)i * DP + j0);
    float x0 = xv.x, x1 = xv.y, g0 = gv.x, g1 = gv.y, v0 = 0.f, v1 = 0.f;
    const float lo0 = P.lo[j0], lo1 = P.lo[j0 + 1], hi0 = P.hi[j0], hi1 = P.hi[j0 + 1];
    for (int t = 0; t < S.n_anti; ++t) {
      if (t > 0) gradient_only<KIND, GM, LPS>(P.obj, S, P.d, x0, x1, g0, g1, g, ec);
      v0 = mu * v0 - alpha * g0;
      v1 = mu * v1 - alpha * g1;
      const float n0 = x0 + v0, n1 = x1 + v1;
      const float c0 = clampf(n0, lo0, hi0), c1 = clampf(n1, lo1, hi1);
      if (c0 != n0) v0 = 0.f;
      if (c1 != n1) v1 = 0.f;
      x0 = c0;
      x1 = c1;
    }
    *reinterpret_cast<float2*>(P.x + (size_t)i * DP + j0) = make_float2(x0, x1);
    if (g.l == 0) P.hlen[i] = 0;
    else ec.evals = ec.grads = 0;
  }
  block_add_u64<NT_OBJ>(ec.evals, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ec.grads, &P.cnt->grads);
}

// ------------------------------------------------------------------ plain evaluation
// f and (optionally) grad f at n caller points x[n][d] (unpadded rows).
template <int KIND, int DP, int GM>
__global__ void __launch_bounds__(NT_OBJ) k_eval(ProbDev P, StepParams S, const float* __restrict__ x,
                                                 int n, float* __restrict__ fout, float* __restrict__ gout) {
  constexpr int LPS = DP / 2;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  if (i >= n) return;
  const int d = P.d, j0 = 2 * g.l;
  const float x0 = j0 < d ? x[(size_t)i * d + j0] : 0.f;
  const float x1 = j0 + 1 < d ? x[(size_t)i * d + j0 + 1] : 0.f;
  EvalCount ec;
  using TE = EvalT<GM>;
  if (gout) {
    float a0, a1;
    const TE f = value_and_gradient<KIND, GM, LPS>(P.obj, S, d, x0, x1, a0, a1, g, ec);
    if (j0 < d) gout[(size_t)i * d + j0] = a0;
    if (j0 + 1 < d) gout[(size_t)i * d + j0 + 1] = a1;
    if (fout && g.l == 0) fout[i] = (float)f;
  } else {
    const TE f = value_noisy<KIND>(P.obj, params_of<GM>(P.obj), S, (TE)x0, (TE)x1, g);
    if (fout && g.l == 0) fout[i] = (float)f;
  }
}

// ------------------------------------------------------------------ launch dispatch
template <int KIND, int DP, int GM>
cudaError_t launch_obj_dp_gm(int which, const ProbDev& P, const StepParams& S, int arg, const EvalArgs* ea,
                             cudaStream_t st) {
  constexpr int LPS = DP / 2;
  const long long rows = (which == OKID_EVAL) ? ea->n : P.n;
  const unsigned blocks = (unsigned)((rows * LPS + NT_OBJ - 1) / NT_OBJ);
  if (rows <= 0) return cudaSuccess;
  switch (which) {
    case OKID_PHASE1:
      k_phase1<KIND, DP, GM><<<blocks, NT_OBJ, 0, st>>>(P, S, arg < 0 ? -arg : arg, arg >= 0 ? 1 : 0);
      break;
    case OKID_DIRECTION:
      k_direction<DP><<<blocks, NT_OBJ, 0, st>>>(P);
      break;
    case OKID_SCALES: {
      constexpr int GPB = NT_SCALES / LPS;
      long long nb = (P.n + GPB - 1) / GPB;
      if (nb > SCALE_BLOCKS) nb = SCALE_BLOCKS;
      if (nb > P.max_part_blocks) nb = P.max_part_blocks;
      k_scales<KIND, DP, GM><<<(unsigned)nb, NT_SCALES, 0, st>>>(P, S);
      break;
    }
    case OKID_HLC:
      k_hlc<KIND, DP, GM><<<blocks, NT_OBJ, 0, st>>>(P, S);
      break;
    case OKID_ANTI:
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

}  // namespace chisao

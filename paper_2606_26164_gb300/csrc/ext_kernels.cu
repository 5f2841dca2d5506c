// Phases 1, 5 and 6 around a *batched* objective evaluator (the tensor-core
// mixture objective): the objective cannot run inside a per-sample kernel (a
// CTA-wide GEMM needs 128 points in lockstep), so each phase is split into
// per-sample kernels that write the points to evaluate and consume the values
// and gradients the evaluator returns.
//
// Phase 1 per L-BFGS iteration (same rules as the fused k_phase1):
//   k_ext_dir     two-loop direction from the history in HBM, descent check,
//                 first trial point x + alpha0 p (box-projected), pending list;
//   round 0:      evaluator on the pending trial points -> k_ext_accept: Armijo
//                 test; accepted samples take the point, value and gradient and
//                 push (s, y, rho) into the history; each of the others gets its
//                 next LS_BATCH trial points alpha0 2^-t, t = 1 .. LS_BATCH;
//   rounds r >= 1: evaluator on all those points at once -> k_ext_accept_multi:
//                 the first passing trial (the largest alpha) is accepted, which is
//                 the step sequential backtracking takes; a sample with none gets
//                 the next LS_BATCH trial points, until T_ls trials are spent.
//   Lists are filled with atomics; every result is per sample, so the order of
//   a list changes nothing.  During Phase 1 the history of each sample is a ring
//   of m slots with a head index, so a push writes one pair in place; after the
//   last iteration k_ext_hist_rotate moves the newest pair back to slot 0.
// Phase 5: k_ext_hlc_points writes x + sigma z_k for all M perturbations, the
//   evaluator returns their gradients, k_ext_hlc_step averages and steps.
// Phase 6: k_ext_anti_step applies the momentum step to the gradient the
//   evaluator returned for the current points.
#include "host.h"
#include "obj_kernels.cuh"

namespace chisao {

// The history of sample i in logical order (slot 0 newest) from its ring.
template <int DP, int V, int LPS>
__device__ __forceinline__ void load_history_ring(const ProbDev& P, int i, int j0, int len, int head, int m,
                                                  float (&s)[MMAX][V], float (&y)[MMAX][V], float (&rho)[MMAX],
                                                  float& gam, const Grp<LPS>& g) {
#pragma unroll
  for (int k = 0; k < MMAX; ++k) {
    if (k < len) {
      const int ph = head + k < m ? head + k : head + k - m;
      const size_t o = ((size_t)i * MMAX + ph) * DP + j0;
      ld_vec<V>(P.hs + o, s[k]);
      ld_vec<V>(P.hy + o, y[k]);
      rho[k] = P.hrho[(size_t)i * MMAX + ph];
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) s[k][v] = y[k][v] = 0.f;
      rho[k] = 0.f;
    }
  }
  gam = 1.f;
  if (len > 0) gam = (1.0f / rho[0]) / g.sum(dotv<V>(y[0], y[0]));
}

template <int DP>
__global__ void __launch_bounds__(NT_OBJ, 4) k_ext_dir(ProbDev P, StepParams S, ExtBuf E, int count_start) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  unsigned long long ev = 0;
  if (i < P.n) {
    const int j0 = V * g.l;
    float G[V], x[V], lo[V], hi[V];
    // the sample's loads that do not depend on another are issued first (one memory
    // round trip for these, one more for the history rows they locate)
    ld_vec<V>(P.g + (size_t)i * DP + j0, G);
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    int len = P.hlen[i];
    const int head = E.head[i];
#pragma unroll
    for (int v = 0; v < V; ++v) G[v] = -G[v];
    float gl = 0.f;
#pragma unroll
    for (int v = 0; v < V; ++v) gl = fmaxf(gl, fabsf(G[v]));
    const float gn = g.maxf(gl);
    if (gn > 0.f) {
      float s[MMAX][V], y[MMAX][V], rho[MMAX], gam, p[V];
      load_history_ring<DP, V, LPS>(P, i, j0, len, head, S.m, s, y, rho, gam, g);
      two_loop<V, LPS>(s, y, rho, len, gam, G, p, g);
      float a0 = len > 0 ? 1.f : fminf(1.f, 1.f / gn);
      if (!(g.sum(dotv<V>(G, p)) <= 0.f)) {          // ascent or not finite: restart
        len = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) p[v] = -G[v];
        a0 = fminf(1.f, 1.f / gn);
        if (g.l == 0) P.hlen[i] = 0;
      }
      ld_vec<V>(P.lo + j0, lo);                      // the box: cache-resident, shared by all samples
      ld_vec<V>(P.hi + j0, hi);
      float c[V];
#pragma unroll
      for (int v = 0; v < V; ++v) c[v] = clampf(fmaf(a0, p[v], x[v]), lo[v], hi[v]);
      st_vec<V>(E.p + (size_t)i * DP + j0, p);
      st_vec<V>(E.xt + (size_t)i * DP + j0, c);
      if (g.l == 0) {
        E.a0[i] = a0;
        E.list0[atomicAdd(&E.cnt[0], 1)] = i;
      }
    }
    if (g.l == 0 && count_start) ev = 1;
  }
  block_add_u64<NT_OBJ>(ev, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ev, &P.cnt->grads);
}

// An accepted trial point c (value -Ft, gradient -Gt of F) of sample i: the pair
// (s, y) = (c - x, Gt - G) is pushed when curved (s^T y summed from exact products in
// double-single, rho = 1 / s^T y finite) into the slot before the ring's head, which
// becomes the head (the oldest pair is overwritten once m are stored); then x, grad f
// and f take the trial's values.
template <int V, int LPS>
__device__ __forceinline__ void ext_take_step(const ProbDev& P, const StepParams& S, const ExtBuf& E, int i,
                                              int j0, int DP, const float (&x)[V], const float (&G)[V],
                                              const float (&c)[V], const float (&Gt)[V], float Ft,
                                              const Grp<LPS>& g) {
  const int head = E.head[i];                          // read by every lane before lane 0 moves it
  const int len = P.hlen[i];
  float sv[V], yv[V], syh = 0.f, syl = 0.f, ss = 0.f, yy = 0.f;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    sv[v] = c[v] - x[v];
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
  if (sy > (float)S.curv_eps * sqrtf(ss) * sqrtf(yy) && 1.0f / sy <= FLT_MAX) {
    const int nh = head > 0 ? head - 1 : S.m - 1;
    const size_t o0 = ((size_t)i * MMAX + nh) * DP + j0;
    st_vec<V>(P.hs + o0, sv);
    st_vec<V>(P.hy + o0, yv);
    __syncwarp(g.mask);                                // the group's head reads are done
    if (g.l == 0) {
      P.hrho[(size_t)i * MMAX + nh] = 1.0f / sy;
      P.hlen[i] = min(len + 1, S.m);
      E.head[i] = nh;
    }
  }
  float gout[V];
#pragma unroll
  for (int v = 0; v < V; ++v) gout[v] = -Gt[v];
  st_vec<V>(P.x + (size_t)i * DP + j0, c);
  st_vec<V>(P.g + (size_t)i * DP + j0, gout);
  if (g.l == 0) P.f[i] = -Ft;
}

// Sample i failed every trial so far, the last being t0 - 1: it goes on the list of
// round r with its trials t0 .. t0 + LS_BATCH - 1 (rows LS_BATCH slot + q of the
// round's buffer; a trial past T_ls is written as x and never looked at), or, with no
// trial left, its search fails (history cleared, x unchanged).  Returns 1 on failure.
template <int V, int LPS>
__device__ __forceinline__ int ext_hand_on(const ProbDev& P, const StepParams& S, const ExtBuf& E, int i, int j0,
                                           int DP, int r, int t0, const float (&x)[V], const Grp<LPS>& g) {
  if (t0 >= S.T_ls) {
    if (g.l == 0) P.hlen[i] = 0;
    return 1;
  }
  const int R = ls_rounds(S.T_ls);
  int slot = 0;
  if (g.l == 0) {
    slot = atomicAdd(&E.cnt[r], 1);
    atomicAdd(&E.cnt[R + 1 + r], LS_BATCH);
    E.mlist[(r - 1) & 1][slot] = i;
  }
  slot = __shfl_sync(g.mask, slot, 0, LPS);
  float p[V], lo[V], hi[V];
  ld_vec<V>(E.p + (size_t)i * DP + j0, p);
  ld_vec<V>(P.lo + j0, lo);
  ld_vec<V>(P.hi + j0, hi);
  const float a0 = E.a0[i];
  const size_t base = (size_t)((r - 1) & 1) * LS_BATCH * P.n + (size_t)LS_BATCH * slot;
#pragma unroll
  for (int q = 0; q < LS_BATCH; ++q) {
    const float a = t0 + q < S.T_ls ? ldexpf(a0, -(t0 + q)) : 0.f;
    float c[V];
#pragma unroll
    for (int v = 0; v < V; ++v) c[v] = clampf(fmaf(a, p[v], x[v]), lo[v], hi[v]);
    st_vec<V>(E.xp + (base + q) * DP + j0, c);
  }
  return 0;
}

// Round 0: the first trial point of every sample the direction kernel listed.
template <int DP>
__global__ void __launch_bounds__(NT_OBJ) k_ext_accept(ProbDev P, StepParams S, ExtBuf E) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int pending = E.cnt[0];
  // a grid of at most 16 blocks per SM strides over the list
  if ((int)(((size_t)blockIdx.x * blockDim.x) / LPS) >= pending) return;
  const int stride = (int)(((size_t)gridDim.x * blockDim.x) / LPS);
  unsigned long long tr = 0, fl = 0;
  for (int jj = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS); jj < pending; jj += stride) {
    const int i = E.list0[jj];
    const int j0 = V * g.l;
    float x[V], G[V], c[V], Gt[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    ld_vec<V>(P.g + (size_t)i * DP + j0, G);
    ld_vec<V>(E.xt + (size_t)i * DP + j0, c);
    ld_vec<V>(E.gt + (size_t)i * DP + j0, Gt);
    float dl = 0.f;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      G[v] = -G[v];
      Gt[v] = -Gt[v];
      dl += G[v] * (c[v] - x[v]);
    }
    const float F = -P.f[i], Ft = -E.ft[i];
    const float dec = g.sum(dl);
    if (g.l == 0) tr += 1;
    if (Ft <= F + (float)S.c1 * dec) {
      ext_take_step<V, LPS>(P, S, E, i, j0, DP, x, G, c, Gt, Ft, g);
    } else {
      const int f = ext_hand_on<V, LPS>(P, S, E, i, j0, DP, 1, 1, x, g);
      if (g.l == 0) fl += (unsigned long long)f;
    }
  }
  block_add_u64<NT_OBJ>(tr, &P.cnt->ls_trials);
  block_add_u64<NT_OBJ>(tr, &P.cnt->evals);
  block_add_u64<NT_OBJ>(tr, &P.cnt->grads);
  block_add_u64<NT_OBJ>(fl, &P.cnt->ls_fail);
}

// Round r >= 1: the trials t = 1 + (r - 1) LS_BATCH + q of every listed sample, all
// evaluated; the first that passes Armijo is taken.
template <int DP>
__global__ void __launch_bounds__(NT_OBJ) k_ext_accept_multi(ProbDev P, StepParams S, ExtBuf E, int r) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int pending = E.cnt[r];
  if ((int)(((size_t)blockIdx.x * blockDim.x) / LPS) >= pending) return;
  const int stride = (int)(((size_t)gridDim.x * blockDim.x) / LPS);
  const int t0 = 1 + (r - 1) * LS_BATCH;
  unsigned long long tr = 0, ev = 0, fl = 0;
  for (int jj = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS); jj < pending; jj += stride) {
    const int i = E.mlist[(r - 1) & 1][jj];
    const int j0 = V * g.l;
    const size_t base = (size_t)((r - 1) & 1) * LS_BATCH * P.n + (size_t)LS_BATCH * jj;
    float x[V], G[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    ld_vec<V>(P.g + (size_t)i * DP + j0, G);
#pragma unroll
    for (int v = 0; v < V; ++v) G[v] = -G[v];
    const float F = -P.f[i];
    if (g.l == 0) {
      ev += LS_BATCH;
      tr += (unsigned long long)min(LS_BATCH, S.T_ls - t0);
    }
    bool done = false;
    for (int q = 0; q < LS_BATCH && t0 + q < S.T_ls; ++q) {
      float c[V], Gt[V];
      ld_vec<V>(E.xp + (base + q) * DP + j0, c);
      ld_vec<V>(E.gp + (base + q) * DP + j0, Gt);
      float dl = 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        Gt[v] = -Gt[v];
        dl += G[v] * (c[v] - x[v]);
      }
      const float Ft = -E.fm[base + q];
      const float dec = g.sum(dl);
      if (Ft <= F + (float)S.c1 * dec) {
        ext_take_step<V, LPS>(P, S, E, i, j0, DP, x, G, c, Gt, Ft, g);
        done = true;
        break;
      }
    }
    if (!done) {
      const int f = ext_hand_on<V, LPS>(P, S, E, i, j0, DP, r + 1, t0 + LS_BATCH, x, g);
      if (g.l == 0) fl += (unsigned long long)f;
    }
  }
  block_add_u64<NT_OBJ>(tr, &P.cnt->ls_trials);
  block_add_u64<NT_OBJ>(ev, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ev, &P.cnt->grads);
  block_add_u64<NT_OBJ>(fl, &P.cnt->ls_fail);
}

// After Phase 1: each sample's ring is rotated so its newest pair is in slot 0 again
// (all len pairs read into registers, then written back), and the head returns to 0.
template <int DP>
__global__ void __launch_bounds__(NT_OBJ) k_ext_hist_rotate(ProbDev P, StepParams S, ExtBuf E) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  if (i >= P.n) return;
  const int head = E.head[i], len = P.hlen[i];
  if (head == 0) return;
  const int j0 = V * g.l;
  if (len > 0) {
    float s[MMAX][V], y[MMAX][V], rho[MMAX];
#pragma unroll
    for (int k = 0; k < MMAX; ++k) {
      if (k < len) {
        const int ph = head + k < S.m ? head + k : head + k - S.m;
        const size_t o = ((size_t)i * MMAX + ph) * DP + j0;
        ld_vec<V>(P.hs + o, s[k]);
        ld_vec<V>(P.hy + o, y[k]);
        rho[k] = P.hrho[(size_t)i * MMAX + ph];
      }
    }
    __syncwarp(g.mask);                                // every lane has read before any writes
#pragma unroll
    for (int k = 0; k < MMAX; ++k) {
      if (k < len) {
        const size_t o = ((size_t)i * MMAX + k) * DP + j0;
        st_vec<V>(P.hs + o, s[k]);
        st_vec<V>(P.hy + o, y[k]);
        if (g.l == 0) P.hrho[(size_t)i * MMAX + k] = rho[k];
      }
    }
  }
  __syncwarp(g.mask);
  if (g.l == 0) E.head[i] = 0;
}

__global__ void k_ext_iota(int* __restrict__ a, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) a[t] = (int)t;
}

// x + sigma z_k for k < M (row k n + i of xp); frozen samples write x itself.
template <int DP>
__global__ void __launch_bounds__(NT_OBJ) k_ext_hlc_points(ProbDev P, StepParams S, ExtBuf E, int t) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  if (i >= P.n) return;
  const int j0 = V * g.l;
  float x[V];
  ld_vec<V>(P.x + (size_t)i * DP + j0, x);
  const bool moving = !bit_of(P.stuck, i) && P.cnt->sc_count > 0;
  const unsigned cyc = (unsigned)P.cnt->cycle + 1u;
  const float sigma = P.cnt->sc_sigma;
  for (int k = 0; k < S.M; ++k) {
    float xp[V];
    if (moving) {
      float z[V];
      normals_lane<V>(S, (unsigned)i, g.l, TAG_HLC, cyc, (unsigned)t, (unsigned)P.obj.prob_index, (unsigned)k, z);
#pragma unroll
      for (int v = 0; v < V; ++v) xp[v] = (j0 + v < P.d) ? fmaf(sigma, z[v], x[v]) : x[v];
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) xp[v] = x[v];
    }
    st_vec<V>(E.xp + ((size_t)k * P.n + i) * DP + j0, xp);
  }
}

template <int DP>
__global__ void __launch_bounds__(NT_OBJ) k_ext_hlc_step(ProbDev P, StepParams S, ExtBuf E) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  unsigned long long ev = 0;
  if (i < P.n && !bit_of(P.stuck, i) && P.cnt->sc_count > 0) {
    const int j0 = V * g.l;
    const float alpha = P.cnt->sc_alpha, invM = 1.0f / (float)S.M;
    float x[V], lo[V], hi[V], acc[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    ld_vec<V>(P.lo + j0, lo);
    ld_vec<V>(P.hi + j0, hi);
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    for (int k = 0; k < S.M; ++k) {
      float a[V];
      ld_vec<V>(E.gp + ((size_t)k * P.n + i) * DP + j0, a);
#pragma unroll
      for (int v = 0; v < V; ++v) acc[v] += a[v];
    }
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = clampf(fmaf(alpha, acc[v] * invM, x[v]), lo[v], hi[v]);
    st_vec<V>(P.x + (size_t)i * DP + j0, x);
    if (g.l == 0) {
      P.hlen[i] = 0;
      ev = (unsigned long long)S.M;
    }
  }
  block_add_u64<NT_OBJ>(ev, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ev, &P.cnt->grads);
}

template <int DP>
__global__ void __launch_bounds__(NT_OBJ) k_ext_anti_step(ProbDev P, StepParams S, ExtBuf E, int t) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int i = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  unsigned long long ev = 0;
  if (i < P.n && !bit_of(P.stuck, i) && P.cnt->sc_count > 0) {
    const int j0 = V * g.l;
    const float alpha = P.cnt->sc_alpha, mu = S.mu;
    float x[V], gr[V], vel[V], lo[V], hi[V];
    ld_vec<V>(P.x + (size_t)i * DP + j0, x);
    ld_vec<V>(P.g + (size_t)i * DP + j0, gr);
    ld_vec<V>(P.lo + j0, lo);
    ld_vec<V>(P.hi + j0, hi);
    if (t == 0) {
#pragma unroll
      for (int v = 0; v < V; ++v) vel[v] = 0.f;
    } else {
      ld_vec<V>(E.vel + (size_t)i * DP + j0, vel);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      vel[v] = mu * vel[v] - alpha * gr[v];
      const float nx = x[v] + vel[v];
      const float cx = clampf(nx, lo[v], hi[v]);
      if (cx != nx) vel[v] = 0.f;
      x[v] = cx;
    }
    st_vec<V>(P.x + (size_t)i * DP + j0, x);
    st_vec<V>(E.vel + (size_t)i * DP + j0, vel);
    if (g.l == 0) {
      P.hlen[i] = 0;
      ev = t > 0 ? 1ull : 0ull;
    }
  }
  block_add_u64<NT_OBJ>(ev, &P.cnt->evals);
  block_add_u64<NT_OBJ>(ev, &P.cnt->grads);
}

// ------------------------------------------------------------------ Laplace widths
// Sec. 3.2.3 keeps a surviving sample's inverse-Hessian estimate for width
// estimation.  The estimate is the matrix H the two-loop recursion applies; its
// column j is H e_j (the recursion on the unit vector e_j), and the Laplace
// approximation at the mode gives the width sqrt(H_jj) along coordinate j.  One
// lane group per survivor, d recursions from the history in registers.
template <int DP>
__global__ void __launch_bounds__(NT_OBJ) k_widths(ProbDev P, int rows, float* __restrict__ w,
                                                   float* __restrict__ cov) {
  constexpr int V = VL, LPS = DP / V;
  const Grp<LPS> g;
  const int r = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) / LPS);
  if (r >= rows || r >= P.cnt->n_surv) return;
  const int i = P.l_surv[r];
  const int j0 = V * g.l, d = P.d;
  const int len = P.hlen[i];
  float s[MMAX][V], y[MMAX][V], rho[MMAX], gam;
  load_history<DP, V, LPS>(P, i, j0, len, s, y, rho, gam, g);
  for (int j = 0; j < d; ++j) {
    float e[V], p[V];
#pragma unroll
    for (int v = 0; v < V; ++v) e[v] = (j0 + v == j) ? 1.f : 0.f;
    two_loop<V, LPS>(s, y, rho, len, gam, e, p, g);          // p = -H e_j
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if (cov && j0 + v < d) cov[((size_t)r * d + j) * d + j0 + v] = -p[v];
      if (j0 + v == j) w[(size_t)r * d + j] = sqrtf(fmaxf(-p[v], 0.f));
    }
  }
}

template <int DP>
static cudaError_t widths_dp(const ProbDev& P, int rows, float* w, float* cov, cudaStream_t st) {
  constexpr int LPS = DP / VL;
  const unsigned blocks = (unsigned)(((long long)rows * LPS + NT_OBJ - 1) / NT_OBJ);
  k_widths<DP><<<blocks, NT_OBJ, 0, st>>>(P, rows, w, cov);
  return cudaGetLastError();
}

// A caller's evaluator writes the d coordinates of each gradient row; the padding
// coordinates d .. dp-1, which the per-sample kernels read as part of their float4
// rows, are set to zero after it.
__global__ void k_zero_padding(float* __restrict__ g, long long rows, int d, int dp) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int w = dp - d;
  if (t >= rows * w) return;
  g[(t / w) * dp + d + t % w] = 0.f;
}

cudaError_t launch_zero_padding(float* g, long long rows, int d, int dp, cudaStream_t st) {
  if (!g || rows <= 0 || d >= dp) return cudaSuccess;
  const long long total = rows * (dp - d);
  k_zero_padding<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g, rows, d, dp);
  return cudaGetLastError();
}

unsigned obj_blocks(long long n, int dp) {
  return (unsigned)((n * (dp / VL) + NT_OBJ - 1) / NT_OBJ);
}

cudaError_t launch_widths(const ProbDev& P, int rows, float* w, float* cov, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  switch (P.dp) {
    case 4: return widths_dp<4>(P, rows, w, cov, st);
    case 8: return widths_dp<8>(P, rows, w, cov, st);
    case 16: return widths_dp<16>(P, rows, w, cov, st);
    case 32: return widths_dp<32>(P, rows, w, cov, st);
    case 64: return widths_dp<64>(P, rows, w, cov, st);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ launchers
template <int DP>
static cudaError_t ext_launch_dp(int which, const ProbDev& P, const StepParams& S, const ExtBuf& E, int arg,
                                 cudaStream_t st) {
  constexpr int LPS = DP / VL;
  const unsigned blocks = (unsigned)(((long long)P.n * LPS + NT_OBJ - 1) / NT_OBJ);
  switch (which) {
    case EXT_DIR: k_ext_dir<DP><<<blocks, NT_OBJ, 0, st>>>(P, S, E, arg); break;
    case EXT_ACCEPT:
    case EXT_ACCEPT_MULTI: {
      static int sms = 0;                              // SM count of the device (queried once)
      if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
          sms = 152;
      }
      const unsigned cap = (unsigned)(16 * sms);
      if (which == EXT_ACCEPT)
        k_ext_accept<DP><<<blocks < cap ? blocks : cap, NT_OBJ, 0, st>>>(P, S, E);
      else
        k_ext_accept_multi<DP><<<blocks < cap ? blocks : cap, NT_OBJ, 0, st>>>(P, S, E, arg);
      break;
    }
    case EXT_HIST_ROTATE: k_ext_hist_rotate<DP><<<blocks, NT_OBJ, 0, st>>>(P, S, E); break;
    case EXT_IOTA: {
      const long long rows = 2ll * LS_BATCH * P.n;
      k_ext_iota<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(E.iota, rows);
      break;
    }
    case EXT_HLC_POINTS: k_ext_hlc_points<DP><<<blocks, NT_OBJ, 0, st>>>(P, S, E, arg); break;
    case EXT_HLC_STEP: k_ext_hlc_step<DP><<<blocks, NT_OBJ, 0, st>>>(P, S, E); break;
    case EXT_ANTI_STEP: k_ext_anti_step<DP><<<blocks, NT_OBJ, 0, st>>>(P, S, E, arg); break;
    case EXT_SCALES:
      k_scales<OBJ_MIXTURE_FULL, DP, GRAD_GIVEN><<<(unsigned)scale_blocks(P), NT_SCALES, 0, st>>>(P, S, 0);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_ext(int which, const ProbDev& P, const StepParams& S, const ExtBuf& E, int arg,
                       cudaStream_t st) {
  switch (P.dp) {
    case 4: return ext_launch_dp<4>(which, P, S, E, arg, st);
    case 8: return ext_launch_dp<8>(which, P, S, E, arg, st);
    case 16: return ext_launch_dp<16>(which, P, S, E, arg, st);
    case 32: return ext_launch_dp<32>(which, P, S, E, arg, st);
    case 64: return ext_launch_dp<64>(which, P, S, E, arg, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace chisao

// Built-in objectives evaluated by one lane group per sample, and the
// gradient modes of Section 3.1 (finite differences or analytic).
//
//  * Gaussian mixture log-density (Appendix D, with per-component weights and
//    diagonal or full covariances): f = log sum_k exp(lc_k),
//      lc_k = c_k - |z_k|^2 / 2,  z_k = L_k^-1 (x - mu_k)   (diag: (x-mu)/sigma),
//    accumulated as an online log-sum-exp so the K components stream once.
//    Adjoint: grad f = sum_k r_k s_k with r = softmax(lc) and
//      s_k = -L_k^-T z_k (diag: -(x - mu_k)/sigma_k^2), folded into the same
//    online pass by rescaling the running sum whenever the running max moves.
//  * Rotated quadratic f = -(x - c)^T A (x - c), A = Q^T diag(lam) Q:
//    u = A (x - c), f = -(x - c)^T u, grad f = -2 u (one matrix-vector product
//    gives both).
//
// The group's lanes each hold two coordinates; products with a d x d matrix
// broadcast the other lanes' coordinates with register shuffles and read the
// matrix as float2/double2 rows that are contiguous across the group.
#pragma once
#include <type_traits>

#include "dev_common.cuh"

namespace chisao {

template <typename T>
__device__ __forceinline__ void lse_push(T& m, T& s, T lc) {
  if (lc > m) {
    s = s * exp(m - lc) + T(1);
    m = lc;
  } else {
    s += exp(lc - m);
  }
}

template <typename T>
__device__ __forceinline__ void lse_push_grad(T& m, T& s, T& G0, T& G1, T lc, T sc0, T sc1) {
  if (lc > m) {
    const T e = exp(m - lc);
    s = s * e + T(1);
    G0 = G0 * e + sc0;
    G1 = G1 * e + sc1;
    m = lc;
  } else {
    const T e = exp(lc - m);
    s += e;
    G0 = fma(e, sc0, G0);
    G1 = fma(e, sc1, G1);
  }
}

template <int KIND>
struct Obj;

// ------------------------------------------------------------ diagonal mixture
template <>
struct Obj<OBJ_MIXTURE_DIAG> {
  template <typename T, int LPS>
  static __device__ __forceinline__ T value(const ObjParams<T>& o, T x0, T x1, const Grp<LPS>& g) {
    T m = -CUDART_INF, s = T(0);
    const T* mu = o.p0 + 2 * g.l;
    const T* a = o.p1 + 2 * g.l;
    for (int k = 0; k < o.K; ++k) {
      const auto mk = ldg2(mu + (size_t)k * o.dp);
      const auto ak = ldg2(a + (size_t)k * o.dp);
      const T r0 = x0 - mk.x, r1 = x1 - mk.y;
      const T q = g.sum(ak.x * r0 * r0 + ak.y * r1 * r1);
      lse_push(m, s, __ldg(o.p2 + k) - T(0.5) * q);
    }
    return m + log(s);
  }
  template <typename T, int LPS>
  static __device__ __forceinline__ T value_grad(const ObjParams<T>& o, T x0, T x1, T& g0, T& g1,
                                                 const Grp<LPS>& g) {
    T m = -CUDART_INF, s = T(0), G0 = T(0), G1 = T(0);
    const T* mu = o.p0 + 2 * g.l;
    const T* a = o.p1 + 2 * g.l;
    for (int k = 0; k < o.K; ++k) {
      const auto mk = ldg2(mu + (size_t)k * o.dp);
      const auto ak = ldg2(a + (size_t)k * o.dp);
      const T r0 = x0 - mk.x, r1 = x1 - mk.y;
      const T q = g.sum(ak.x * r0 * r0 + ak.y * r1 * r1);
      lse_push_grad(m, s, G0, G1, __ldg(o.p2 + k) - T(0.5) * q, -ak.x * r0, -ak.y * r1);
    }
    g0 = G0 / s;
    g1 = G1 / s;
    return m + log(s);
  }
};

// ------------------------------------------------------------ full-covariance mixture
template <>
struct Obj<OBJ_MIXTURE_FULL> {
  template <typename T, int LPS>
  static __device__ __forceinline__ void whiten(const ObjParams<T>& o, int k, T x0, T x1, T& z0, T& z1,
                                                const Grp<LPS>& g) {
    const auto mk = ldg2(o.p0 + (size_t)k * o.dp + 2 * g.l);
    const T r0 = x0 - mk.x, r1 = x1 - mk.y;
    const T* LT = o.p3 + (size_t)k * o.dp * o.dp + 2 * g.l;   // LT[j][i] = L^-1[i][j]
    z0 = T(0);
    z1 = T(0);
#pragma unroll 4
    for (int j = 0; j < o.d; ++j) {
      const T rj = g.bcast((j & 1) ? r1 : r0, j >> 1);
      const auto lt = ldg2(LT + (size_t)j * o.dp);
      z0 = fma(lt.x, rj, z0);
      z1 = fma(lt.y, rj, z1);
    }
  }
  template <typename T, int LPS>
  static __device__ __forceinline__ T value(const ObjParams<T>& o, T x0, T x1, const Grp<LPS>& g) {
    T m = -CUDART_INF, s = T(0);
    for (int k = 0; k < o.K; ++k) {
      T z0, z1;
      whiten(o, k, x0, x1, z0, z1, g);
      const T q = g.sum(z0 * z0 + z1 * z1);
      lse_push(m, s, __ldg(o.p2 + k) - T(0.5) * q);
    }
    return m + log(s);
  }
  template <typename T, int LPS>
  static __device__ __forceinline__ T value_grad(const ObjParams<T>& o, T x0, T x1, T& g0, T& g1,
                                                 const Grp<LPS>& g) {
    T m = -CUDART_INF, s = T(0), G0 = T(0), G1 = T(0);
    for (int k = 0; k < o.K; ++k) {
      T z0, z1;
      whiten(o, k, x0, x1, z0, z1, g);
      const T q = g.sum(z0 * z0 + z1 * z1);
      const T* L = o.p1 + (size_t)k * o.dp * o.dp + 2 * g.l;  // L^-1[i][2l..2l+1]
      T s0 = T(0), s1 = T(0);
#pragma unroll 4
      for (int i = 0; i < o.d; ++i) {
        const T zi = g.bcast((i & 1) ? z1 : z0, i >> 1);
        const auto li = ldg2(L + (size_t)i * o.dp);
        s0 = fma(li.x, zi, s0);
        s1 = fma(li.y, zi, s1);
      }
      lse_push_grad(m, s, G0, G1, __ldg(o.p2 + k) - T(0.5) * q, -s0, -s1);
    }
    g0 = G0 / s;
    g1 = G1 / s;
    return m + log(s);
  }
};

// ------------------------------------------------------------ rotated quadratic
template <>
struct Obj<OBJ_QUADRATIC> {
  template <typename T, int LPS>
  static __device__ __forceinline__ T form(const ObjParams<T>& o, T x0, T x1, T& u0, T& u1,
                                           const Grp<LPS>& g) {
    const auto c = ldg2(o.p0 + 2 * g.l);
    const T r0 = x0 - c.x, r1 = x1 - c.y;
    const T* A = o.p1 + 2 * g.l;                                // A symmetric: row j = column j
    u0 = T(0);
    u1 = T(0);
#pragma unroll 8
    for (int j = 0; j < o.d; ++j) {
      const T rj = g.bcast((j & 1) ? r1 : r0, j >> 1);
      const auto a = ldg2(A + (size_t)j * o.dp);
      u0 = fma(a.x, rj, u0);
      u1 = fma(a.y, rj, u1);
    }
    return -g.sum(r0 * u0 + r1 * u1);
  }
  template <typename T, int LPS>
  static __device__ __forceinline__ T value(const ObjParams<T>& o, T x0, T x1, const Grp<LPS>& g) {
    T u0, u1;
    return form(o, x0, x1, u0, u1, g);
  }
  template <typename T, int LPS>
  static __device__ __forceinline__ T value_grad(const ObjParams<T>& o, T x0, T x1, T& g0, T& g1,
                                                 const Grp<LPS>& g) {
    T u0, u1;
    const T f = form(o, x0, x1, u0, u1, g);
    g0 = T(-2) * u0;
    g1 = T(-2) * u1;
    return f;
  }
};

// ------------------------------------------------------------ evaluation noise
// Sec. 5.6 noise model f~ = f + eps, eps ~ N(0, sigma_noise^2).  Each
// evaluation point gets its own draw: its binary32 coordinates are mixed with
// Wellons' lowbias32 finalizer, v_j = lowbias32(bits(x_j) ^ j * 0x9E3779B9),
// into the words (sum_j v_j, xor_j v_j (2j + 1)) that form the Philox counter
// (with the noise tag and the problem index); Box-Muller on the first two
// output words gives the normal.
__device__ __forceinline__ unsigned lowbias32(unsigned v) {
  v ^= v >> 16;
  v *= 0x7FEB352Du;
  v ^= v >> 15;
  v *= 0x846CA68Bu;
  v ^= v >> 16;
  return v;
}

template <typename T, int LPS>
__device__ __forceinline__ float point_noise(const ObjDev& O, const StepParams& S, int d, T x0, T x1,
                                             const Grp<LPS>& g) {
  const unsigned j0 = 2u * (unsigned)g.l;
  unsigned h1 = 0u, h2 = 0u;
  if ((int)j0 < d) {
    const unsigned v = lowbias32(__float_as_uint((float)x0) ^ (j0 * 0x9E3779B9u));
    h1 += v;
    h2 ^= v * (2u * j0 + 1u);
  }
  if ((int)j0 + 1 < d) {
    const unsigned v = lowbias32(__float_as_uint((float)x1) ^ ((j0 + 1u) * 0x9E3779B9u));
    h1 += v;
    h2 ^= v * (2u * j0 + 3u);
  }
  h1 = g.sum(h1);
  h2 = g.xor_all(h2);
  const uint4 w = philox4x32_10(make_uint4(h1, h2, TAG_NOISE << 24, ((unsigned)O.prob_index & 0xffffu) << 16),
                                make_uint2(S.seed_lo, S.seed_hi));
  return O.noise_sigma * sqrtf(-2.0f * logf(u01f(w.x))) * cospif(2.0f * u01f(w.y));
}

// f (+ noise) at a point, in the precision T of the parameters o.
template <int KIND, typename T, int LPS>
__device__ __forceinline__ T value_noisy(const ObjDev& O, const ObjParams<T>& o, const StepParams& S, T x0, T x1,
                                         const Grp<LPS>& g) {
  T f = Obj<KIND>::value(o, x0, x1, g);
  if (O.noise_sigma != 0.f) f += (T)point_noise(O, S, o.d, x0, x1, g);
  return f;
}

// f (+ noise) and the exact gradient of the noise-free f (the noise is constant in x).
template <int KIND, int LPS>
__device__ __forceinline__ float value_grad_noisy(const ObjDev& O, const StepParams& S, float x0, float x1,
                                                  float& g0, float& g1, const Grp<LPS>& g) {
  float f = Obj<KIND>::value_grad(O.f32, x0, x1, g0, g1, g);
  if (O.noise_sigma != 0.f) f += point_noise(O, S, O.f32.d, x0, x1, g);
  return f;
}

// ------------------------------------------------------------ gradient modes
// TE: the precision objective values are computed in (FP64 for the FD64 mode).
template <int GM>
using EvalT = typename std::conditional<GM == GRAD_FD64, double, float>::type;

template <int GM>
__device__ __forceinline__ const ObjParams<EvalT<GM>>& params_of(const ObjDev& O);
template <>
__device__ __forceinline__ const ObjParams<double>& params_of<GRAD_FD64>(const ObjDev& O) { return O.f64; }
template <>
__device__ __forceinline__ const ObjParams<float>& params_of<GRAD_FD32>(const ObjDev& O) { return O.f32; }
template <>
__device__ __forceinline__ const ObjParams<float>& params_of<GRAD_ADJOINT>(const ObjDev& O) { return O.f32; }

struct EvalCount {
  unsigned long long evals = 0, grads = 0;
};

// Central differences on the coordinates j < d: g_j = (f(x + h_j e_j) - f(x - h_j e_j)) / (x+_j - x-_j),
// the stencil points regenerated one at a time in registers.
template <int KIND, int GM, int LPS>
__device__ __forceinline__ void fd_gradient(const ObjDev& O, const StepParams& S, int d, float x0f, float x1f,
                                            float& g0, float& g1, const Grp<LPS>& g, EvalCount& ec) {
  using TE = EvalT<GM>;
  const auto& o = params_of<GM>(O);
  const TE x0 = (TE)x0f, x1 = (TE)x1f;
  g0 = 0.f;
  g1 = 0.f;
  for (int j = 0; j < d; ++j) {
    const int own = j >> 1, comp = j & 1;
    const TE xj = g.bcast(comp ? x1 : x0, own);
    const TE hj = (GM == GRAD_FD32) ? (TE)S.h_rel * fmax((TE)1, fabs(xj)) : (TE)S.h;
    const TE xp = xj + hj, xm = xj - hj;
    const bool mine = (g.l == own);
    const TE fp = value_noisy<KIND>(O, o, S, (mine && !comp) ? xp : x0, (mine && comp) ? xp : x1, g);
    const TE fm = value_noisy<KIND>(O, o, S, (mine && !comp) ? xm : x0, (mine && comp) ? xm : x1, g);
    const TE gj = (fp - fm) / (xp - xm);
    if (mine) {
      if (comp) g1 = (float)gj; else g0 = (float)gj;
    }
  }
  ec.evals += 2ull * d;
  ec.grads += 1ull;
}

// Value (in TE) and gradient of f at the float point (x0, x1).
template <int KIND, int GM, int LPS>
__device__ __forceinline__ EvalT<GM> value_and_gradient(const ObjDev& O, const StepParams& S, int d, float x0,
                                                        float x1, float& g0, float& g1, const Grp<LPS>& g,
                                                        EvalCount& ec) {
  using TE = EvalT<GM>;
  if constexpr (GM == GRAD_ADJOINT) {
    float a0, a1;
    const float f = value_grad_noisy<KIND>(O, S, x0, x1, a0, a1, g);
    g0 = a0;
    g1 = a1;
    ec.evals += 1;
    ec.grads += 1;
    return f;
  } else {
    const TE f = value_noisy<KIND>(O, params_of<GM>(O), S, (TE)x0, (TE)x1, g);
    ec.evals += 1;
    fd_gradient<KIND, GM, LPS>(O, S, d, x0, x1, g0, g1, g, ec);
    return f;
  }
}

// Gradient only (the value is not needed).
template <int KIND, int GM, int LPS>
__device__ __forceinline__ void gradient_only(const ObjDev& O, const StepParams& S, int d, float x0, float x1,
                                              float& g0, float& g1, const Grp<LPS>& g, EvalCount& ec) {
  if constexpr (GM == GRAD_ADJOINT) {
    Obj<KIND>::value_grad(O.f32, x0, x1, g0, g1, g);
    ec.evals += 1;
    ec.grads += 1;
  } else {
    fd_gradient<KIND, GM, LPS>(O, S, d, x0, x1, g0, g1, g, ec);
  }
}

}  // namespace chisao

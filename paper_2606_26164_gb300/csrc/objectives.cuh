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
//  * The Appendix D benchmark functions (separable sums, Ackley's two group
//    sums, Trid's neighbour products), one kind with a runtime function id.
//
// Lane l of a group holds the V consecutive coordinates V l .. V l + V - 1.
// A product with a d x d matrix walks the rows in blocks of V: in binary32 the
// group's vector is staged once in shared memory and each block of V values is
// one broadcast load (FP64: register shuffles from the owner lane), and the
// matrix row is read as one V-wide vector contiguous across the group (all
// groups of a warp read the same row, so the load is shared).  The quadratic's
// binary32 product uses that A is symmetric and reads about half of it
// (sym_times).
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

template <typename T, int V>
__device__ __forceinline__ void lse_push_grad(T& m, T& s, T (&G)[V], T lc, const T (&sc)[V]) {
  if (lc > m) {
    const T e = exp(m - lc);
    s = s * e + T(1);
#pragma unroll
    for (int v = 0; v < V; ++v) G[v] = G[v] * e + sc[v];
    m = lc;
  } else {
    const T e = exp(lc - m);
    s += e;
#pragma unroll
    for (int v = 0; v < V; ++v) G[v] = fma(e, sc[v], G[v]);
  }
}

// out[w] = sum_j M[j][V l + w] * r_j over the rows j < d (M row-major, stride dp).
// One accumulator per output: splitting the chains raised Phase 1's register
// count from 168 to 205 and cost more in occupancy than it won in ILP
// (measured: 2.46 vs 2.02 ms at d = 64, N = 65536).
// In binary32 the pairs of outputs use the packed two-lane FMA (each half an
// ordinary round-to-nearest FMA, so the results equal the scalar chain's).
// TRI names the nonzero triangle of a triangular M (the full-covariance mixture's factors),
// whose other rows a lane skips: row block jb (rows 4 jb .. 4 jb + 3) meets lane l's outputs
// only if jb <= l (TRI_LOWER: M[j][i] = 0 for j > i) or jb >= l (TRI_UPPER: M[j][i] = 0 for
// j < i).  The skipped terms are exact zeros, so only the sign of an exact zero can change;
// the warp still walks every block, but its idle lanes load nothing, which halves the bytes
// on the L1 path.
constexpr int TRI_DENSE = 0, TRI_LOWER = 1, TRI_UPPER = 2;
template <typename T, int V, int LPS, int TRI = TRI_DENSE>
__device__ __forceinline__ void rows_times(const T* M, int dp, int d, const T (&r)[V], T (&out)[V],
                                           const Grp<LPS>& g) {
  if constexpr (std::is_same<T, float>::value && V == 4) {
    // the group's vector r is staged once in shared memory (each lane its four values)
    // and read back four at a time as one broadcast load, instead of a register shuffle
    // per element
    __shared__ float4 rstage[256];                // the largest block of the objective kernels
    rstage[threadIdx.x] = make_float4(r[0], r[1], r[2], r[3]);
    __syncwarp(g.mask);
    const float4* grp = rstage + (threadIdx.x - g.l);
    float2 acc[V / 2];
#pragma unroll
    for (int w = 0; w < V / 2; ++w) acc[w] = make_float2(0.f, 0.f);
    const float* col = M + V * g.l;
    const int nb = (d + V - 1) / V;
#pragma unroll 1
    for (int jb = 0; jb < nb; ++jb) {
      if (TRI == TRI_LOWER && jb > (int)g.l) continue;
      if (TRI == TRI_UPPER && jb < (int)g.l) continue;
      const float4 rb = grp[jb];
      const float rv[4] = {rb.x, rb.y, rb.z, rb.w};
#pragma unroll
      for (int v = 0; v < V; ++v) {
        float a[V];
        ldg_vec<float, V>(col + (size_t)(jb * V + v) * dp, a);
        const float2 r2 = make_float2(rv[v], rv[v]);
#pragma unroll
        for (int w = 0; w < V / 2; ++w) acc[w] = __ffma2_rn(make_float2(a[2 * w], a[2 * w + 1]), r2, acc[w]);
      }
    }
    __syncwarp(g.mask);                           // the stage is reused by the next product
#pragma unroll
    for (int w = 0; w < V / 2; ++w) {
      out[2 * w] = acc[w].x;
      out[2 * w + 1] = acc[w].y;
    }
  } else {
#pragma unroll
    for (int w = 0; w < V; ++w) out[w] = T(0);
    const T* col = M + V * g.l;
    const int nb = (d + V - 1) / V;
#pragma unroll 2
    for (int jb = 0; jb < nb; ++jb) {
      const bool skip = (TRI == TRI_LOWER && jb > (int)g.l) || (TRI == TRI_UPPER && jb < (int)g.l);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const T rj = g.bcast(r[v], jb);              // every lane takes part in the broadcast
        if (skip) continue;
        T a[V];
        ldg_vec<T, V>(col + (size_t)(jb * V + v) * dp, a);
#pragma unroll
        for (int w = 0; w < V; ++w) out[w] = fma(a[w], rj, out[w]);
      }
    }
  }
}

// Two products with the same matrix at once (two evaluation points of one lane
// group): each row block is read once for both; each output keeps the FMA order of
// rows_times, so the results are the same bit for bit.
template <int LPS>
__device__ __forceinline__ void rows_times2(const float* M, int dp, int d, const float (&r1)[4],
                                            const float (&r2)[4], float (&out1)[4], float (&out2)[4],
                                            const Grp<LPS>& g) {
  __shared__ float4 rpair[2][256];                // the largest block of the objective kernels
  rpair[0][threadIdx.x] = make_float4(r1[0], r1[1], r1[2], r1[3]);
  rpair[1][threadIdx.x] = make_float4(r2[0], r2[1], r2[2], r2[3]);
  __syncwarp(g.mask);
  const float4* grp1 = rpair[0] + (threadIdx.x - g.l);
  const float4* grp2 = rpair[1] + (threadIdx.x - g.l);
  float2 a1[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, a2[2] = {a1[0], a1[1]};
  const float* col = M + 4 * g.l;
  const int nb = (d + 3) / 4;
#pragma unroll 1
  for (int jb = 0; jb < nb; ++jb) {
    const float4 b1 = grp1[jb], b2 = grp2[jb];
    const float v1[4] = {b1.x, b1.y, b1.z, b1.w}, v2[4] = {b2.x, b2.y, b2.z, b2.w};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float a[4];
      ldg_vec<float, 4>(col + (size_t)(jb * 4 + v) * dp, a);
      const float2 s1 = make_float2(v1[v], v1[v]), s2 = make_float2(v2[v], v2[v]);
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        const float2 aw = make_float2(a[2 * w], a[2 * w + 1]);
        a1[w] = __ffma2_rn(aw, s1, a1[w]);
        a2[w] = __ffma2_rn(aw, s2, a2[w]);
      }
    }
  }
  __syncwarp(g.mask);
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    out1[2 * w] = a1[w].x;
    out1[2 * w + 1] = a1[w].y;
    out2[2 * w] = a2[w].x;
    out2[2 * w + 1] = a2[w].y;
  }
}

// NP products with the same matrix at once (NP evaluation points of one lane group):
// each row block is read once for all of them; every output keeps the FMA order of
// rows_times, so the results are the same bit for bit.
template <int NP, int LPS>
__device__ __forceinline__ void rows_timesn(const float* M, int dp, int d, const float (&r)[NP][4],
                                            float (&out)[NP][4], const Grp<LPS>& g) {
  __shared__ float4 rmulti[NP][256];              // the largest block of the objective kernels
#pragma unroll
  for (int p = 0; p < NP; ++p) rmulti[p][threadIdx.x] = make_float4(r[p][0], r[p][1], r[p][2], r[p][3]);
  __syncwarp(g.mask);
  const int base = threadIdx.x - g.l;
  float2 acc[NP][2];
#pragma unroll
  for (int p = 0; p < NP; ++p) acc[p][0] = acc[p][1] = make_float2(0.f, 0.f);
  const float* col = M + 4 * g.l;
  const int nb = (d + 3) / 4;
#pragma unroll 1
  for (int jb = 0; jb < nb; ++jb) {
    float4 b[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) b[p] = rmulti[p][base + jb];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float a[4];
      ldg_vec<float, 4>(col + (size_t)(jb * 4 + v) * dp, a);
      const float2 a0 = make_float2(a[0], a[1]), a1 = make_float2(a[2], a[3]);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float s = v == 0 ? b[p].x : v == 1 ? b[p].y : v == 2 ? b[p].z : b[p].w;
        const float2 s2 = make_float2(s, s);
        acc[p][0] = __ffma2_rn(a0, s2, acc[p][0]);
        acc[p][1] = __ffma2_rn(a1, s2, acc[p][1]);
      }
    }
  }
  __syncwarp(g.mask);
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    out[p][0] = acc[p][0].x;
    out[p][1] = acc[p][0].y;
    out[p][2] = acc[p][1].x;
    out[p][3] = acc[p][1].y;
  }
}

// u = A r for a symmetric A (the quadratic) from its packed block table S: lane l
// owns block l (coordinates 4l .. 4l+3) of L = LPS blocks and at step k reads
// A[l][b], b = (l + k) mod L, as four float4 columns (table layout: capi.cu,
// quad_sym_table).  For 0 < k < L/2 the block serves both triangles: lane l adds
// A[l][b] r_b to its own outputs and hands A[l][b]^T r_l to lane b, which receives
// it from lane (b - k) mod L in the same step.  The diagonal block (k = 0) and, for
// L > 1, the block at k = L/2 (read by both partners for themselves) complete the
// product: L/2 + 1 blocks per lane instead of L, so a quarter fewer bytes cross
// the L1 data path per evaluation.  Each output is one chain in a fixed order:
// per step and column, the own term (packed FMA), then the received term.
template <int LPS>
__device__ __forceinline__ void sym_times(const float* S, const float (&r)[4], float (&out)[4],
                                          const Grp<LPS>& g) {
  constexpr int L = LPS;
  __shared__ float4 sstage[256];                  // the largest block of the objective kernels
  sstage[threadIdx.x] = make_float4(r[0], r[1], r[2], r[3]);
  __syncwarp(g.mask);
  const float4* grp = sstage + (threadIdx.x - g.l);
  const float4* tab = reinterpret_cast<const float4*>(S) + g.l;
  float2 acc[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  // one step: the block's four columns one at a time (own term with the packed FMA;
  // with `both` also the transposed term, sent to its owner at once and added to the
  // receiver's output c after that column's own term)
  auto step = [&](int k, bool both) {
    const float4 rb = grp[(g.l + k) & (L - 1)];
    const float rv[4] = {rb.x, rb.y, rb.z, rb.w};
    const int src = (g.l - k) & (L - 1);
    const float4* tk = tab + k * (4 * L);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float4 a = __ldg(tk + c * L);
      const float2 r2 = make_float2(rv[c], rv[c]);
      acc[0] = __ffma2_rn(make_float2(a.x, a.y), r2, acc[0]);
      acc[1] = __ffma2_rn(make_float2(a.z, a.w), r2, acc[1]);
      if (both) {
        const float t = fmaf(a.w, r[3], fmaf(a.z, r[2], fmaf(a.y, r[1], a.x * r[0])));
        const float rc = __shfl_sync(g.mask, t, src, L);
        if (c & 1) acc[c >> 1].y += rc; else acc[c >> 1].x += rc;
      }
    }
  };
  step(0, false);
#pragma unroll 1
  for (int k = 1; 2 * k < L; ++k) step(k, true);
  if (L > 1) step(L / 2, false);
  __syncwarp(g.mask);                             // the stage is reused by the next product
  out[0] = acc[0].x;
  out[1] = acc[0].y;
  out[2] = acc[1].x;
  out[3] = acc[1].y;
}

template <int KIND>
struct Obj;

// Objectives that evaluate two points of one lane group sharing their parameter loads
// (binary32 value and gradient).  Each point's arithmetic is that of a single
// evaluation in row order: value_grad's own for the diagonal mixture; for the
// quadratic, whose value_grad sums the symmetric block product (sym_times) in another
// order, the row walk of rows_times, so there the results can differ from
// value_grad's in the last bits.
template <int KIND>
struct HasPair : std::false_type {};
// ... and several points (value_grad_multi<NP>) sharing one pass over them.
template <int KIND>
struct HasMulti : std::false_type {};

// ------------------------------------------------------------ diagonal mixture
// The components go in steps of CK: their parameter loads, the lane's share of each
// |A^(1/2)(x - mu_k)|^2 and the CK group sums are independent and overlap; the
// log-sum-exp then takes them in component order.  Every operation and its order is
// that of one component at a time, so the results are the same bits for every CK; CK
// trades the overlap against registers (the batched contexts' tuner picks it per group).
template <int CK_>
struct DiagMixture {
  static constexpr int CK = CK_;
  template <typename T, int V, int LPS>
  static __device__ __forceinline__ void comp_terms(const ObjParams<T>& o, int k, const T (&x)[V], T& q,
                                                    T (&sc)[V], const Grp<LPS>& g) {
    T mk[V], ak[V];
    ldg_vec<T, V>(o.p0 + (size_t)k * o.dp + V * g.l, mk);
    ldg_vec<T, V>(o.p1 + (size_t)k * o.dp + V * g.l, ak);
    q = T(0);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const T r = x[v] - mk[v];
      q = fma(ak[v] * r, r, q);
      sc[v] = -ak[v] * r;
    }
  }
  template <typename T, int V, int LPS>
  static __device__ __forceinline__ T value(const ObjParams<T>& o, const T (&x)[V], const Grp<LPS>& g) {
    T m = -CUDART_INF, s = T(0);
    int k = 0;
    for (; k + CK <= o.K; k += CK) {
      T q[CK], sc[CK][V];
#pragma unroll
      for (int c = 0; c < CK; ++c) comp_terms<T, V, LPS>(o, k + c, x, q[c], sc[c], g);
#pragma unroll
      for (int c = 0; c < CK; ++c) q[c] = g.sum(q[c]);
#pragma unroll
      for (int c = 0; c < CK; ++c) lse_push(m, s, __ldg(o.p2 + k + c) - T(0.5) * q[c]);
    }
    for (; k < o.K; ++k) {
      T q, sc[V];
      comp_terms<T, V, LPS>(o, k, x, q, sc, g);
      q = g.sum(q);
      lse_push(m, s, __ldg(o.p2 + k) - T(0.5) * q);
    }
    return m + log(s);
  }
  template <typename T, int V, int LPS>
  static __device__ __forceinline__ T value_grad(const ObjParams<T>& o, const T (&x)[V], T (&gr)[V],
                                                 const Grp<LPS>& g) {
    T m = -CUDART_INF, s = T(0), G[V];
#pragma unroll
    for (int v = 0; v < V; ++v) G[v] = T(0);
    int k = 0;
    for (; k + CK <= o.K; k += CK) {
      T q[CK], sc[CK][V];
#pragma unroll
      for (int c = 0; c < CK; ++c) comp_terms<T, V, LPS>(o, k + c, x, q[c], sc[c], g);
#pragma unroll
      for (int c = 0; c < CK; ++c) q[c] = g.sum(q[c]);
#pragma unroll
      for (int c = 0; c < CK; ++c) lse_push_grad<T, V>(m, s, G, __ldg(o.p2 + k + c) - T(0.5) * q[c], sc[c]);
    }
    for (; k < o.K; ++k) {
      T q, sc[V];
      comp_terms<T, V, LPS>(o, k, x, q, sc, g);
      q = g.sum(q);
      lse_push_grad<T, V>(m, s, G, __ldg(o.p2 + k) - T(0.5) * q, sc);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) gr[v] = G[v] / s;
    return m + log(s);
  }
  template <int V, int LPS>
  static __device__ __forceinline__ void value_grad_pair(const ObjParams<float>& o, const float (&x1)[V],
                                                         const float (&x2)[V], float (&g1)[V], float (&g2)[V],
                                                         float& f1, float& f2, const Grp<LPS>& g) {
    float m1 = -CUDART_INF_F, s1 = 0.f, G1[V], m2 = -CUDART_INF_F, s2 = 0.f, G2[V];
#pragma unroll
    for (int v = 0; v < V; ++v) G1[v] = G2[v] = 0.f;
    constexpr int CP = CK / 2 > 0 ? CK / 2 : 1;       // two points share each component's loads
    int k = 0;
    for (; k + CP <= o.K; k += CP) {
      float q1[CP], q2[CP], sc1[CP][V], sc2[CP][V];
#pragma unroll
      for (int c = 0; c < CP; ++c) {
        float mk[V], ak[V];
        ldg_vec<float, V>(o.p0 + (size_t)(k + c) * o.dp + V * g.l, mk);
        ldg_vec<float, V>(o.p1 + (size_t)(k + c) * o.dp + V * g.l, ak);
        q1[c] = q2[c] = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const float r1 = x1[v] - mk[v], r2 = x2[v] - mk[v];
          q1[c] = fmaf(ak[v] * r1, r1, q1[c]);
          q2[c] = fmaf(ak[v] * r2, r2, q2[c]);
          sc1[c][v] = -ak[v] * r1;
          sc2[c][v] = -ak[v] * r2;
        }
      }
#pragma unroll
      for (int c = 0; c < CP; ++c) {
        q1[c] = g.sum(q1[c]);
        q2[c] = g.sum(q2[c]);
      }
#pragma unroll
      for (int c = 0; c < CP; ++c) {
        const float ck = __ldg(o.p2 + k + c);
        lse_push_grad<float, V>(m1, s1, G1, ck - 0.5f * q1[c], sc1[c]);
        lse_push_grad<float, V>(m2, s2, G2, ck - 0.5f * q2[c], sc2[c]);
      }
    }
    for (; k < o.K; ++k) {
      float mk[V], ak[V], sc1[V], sc2[V];
      ldg_vec<float, V>(o.p0 + (size_t)k * o.dp + V * g.l, mk);
      ldg_vec<float, V>(o.p1 + (size_t)k * o.dp + V * g.l, ak);
      float q1 = 0.f, q2 = 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const float r1 = x1[v] - mk[v], r2 = x2[v] - mk[v];
        q1 = fmaf(ak[v] * r1, r1, q1);
        q2 = fmaf(ak[v] * r2, r2, q2);
        sc1[v] = -ak[v] * r1;
        sc2[v] = -ak[v] * r2;
      }
      q1 = g.sum(q1);
      q2 = g.sum(q2);
      const float ck = __ldg(o.p2 + k);
      lse_push_grad<float, V>(m1, s1, G1, ck - 0.5f * q1, sc1);
      lse_push_grad<float, V>(m2, s2, G2, ck - 0.5f * q2, sc2);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      g1[v] = G1[v] / s1;
      g2[v] = G2[v] / s2;
    }
    f1 = m1 + logf(s1);
    f2 = m2 + logf(s2);
  }
};
template <>
struct Obj<OBJ_MIXTURE_DIAG> : DiagMixture<4> {};
template <>
struct Obj<OBJ_MIXDIAG_C2> : DiagMixture<2> {};
template <>
struct Obj<OBJ_MIXDIAG_C8> : DiagMixture<8> {};
template <>
struct HasPair<OBJ_MIXTURE_DIAG> : std::true_type {};
template <>
struct HasPair<OBJ_MIXDIAG_C2> : std::true_type {};
template <>
struct HasPair<OBJ_MIXDIAG_C8> : std::true_type {};

// ------------------------------------------------------------ full-covariance mixture
template <>
struct Obj<OBJ_MIXTURE_FULL> {
  // z = L^-1 (x - mu_k).  The value and gradient pass skips the zero triangle (each lane
  // loads only the rows that meet its outputs: fewer bytes on the L1 path, 1.94 -> 1.67 s
  // per d = 64, K = 256 cycle at N = 65536); the value alone walks the dense rows, which is
  // faster at the small populations where these products are latency-bound.
  template <typename T, int V, int LPS, int TRI = TRI_DENSE>
  static __device__ __forceinline__ void whiten(const ObjParams<T>& o, int k, const T (&x)[V], T (&z)[V],
                                                const Grp<LPS>& g) {
    T mk[V], r[V];
    ldg_vec<T, V>(o.p0 + (size_t)k * o.dp + V * g.l, mk);
#pragma unroll
    for (int v = 0; v < V; ++v) r[v] = x[v] - mk[v];
    rows_times<T, V, LPS, TRI>(o.p3 + (size_t)k * o.dp * o.dp, o.dp, o.d, r, z, g);   // (L^-1)^T rows
  }
  template <typename T, int V, int LPS>
  static __device__ __forceinline__ T value(const ObjParams<T>& o, const T (&x)[V], const Grp<LPS>& g) {
    T m = -CUDART_INF, s = T(0);
    for (int k = 0; k < o.K; ++k) {
      T z[V];
      whiten<T, V, LPS>(o, k, x, z, g);
      T q = T(0);
#pragma unroll
      for (int v = 0; v < V; ++v) q = fma(z[v], z[v], q);
      lse_push(m, s, __ldg(o.p2 + k) - T(0.5) * g.sum(q));
    }
    return m + log(s);
  }
  template <typename T, int V, int LPS>
  static __device__ __forceinline__ T value_grad(const ObjParams<T>& o, const T (&x)[V], T (&gr)[V],
                                                 const Grp<LPS>& g) {
    T m = -CUDART_INF, s = T(0), G[V];
#pragma unroll
    for (int v = 0; v < V; ++v) G[v] = T(0);
    for (int k = 0; k < o.K; ++k) {
      T z[V], sc[V];
      whiten<T, V, LPS, TRI_LOWER>(o, k, x, z, g);
      T q = T(0);
#pragma unroll
      for (int v = 0; v < V; ++v) q = fma(z[v], z[v], q);
      q = g.sum(q);
      rows_times<T, V, LPS, TRI_UPPER>(o.p1 + (size_t)k * o.dp * o.dp, o.dp, o.d, z, sc, g);  // L^-1 rows: (L^-T z)
#pragma unroll
      for (int v = 0; v < V; ++v) sc[v] = -sc[v];
      lse_push_grad<T, V>(m, s, G, __ldg(o.p2 + k) - T(0.5) * q, sc);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) gr[v] = G[v] / s;
    return m + log(s);
  }
};

// ------------------------------------------------------------ rotated quadratic
template <>
struct Obj<OBJ_QUADRATIC> {
  template <typename T, int V, int LPS>
  static __device__ __forceinline__ T form(const ObjParams<T>& o, const T (&x)[V], T (&u)[V], const Grp<LPS>& g) {
    T c[V], r[V];
    ldg_vec<T, V>(o.p0 + V * g.l, c);
#pragma unroll
    for (int v = 0; v < V; ++v) r[v] = x[v] - c[v];
    if constexpr (std::is_same<T, float>::value && V == 4)
      sym_times<LPS>(o.p2, r, u, g);                                  // half the off-diagonal blocks
    else
      rows_times<T, V, LPS>(o.p1, o.dp, o.d, r, u, g);               // A symmetric: row j = column j
    T acc = T(0);
#pragma unroll
    for (int v = 0; v < V; ++v) acc = fma(r[v], u[v], acc);
    return -g.sum(acc);
  }
  template <typename T, int V, int LPS>
  static __device__ __forceinline__ T value(const ObjParams<T>& o, const T (&x)[V], const Grp<LPS>& g) {
    T u[V];
    return form<T, V, LPS>(o, x, u, g);
  }
  template <typename T, int V, int LPS>
  static __device__ __forceinline__ T value_grad(const ObjParams<T>& o, const T (&x)[V], T (&gr)[V],
                                                 const Grp<LPS>& g) {
    T u[V];
    const T f = form<T, V, LPS>(o, x, u, g);
#pragma unroll
    for (int v = 0; v < V; ++v) gr[v] = T(-2) * u[v];
    return f;
  }
  template <int V, int LPS>
  static __device__ __forceinline__ void value_grad_pair(const ObjParams<float>& o, const float (&x1)[V],
                                                         const float (&x2)[V], float (&g1)[V], float (&g2)[V],
                                                         float& f1, float& f2, const Grp<LPS>& g) {
    float c[V], r1[V], r2[V], u1[V], u2[V];
    ldg_vec<float, V>(o.p0 + V * g.l, c);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      r1[v] = x1[v] - c[v];
      r2[v] = x2[v] - c[v];
    }
    rows_times2<LPS>(o.p1, o.dp, o.d, r1, r2, u1, u2, g);
    float acc1 = 0.f, acc2 = 0.f;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      acc1 = fmaf(r1[v], u1[v], acc1);
      acc2 = fmaf(r2[v], u2[v], acc2);
      g1[v] = -2.f * u1[v];
      g2[v] = -2.f * u2[v];
    }
    f1 = -g.sum(acc1);
    f2 = -g.sum(acc2);
  }
  template <int NP, int V, int LPS>
  static __device__ __forceinline__ void value_grad_multi(const ObjParams<float>& o, const float (&x)[NP][V],
                                                          float (&gr)[NP][V], float (&f)[NP], const Grp<LPS>& g) {
    static_assert(V == 4, "four coordinates per lane");
    float c[V], r[NP][V], u[NP][V];
    ldg_vec<float, V>(o.p0 + V * g.l, c);
#pragma unroll
    for (int p = 0; p < NP; ++p)
#pragma unroll
      for (int v = 0; v < V; ++v) r[p][v] = x[p][v] - c[v];
    rows_timesn<NP, LPS>(o.p1, o.dp, o.d, r, u, g);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      float acc = 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        acc = fmaf(r[p][v], u[p][v], acc);
        gr[p][v] = -2.f * u[p][v];
      }
      f[p] = -g.sum(acc);
    }
  }
};
template <>
struct HasPair<OBJ_QUADRATIC> : std::true_type {};
template <>
struct HasMulti<OBJ_QUADRATIC> : std::true_type {};

// ------------------------------------------------------------ Appendix D benchmark functions
// Negated (maximisation) forms, coordinate i = j + 1 for the lane's coordinate j;
// padded coordinates (j >= d) contribute nothing.  Non-differentiable points take
// the zero subgradient of the offending term (Ackley at x = 0, Bukin N.6 on its
// ridge and at x_1 = -10).
template <typename T>
__device__ __forceinline__ T cospi_t(T v) {
  if constexpr (std::is_same<T, float>::value) return cospif(v); else return cospi(v);
}
template <typename T>
__device__ __forceinline__ T sinpi_t(T v) {
  if constexpr (std::is_same<T, float>::value) return sinpif(v); else return sinpi(v);
}
template <typename T>
__device__ __forceinline__ T sgn(T v) {
  return (T)((v > T(0)) - (v < T(0)));
}

template <>
struct Obj<OBJ_BENCH> {
  // f, and with GR the gradient, at the lane group's point
  template <bool GR, typename T, int V, int LPS>
  static __device__ __forceinline__ T eval(const ObjParams<T>& o, const T (&x)[V], T (&gr)[V], const Grp<LPS>& g) {
    const int d = o.d;
    const int j0 = V * g.l;
    T acc = T(0);
    switch (o.fn) {
      case FN_RASTRIGIN: {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const bool in = j0 + v < d;
          const T c = cospi_t(T(2) * x[v]);
          if (in) acc -= x[v] * x[v] - T(10) * c + T(10);
          if (GR) gr[v] = in ? -(T(2) * x[v] + T(2) * T(CUDART_PI) * T(10) * sinpi_t(T(2) * x[v])) : T(0);
        }
        return g.sum(acc);
      }
      case FN_ACKLEY: {
        T s2 = T(0), sc = T(0);
#pragma unroll
        for (int v = 0; v < V; ++v)
          if (j0 + v < d) {
            s2 += x[v] * x[v];
            sc += cospi_t(T(2) * x[v]);
          }
        s2 = g.sum(s2);
        sc = g.sum(sc);
        const T r = sqrt(s2 / T(d));
        const T e1 = exp(T(-0.2) * r), e2 = exp(sc / T(d));
        if (GR) {
          const T radial = r > T(0) ? T(-20) * T(0.2) * e1 / (T(d) * r) : T(0);
#pragma unroll
          for (int v = 0; v < V; ++v)
            gr[v] = (j0 + v < d) ? radial * x[v] - T(2) * T(CUDART_PI) / T(d) * e2 * sinpi_t(T(2) * x[v]) : T(0);
        }
        return T(20) * e1 + e2 - T(20) - T(2.718281828459045);
      }
      case FN_SCHWEFEL: {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const bool in = j0 + v < d;
          const T s = sqrt(fabs(x[v]));
          const T sn = sin(s);
          if (in) acc += x[v] * sn;
          if (GR) gr[v] = in ? sn + T(0.5) * s * cos(s) : T(0);
        }
        return g.sum(acc) - T(418.9829) * T(d);
      }
      case FN_STYBLINSKI_TANG: {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const bool in = j0 + v < d;
          const T x2 = x[v] * x[v];
          if (in) acc += x2 * x2 - T(16) * x2 + T(5) * x[v];
          if (GR) gr[v] = in ? T(-0.5) * (T(4) * x2 * x[v] - T(32) * x[v] + T(5)) : T(0);
        }
        return T(-0.5) * g.sum(acc);
      }
      case FN_MICHALEWICZ: {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const bool in = j0 + v < d;
          const T i = T(j0 + v + 1);
          const T u = i * x[v] * x[v] / T(CUDART_PI);
          const T su = sin(u), s2 = su * su, s4 = s2 * s2, s8 = s4 * s4, s16 = s8 * s8;
          const T s20 = s16 * s4, s19 = s16 * s2 * su;
          const T sx = sin(x[v]);
          if (in) acc += sx * s20;
          if (GR)
            gr[v] = in ? cos(x[v]) * s20 + sx * T(20) * s19 * cos(u) * (T(2) * i * x[v] / T(CUDART_PI)) : T(0);
        }
        return g.sum(acc);
      }
      case FN_TRID: {
        // neighbours across the lane boundary come from the previous / next lane
        const T prev_last = g.from_prev(x[V - 1]);
        const T next_first = g.from_next(x[0]);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int j = j0 + v;
          const bool in = j < d;
          const T prev = v > 0 ? x[v - 1] : prev_last;
          const T next = v < V - 1 ? x[v + 1] : next_first;
          const T dm = x[v] - T(1);
          if (in) acc += -dm * dm + (j >= 1 ? x[v] * prev : T(0));
          if (GR) gr[v] = in ? T(-2) * dm + (j >= 1 ? prev : T(0)) + (j + 1 < d ? next : T(0)) : T(0);
        }
        return g.sum(acc);
      }
      default: {                                    // FN_BUKIN6: d = 2, both coordinates in lane 0
        T f = T(0);
        if (GR) {
#pragma unroll
          for (int v = 0; v < V; ++v) gr[v] = T(0);
        }
        if (g.l == 0) {
          const T w = x[1] - T(0.01) * x[0] * x[0];
          const T aw = fabs(w);
          f = T(-100) * sqrt(aw) - T(0.01) * fabs(x[0] + T(10));
          if (GR) {
            const T dw = aw > T(0) ? T(-50) * sgn(w) / sqrt(aw) : T(0);
            gr[0] = dw * (T(-0.02) * x[0]) - T(0.01) * sgn(x[0] + T(10));
            gr[1] = dw;
          }
        }
        return g.sum(f);
      }
    }
  }
  template <typename T, int V, int LPS>
  static __device__ __forceinline__ T value(const ObjParams<T>& o, const T (&x)[V], const Grp<LPS>& g) {
    T unused[V];
    return eval<false, T, V, LPS>(o, x, unused, g);
  }
  template <typename T, int V, int LPS>
  static __device__ __forceinline__ T value_grad(const ObjParams<T>& o, const T (&x)[V], T (&gr)[V],
                                                 const Grp<LPS>& g) {
    return eval<true, T, V, LPS>(o, x, gr, g);
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

template <typename T, int V, int LPS>
__device__ __forceinline__ float point_noise(const ObjDev& O, const StepParams& S, int d, const T (&x)[V],
                                             const Grp<LPS>& g) {
  unsigned h1 = 0u, h2 = 0u;
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const unsigned j = (unsigned)(V * g.l + v);
    if ((int)j < d) {
      const unsigned w = lowbias32(__float_as_uint((float)x[v]) ^ (j * 0x9E3779B9u));
      h1 += w;
      h2 ^= w * (2u * j + 1u);
    }
  }
  h1 = g.sum(h1);
  h2 = g.xor_all(h2);
  const uint4 w = philox4x32_10(make_uint4(h1, h2, TAG_NOISE << 24, ((unsigned)O.prob_index & 0xffffu) << 16),
                                make_uint2(S.seed_lo, S.seed_hi));
  return O.noise_sigma * sqrtf(-2.0f * logf(u01f(w.x))) * cospif(2.0f * u01f(w.y));
}

// f (+ noise) at a point, in the precision T of the parameters o.
template <int KIND, typename T, int V, int LPS>
__device__ __forceinline__ T value_noisy(const ObjDev& O, const ObjParams<T>& o, const StepParams& S,
                                         const T (&x)[V], const Grp<LPS>& g) {
  T f = Obj<KIND>::template value<T, V, LPS>(o, x, g);
  if (O.noise_sigma != 0.f) f += (T)point_noise<T, V, LPS>(O, S, o.d, x, g);
  return f;
}

// f (+ noise) and the exact gradient of the noise-free f (the noise is constant in x).
template <int KIND, int V, int LPS>
__device__ __forceinline__ float value_grad_noisy(const ObjDev& O, const StepParams& S, const float (&x)[V],
                                                  float (&gr)[V], const Grp<LPS>& g) {
  float f = Obj<KIND>::template value_grad<float, V, LPS>(O.f32, x, gr, g);
  if (O.noise_sigma != 0.f) f += point_noise<float, V, LPS>(O, S, O.f32.d, x, g);
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

// f (+ noise) at a binary32 point, in the evaluation precision of the gradient mode.
template <int KIND, int GM, int V, int LPS>
__device__ __forceinline__ EvalT<GM> value_at(const ObjDev& O, const StepParams& S, const float (&xf)[V],
                                              const Grp<LPS>& g, EvalCount& ec) {
  using TE = EvalT<GM>;
  TE x[V];
#pragma unroll
  for (int v = 0; v < V; ++v) x[v] = (TE)xf[v];
  ec.evals += 1;
  return value_noisy<KIND, TE, V, LPS>(O, params_of<GM>(O), S, x, g);
}

// The stencil coordinates x_j +- h_j, each one rounded sum (never fused with the product that
// forms h_j), so every kernel that forms them gets the same bits.
__device__ __forceinline__ float stencil_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float stencil_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double stencil_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double stencil_sub(double a, double b) { return __dsub_rn(a, b); }

// Central differences on the coordinates j < d: g_j = (f(x + h_j e_j) - f(x - h_j e_j)) / (x+_j - x-_j),
// the stencil points regenerated one at a time in registers.
template <int KIND, int GM, int V, int LPS>
__device__ __forceinline__ void fd_gradient(const ObjDev& O, const StepParams& S, int d, const float (&xf)[V],
                                            float (&gr)[V], const Grp<LPS>& g, EvalCount& ec) {
  using TE = EvalT<GM>;
  const auto& o = params_of<GM>(O);
  TE x[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    x[v] = (TE)xf[v];
    gr[v] = 0.f;
  }
  const int nb = (d + V - 1) / V;
  for (int jl = 0; jl < nb; ++jl) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if (jl * V + v < d) {
        const TE xj = g.bcast(x[v], jl);
        const TE hj = (GM == GRAD_FD32) ? (TE)S.h_rel * fmax((TE)1, fabs(xj)) : (TE)S.h;
        const TE xp = stencil_add(xj, hj), xm = stencil_sub(xj, hj);
        const bool mine = (g.l == jl);
        TE y[V];
#pragma unroll
        for (int w = 0; w < V; ++w) y[w] = x[w];
        if (mine) y[v] = xp;
        const TE fp = value_noisy<KIND, TE, V, LPS>(O, o, S, y, g);
        if (mine) y[v] = xm;
        const TE fm = value_noisy<KIND, TE, V, LPS>(O, o, S, y, g);
        if (mine) gr[v] = (float)((fp - fm) / (xp - xm));
      }
    }
  }
  ec.evals += 2ull * d;
  ec.grads += 1ull;
}

// Value (in TE) and gradient of f at the float point x.
template <int KIND, int GM, int V, int LPS>
__device__ __forceinline__ EvalT<GM> value_and_gradient(const ObjDev& O, const StepParams& S, int d,
                                                        const float (&x)[V], float (&gr)[V], const Grp<LPS>& g,
                                                        EvalCount& ec) {
  using TE = EvalT<GM>;
  if constexpr (GM == GRAD_ADJOINT) {
    ec.evals += 1;
    ec.grads += 1;
    return value_grad_noisy<KIND, V, LPS>(O, S, x, gr, g);
  } else {
    TE xe[V];
#pragma unroll
    for (int v = 0; v < V; ++v) xe[v] = (TE)x[v];
    const TE f = value_noisy<KIND, TE, V, LPS>(O, params_of<GM>(O), S, xe, g);
    ec.evals += 1;
    fd_gradient<KIND, GM, V, LPS>(O, S, d, x, gr, g, ec);
    return f;
  }
}

// Gradient only (the value is not needed).
template <int KIND, int GM, int V, int LPS>
__device__ __forceinline__ void gradient_only(const ObjDev& O, const StepParams& S, int d, const float (&x)[V],
                                              float (&gr)[V], const Grp<LPS>& g, EvalCount& ec) {
  if constexpr (GM == GRAD_ADJOINT) {
    Obj<KIND>::template value_grad<float, V, LPS>(O.f32, x, gr, g);
    ec.evals += 1;
    ec.grads += 1;
  } else {
    fd_gradient<KIND, GM, V, LPS>(O, S, d, x, gr, g, ec);
  }
}

}  // namespace chisao

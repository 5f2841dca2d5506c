// Objective-independent kernels of one oscillation cycle: f_max and the stick
// test (Phase 2, Eq. 3), ordered compaction of the sample sets, L-infinity
// deduplication (Phase 3, Eq. 4), the reseeding strategies (Phase 4,
// Sec. 3.2.4) with the Golden Rooster's FP64 Householder QR, and the scale
// estimates' final reduction (Phases 5/6).
#include <algorithm>

#include "host.h"
#include "dev_common.cuh"

namespace chisao {

constexpr int NT_LIN = 256;       // threads of the elementwise kernels
constexpr int NT_ONE = 1024;      // threads of the single-block kernels

// ------------------------------------------------------------ cycle bookkeeping
// Every kernel below is a body taking its block index b and block count nb within the
// problem, wrapped once as a launch over one problem (b = blockIdx.x, nb = gridDim.x)
// and once as a launch over all the problems of a context (the *_all kernels: the block's
// problem and position from the launch's AllTab), which computes the same bits.
#define CHISAO_ALL_KERNEL(NAME, NT, BODY_CALL)                              \
  __global__ void __launch_bounds__(NT) NAME##_all(AllTab T) {             \
    const BlkPos pos = all_pos(T);                                        \
    const ProbDev& P = T.probs[pos.q];                                    \
    const StepParams& S = T.sps[pos.q];                                   \
    (void)S;                                                              \
    BODY_CALL;                                                            \
  }

__device__ __forceinline__ void cycle_begin_body(const ProbDev& P, unsigned b, unsigned nb) {
  for (int w = b * blockDim.x + threadIdx.x; w < P.nwords; w += nb * blockDim.x) {
    P.stuck[w] = 0u;                 // Phase 1: release all
    P.removed[w] = 0u;
  }
  if (b == 0 && threadIdx.x == 0) {
    P.cnt->fmax_key = 0u;
    P.cnt->n_stuck0 = 0;
    P.cnt->reseed_mode = RESEED_NONE;
  }
}
__global__ void k_cycle_begin(ProbDev P) { cycle_begin_body(P, blockIdx.x, gridDim.x); }
CHISAO_ALL_KERNEL(k_cycle_begin, 256, cycle_begin_body(P, pos.b, pos.nb))

__global__ void k_cycle_end(ProbDev P) {
  if (threadIdx.x == 0) P.cnt->cycle += 1;
}
CHISAO_ALL_KERNEL(k_cycle_end, 32, if (threadIdx.x == 0) P.cnt->cycle += 1)

__global__ void k_set_cycle(ProbDev P, int completed) {
  if (threadIdx.x == 0) P.cnt->cycle = completed;
}

// ------------------------------------------------------------ Phase 2
// f_max over the finite f (max is order-independent, so atomics are exact).
__device__ __forceinline__ void fmax_body(const ProbDev& P, unsigned b, unsigned nb) {
  unsigned key = 0u;
  for (int i = b * blockDim.x + threadIdx.x; i < P.n; i += nb * blockDim.x) {
    const float v = P.f[i];
    if (isfinite(v)) key = max(key, fkey(v));
  }
  block_max_key<NT_LIN>(key, &P.cnt->fmax_key);
}
__global__ void __launch_bounds__(NT_LIN) k_fmax(ProbDev P) { fmax_body(P, blockIdx.x, gridDim.x); }
CHISAO_ALL_KERNEL(k_fmax, NT_LIN, fmax_body(P, pos.b, pos.nb))

// stuck_i = (|g_i|_inf < eps_grad) and (f_i >= fl(f_max + log delta)), binary32
// compares; one warp ballot per 32 samples writes one mask word.
__device__ __forceinline__ void freeze_body(const ProbDev& P, const StepParams& S, unsigned blk) {
  const int i = blk * blockDim.x + threadIdx.x;
  const unsigned key = P.cnt->fmax_key;
  const float fmax = key ? fkey_inv(key) : -CUDART_INF_F;
  const float thr = fmax + S.log_delta;
  bool st = false;
  if (i < P.n) {
    float gm = 0.f;
    bool bad = false;
    const float4* row = reinterpret_cast<const float4*>(P.g + (size_t)i * P.dp);
    for (int q = 0; q < P.dp / 4; ++q) {
      const float4 v = row[q];
      const float a = fabsf(v.x), b = fabsf(v.y), c = fabsf(v.z), e = fabsf(v.w);
      bad |= (a != a) | (b != b) | (c != c) | (e != e);
      gm = fmaxf(gm, fmaxf(fmaxf(a, b), fmaxf(c, e)));
    }
    st = !bad && (gm < S.eps_grad) && (P.f[i] >= thr);
  }
  const unsigned b = __ballot_sync(0xffffffffu, st);
  if ((threadIdx.x & 31) == 0 && (i >> 5) < P.nwords) {
    P.stuck[i >> 5] = b;
    if (b) atomicAdd(&P.cnt->n_stuck0, __popc(b));
  }
  if (i == 0) P.cnt->fmax = fmax;
}
__global__ void __launch_bounds__(NT_LIN) k_freeze(ProbDev P, StepParams S) { freeze_body(P, S, blockIdx.x); }
CHISAO_ALL_KERNEL(k_freeze, NT_LIN, freeze_body(P, S, pos.b))

// ------------------------------------------------------------ ordered compaction
// One block; warp w owns a contiguous run of mask words; a block scan of the per-warp
// counts gives each run its output offset, so the list comes out in increasing sample
// index.  Within a run the warp takes 32 words at a time and writes them one word after
// another, lane j storing bit j: consecutive set bits go to consecutive positions, so
// each store is coalesced.
template <class WordFn>
__device__ int block_compact(int nwords, WordFn word_of, int* out) {
  constexpr int NWARP = NT_ONE / 32;
  __shared__ int scan[NWARP];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int per = (nwords + NWARP - 1) / NWARP;
  const int w0 = min(nwords, warp * per), w1 = min(nwords, w0 + per);
  int c = 0;
  for (int w = w0 + lane; w < w1; w += 32) c += __popc(word_of(w));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) scan[warp] = c;
  __syncthreads();
  int base = 0, total = 0;
  for (int k = 0; k < NWARP; ++k) {                 // every thread scans the 32 counts itself
    const int v = scan[k];
    if (k < warp) base += v;
    total += v;
  }
  const unsigned below = (1u << lane) - 1u;
  for (int r0 = w0; r0 < w1; r0 += 32) {
    const unsigned m = r0 + lane < w1 ? word_of(r0 + lane) : 0u;
    const int pc = __popc(m);
    int ex = pc;                                     // inclusive scan of the round's counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, ex, o);
      if (lane >= o) ex += u;
    }
    const int round_total = __shfl_sync(0xffffffffu, ex, 31);
    ex -= pc;
    const int nk = min(32, w1 - r0);
    for (int k = 0; k < nk; ++k) {
      const unsigned mk = __shfl_sync(0xffffffffu, m, k);
      const int ok = __shfl_sync(0xffffffffu, ex, k);
      if ((mk >> lane) & 1u) out[base + ok + __popc(mk & below)] = (r0 + k) * 32 + lane;
    }
    base += round_total;
  }
  __syncthreads();
  return total;
}

__device__ __forceinline__ unsigned valid_mask(const ProbDev& P, int w) {
  const int rem = P.n - w * 32;
  return rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u);
}

__device__ __forceinline__ void compact_stuck_body(const ProbDev& P) {
  const int S = block_compact(P.nwords, [&](int w) { return P.stuck[w]; }, P.l_stuck);
  if (threadIdx.x == 0) P.cnt->n_stuck0 = S;
}
__global__ void __launch_bounds__(NT_ONE) k_compact_stuck(ProbDev P) { compact_stuck_body(P); }
CHISAO_ALL_KERNEL(k_compact_stuck, NT_ONE, compact_stuck_body(P))

// After deduplication: stuck &= ~removed, then the free-slot list (removed),
// the unfrozen list (neither stuck nor removed) and the survivor list.
__device__ __forceinline__ void compact_dedup_body(const ProbDev& P) {
  for (int w = threadIdx.x; w < P.nwords; w += NT_ONE) P.stuck[w] &= ~P.removed[w];
  __syncthreads();
  const int K = block_compact(P.nwords, [&](int w) { return P.removed[w]; }, P.l_free);
  const int U = block_compact(P.nwords, [&](int w) { return ~(P.stuck[w] | P.removed[w]) & valid_mask(P, w); },
                              P.l_unf);
  const int S = block_compact(P.nwords, [&](int w) { return P.stuck[w]; }, P.l_surv);
  if (threadIdx.x == 0) {
    Counters* c = P.cnt;
    c->n_removed = K;
    c->n_free = K;
    c->n_unfrozen = U;
    c->n_surv = S;
    c->n_stuck = S;
  }
}
__global__ void __launch_bounds__(NT_ONE) k_compact_dedup(ProbDev P) { compact_dedup_body(P); }
CHISAO_ALL_KERNEL(k_compact_dedup, NT_ONE, compact_dedup_body(P))

// ------------------------------------------------------------ Phase 3
// For every stuck x_j: removed iff some other stuck x_i ranks above it
// (f desc, index asc) and max_k |x_ik - x_jk| < eps_dup (binary32).
//
// Candidates come from a spatial hash (App. A: the L-inf ball is a hypercube):
// each stuck sample is filed under the cells floor((x_a - lo_a) / h) of the three
// coordinates a along which the stuck set is most spread, h = eps_dup (1 + 1e-6).
// Any pair the binary32 test can accept is closer than eps_dup (1 + 2^-23) in
// every coordinate, so with h slightly above that (and the cell computed in FP64)
// their cells differ by at most one along each hashed axis: the 27 neighbouring
// cells hold every candidate, and the exact test on them decides as the pairwise
// scan would.  The outcome is order-free, so the mask is the same bit for bit.
constexpr unsigned long long HASH_EMPTY = ~0ull;

__device__ __forceinline__ unsigned ordered_bits(float v) {   // monotone map float -> unsigned
  const unsigned u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered_bits(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ unsigned long long cell_key(long long c0, long long c1, long long c2) {
  unsigned long long k = (unsigned long long)c0 * 0x9E3779B97F4A7C15ull;      // splitmix-style mixing
  k ^= (unsigned long long)c1 * 0xC2B2AE3D27D4EB4Full + (k >> 29);
  k ^= (unsigned long long)c2 * 0x165667B19E3779F9ull + (k >> 31);
  k ^= k >> 33;
  k *= 0xFF51AFD7ED558CCDull;
  k ^= k >> 33;
  return k == HASH_EMPTY ? 0ull : k;
}
__device__ __forceinline__ long long cell_of(float x, float lo, double h) {
  return (long long)floor(((double)x - (double)lo) / h);
}

// table slots empty, coordinate spreads reset
__device__ __forceinline__ void hash_clear_body(const ProbDev& P, unsigned b, unsigned nb) {
  const int t = b * blockDim.x + threadIdx.x;
  if (P.cnt->n_stuck0 == 0) return;
  for (int s = t; s <= P.hmask; s += nb * blockDim.x) {
    P.hkey[s] = HASH_EMPTY;
    P.hbest[s] = 0ull;
    P.hhead[s] = -1;
  }
  if (t < P.dp) {
    P.hspread[t] = 0xFFFFFFFFu;
    P.hspread[P.dp + t] = 0u;
  }
}
__global__ void __launch_bounds__(NT_LIN) k_hash_clear(ProbDev P) { hash_clear_body(P, blockIdx.x, gridDim.x); }
CHISAO_ALL_KERNEL(k_hash_clear, NT_LIN, hash_clear_body(P, pos.b, pos.nb))

// per-coordinate min and max over the stuck set
__device__ __forceinline__ void hash_spread_body(const ProbDev& P, unsigned b) {
  const long long t = (long long)b * blockDim.x + threadIdx.x;
  const int Sn = P.cnt->n_stuck0;
  if (t >= (long long)Sn * P.d) return;
  const int jj = (int)(t / P.d), a = (int)(t % P.d);
  const unsigned k = ordered_bits(P.x[(size_t)P.l_stuck[jj] * P.dp + a]);
  atomicMin(&P.hspread[a], k);
  atomicMax(&P.hspread[P.dp + a], k);
}
__global__ void __launch_bounds__(NT_LIN) k_hash_spread(ProbDev P) { hash_spread_body(P, blockIdx.x); }
CHISAO_ALL_KERNEL(k_hash_spread, NT_LIN, hash_spread_body(P, pos.b))

// the (up to) three coordinates of largest spread, largest first (ties: lower index)
__device__ __forceinline__ void hash_axes_body(const ProbDev& P) {
  if (threadIdx.x != 0 || P.cnt->n_stuck0 == 0) return;
  int ax[3] = {-1, -1, -1};
  float sp[3] = {-1.f, -1.f, -1.f};
  for (int a = 0; a < P.d; ++a) {
    const float w = from_ordered_bits(P.hspread[P.dp + a]) - from_ordered_bits(P.hspread[a]);
    for (int r = 0; r < 3; ++r) {
      if (w > sp[r]) {
        for (int q = 2; q > r; --q) {
          sp[q] = sp[q - 1];
          ax[q] = ax[q - 1];
        }
        sp[r] = w;
        ax[r] = a;
        break;
      }
    }
  }
  for (int r = 0; r < 3; ++r) P.haxes[r] = ax[r];
}
__global__ void k_hash_axes(ProbDev P) { hash_axes_body(P); }
CHISAO_ALL_KERNEL(k_hash_axes, 32, hash_axes_body(P))

__device__ __forceinline__ void sample_cells(const ProbDev& P, int i, double h, long long (&c)[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int a = P.haxes[r];
    c[r] = a >= 0 ? cell_of(P.x[(size_t)i * P.dp + a], P.lo[a], h) : 0;
  }
}

// Rank key of sample i: larger for higher f, then for lower index (nonzero for any f);
// -0 is taken as +0 so that the key orders exactly as the (f desc, index asc) rank.
__device__ __forceinline__ unsigned long long rank_key(float f, int i) {
  return ((unsigned long long)ordered_bits(f == 0.f ? 0.f : f) << 32) |
         (unsigned long long)(0xFFFFFFFFu - (unsigned)i);
}

// file every stuck sample under its cell key; each cell also keeps its top-ranked member
__device__ __forceinline__ void hash_insert_body(const ProbDev& P, const StepParams& S, unsigned b) {
  const int jj = b * blockDim.x + threadIdx.x;
  if (jj >= P.cnt->n_stuck0) return;
  const double h = (double)S.eps_dup * (1.0 + 1e-6);
  long long c[3];
  const int j = P.l_stuck[jj];
  sample_cells(P, j, h, c);
  const unsigned long long key = cell_key(c[0], c[1], c[2]);
  unsigned slot = (unsigned)key & (unsigned)P.hmask;
  for (int probe = 0; probe <= P.hmask; ++probe) {     // the table has at least 2 n slots: a free one exists
    const unsigned long long prev = atomicCAS(&P.hkey[slot], HASH_EMPTY, key);
    if (prev == HASH_EMPTY || prev == key) break;
    slot = (slot + 1) & (unsigned)P.hmask;
  }
  P.hnext[jj] = atomicExch(&P.hhead[slot], jj);
  atomicMax(&P.hbest[slot], rank_key(P.f[j], j));
}
__global__ void __launch_bounds__(NT_LIN) k_hash_insert(ProbDev P, StepParams S) { hash_insert_body(P, S, blockIdx.x); }
CHISAO_ALL_KERNEL(k_hash_insert, NT_LIN, hash_insert_body(P, S, pos.b))

template <int DP>
__device__ __forceinline__ void dedup_body(const ProbDev& P, const StepParams& S, unsigned b) {
  constexpr int LPS = DP / 2;
  const Grp<LPS> g;
  const int jj = (int)(((size_t)b * blockDim.x + threadIdx.x) / LPS);
  const int Sn = P.cnt->n_stuck0;
  if (jj >= Sn) return;
  const int j = P.l_stuck[jj];
  const int c0 = 2 * g.l;
  const float2 xj = *reinterpret_cast<const float2*>(P.x + (size_t)j * DP + c0);
  const float fj = P.f[j];
  const float eps = S.eps_dup;
  const double h = (double)eps * (1.0 + 1e-6);
  long long cj[3];
  sample_cells(P, j, h, cj);
  const int na = (P.haxes[0] >= 0) + (P.haxes[1] >= 0) + (P.haxes[2] >= 0);
  int span[3];
  for (int r = 0; r < 3; ++r) span[r] = r < na ? 1 : 0;
  // the slot of a cell key, or -1 when no stuck sample is filed under it
  auto find_slot = [&](unsigned long long key) -> int {
    unsigned slot = (unsigned)key & (unsigned)P.hmask;
    for (int probe = 0; probe <= P.hmask; ++probe) {
      const unsigned long long k = P.hkey[slot];
      if (k == key) return (int)slot;
      if (k == HASH_EMPTY) return -1;
      slot = (slot + 1) & (unsigned)P.hmask;
    }
    return -1;
  };
  // does sample i rank above j and lie within eps_dup of it (the binary32 test of Eq. 4)?
  auto removes = [&](int i) -> bool {
    if (i == j) return false;
    const float fi = P.f[i];
    if (!(fi > fj || (fi == fj && i < j))) return false;
    const float2 xi = *reinterpret_cast<const float2*>(P.x + (size_t)i * DP + c0);
    return g.all(fabsf(xi.x - xj.x) < eps && fabsf(xi.y - xj.y) < eps);
  };
  bool rem = false;
  // pass 1: the top-ranked member of each neighbouring cell.  In a cluster of duplicates
  // the cluster's top is within eps_dup of most members and is the top of its own cell,
  // so most members are decided here in 27 tests.
  for (int d0 = -span[0]; d0 <= span[0] && !rem; ++d0)
    for (int d1 = -span[1]; d1 <= span[1] && !rem; ++d1)
      for (int d2 = -span[2]; d2 <= span[2] && !rem; ++d2) {
        const int slot = find_slot(cell_key(cj[0] + d0, cj[1] + d1, cj[2] + d2));
        if (slot < 0) continue;
        const unsigned long long best = P.hbest[slot];
        if (best != 0ull && removes((int)(0xFFFFFFFFu - (unsigned)(best & 0xFFFFFFFFull)))) rem = true;
      }
  // pass 2: the members of the neighbouring cells whose top ranks above j (a cell whose top
  // is j or ranks below it holds nobody above j), so a cluster's top scans no list at all
  const unsigned long long kj = rank_key(fj, j);
  for (int d0 = -span[0]; d0 <= span[0] && !rem; ++d0)
    for (int d1 = -span[1]; d1 <= span[1] && !rem; ++d1)
      for (int d2 = -span[2]; d2 <= span[2] && !rem; ++d2) {
        const int slot = find_slot(cell_key(cj[0] + d0, cj[1] + d1, cj[2] + d2));
        if (slot < 0 || P.hbest[slot] <= kj) continue;
        for (int ii = P.hhead[slot]; ii >= 0 && !rem; ii = P.hnext[ii])
          if (removes(P.l_stuck[ii])) rem = true;
      }
  if (rem && g.l == 0) atomicOr(&P.removed[j >> 5], 1u << (j & 31));
}
template <int DP>
__global__ void __launch_bounds__(128) k_dedup_impl(ProbDev P, StepParams S) { dedup_body<DP>(P, S, blockIdx.x); }
template <int DP>
CHISAO_ALL_KERNEL(k_dedup_impl, 128, dedup_body<DP>(P, S, pos.b))

// ------------------------------------------------------------ initial populations
// Uniform: x_a = lo_a + u (hi_a - lo_a), u from the TAG_SEED stream (c0 = sample,
// c1 = coordinate block of four, step 1).  Carry Tiger (reading of Sec. 5.1): the
// ray from the box centre c to an anchor, x = c + t (e * half): class i % 3 = face
// centre (axis q / 2, side q % 2, q = (i / 3) mod 2d), edge midpoint (free axis
// (i / 3) mod d, other coordinates +-1 from the sign bits), vertex (all +-1); t is
// word 0 of the stream with c1 = 0, the signs the bits of the words with c1 = 1.
constexpr unsigned TAG_SEED = 8;

__global__ void __launch_bounds__(NT_LIN) k_seed(ProbDev P, StepParams S, int method) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  const int d = P.d, dp = P.dp;
  const unsigned pq = (unsigned)P.obj.prob_index;
  float* xr = P.x + (size_t)i * dp;
  if (method == 0) {
    for (int blk = 0; blk < (d + 3) / 4; ++blk) {
      const uint4 w = rng_words(S, (unsigned)i, (unsigned)blk, TAG_SEED, 0u, 1u, pq, 0u);
      const unsigned ws[4] = {w.x, w.y, w.z, w.w};
      for (int v = 0; v < 4; ++v) {
        const int a = 4 * blk + v;
        if (a < d) xr[a] = fmaf(u01f(ws[v]), P.hi[a] - P.lo[a], P.lo[a]);
      }
    }
  } else {
    const float t = u01f(rng_words(S, (unsigned)i, 0u, TAG_SEED, 0u, 0u, pq, 0u).x);
    const uint4 w = rng_words(S, (unsigned)i, 1u, TAG_SEED, 0u, 0u, pq, 0u);
    const unsigned ws[4] = {w.x, w.y, w.z, w.w};
    const int cls = i % 3, j = i / 3;
    const int q = j % (2 * d), free_ax = j % d;
    for (int a = 0; a < d; ++a) {
      const float sgn = ((ws[a >> 5] >> (a & 31)) & 1u) ? 1.f : -1.f;
      float e;
      if (cls == 0) e = (a == q / 2) ? ((q & 1) ? 1.f : -1.f) : 0.f;
      else if (cls == 1) e = (a == free_ax) ? 0.f : sgn;
      else e = sgn;
      const float c = 0.5f * (P.lo[a] + P.hi[a]), half = 0.5f * (P.hi[a] - P.lo[a]);
      xr[a] = fmaf(t, e * half, c);
    }
  }
  for (int a = d; a < dp; ++a) xr[a] = 0.f;
}

// ------------------------------------------------------------ Phase 4
// Strategy choice and Golden Rooster bookkeeping (single thread):
//   K_lost = 0 -> none; >= rm_min unfrozen -> Repulse Monkey; else Golden
//   Rooster while enabled and some survivor exists; it disables itself after
//   gr_patience successive generations whose survivor count did not grow;
//   otherwise a uniform redraw.
__device__ __forceinline__ void reseed_decide_body(const ProbDev& P, const StepParams& S) {
  if (threadIdx.x != 0) return;
  Counters* c = P.cnt;
  const int K = c->n_free, U = c->n_unfrozen, Sv = c->n_surv;
  int mode = RESEED_NONE;
  if (K > 0) {
    mode = RESEED_UNIFORM;
    if (U >= S.rm_min) {
      mode = RESEED_RM;
    } else if (c->gr_enabled && Sv > 0) {
      if (c->gr_prev_surv >= 0) c->gr_noprog = (Sv > c->gr_prev_surv) ? 0 : c->gr_noprog + 1;
      if (c->gr_noprog >= S.gr_patience) {
        c->gr_enabled = 0;
      } else {
        mode = RESEED_GR;
        c->gr_prev_surv = Sv;
      }
    }
  }
  c->reseed_mode = mode;
}
__global__ void k_reseed_decide(ProbDev P, StepParams S) { reseed_decide_body(P, S); }
CHISAO_ALL_KERNEL(k_reseed_decide, 32, reseed_decide_body(P, S))

// Survivors ranked by (f desc, index asc): rank_j = #{i : i above j}.
__device__ __forceinline__ void gr_rank_body(const ProbDev& P, unsigned b) {
  if (P.cnt->reseed_mode != RESEED_GR) return;
  const int Sv = P.cnt->n_surv;
  const int jj = b * blockDim.x + threadIdx.x;
  if (jj >= Sv) return;
  const int j = P.l_surv[jj];
  const float fj = P.f[j];
  int r = 0;
  for (int ii = 0; ii < Sv; ++ii) {
    const int i = P.l_surv[ii];
    const float fi = P.f[i];
    r += (fi > fj || (fi == fj && i < j)) ? 1 : 0;
  }
  P.l_rank[r] = j;
}
__global__ void __launch_bounds__(NT_LIN) k_gr_rank(ProbDev P) { gr_rank_body(P, blockIdx.x); }
CHISAO_ALL_KERNEL(k_gr_rank, NT_LIN, gr_rank_body(P, pos.b))

// One Gaussian d x d matrix per Golden Rooster generation (FP64 Box-Muller on
// the GR stream, row i / column block b), its Householder QR (Golub & Van
// Loan, Algorithm 5.2.1) with Q accumulated explicitly, columns of Q flipped
// so that diag(R) > 0.  Q is written column-major to grq.
__device__ __forceinline__ void gr_qr_body(const ProbDev& P, const StepParams& S) {
  if (P.cnt->reseed_mode != RESEED_GR) return;
  extern __shared__ double sm[];
  const int d = P.d;
  double* A = sm;              // [d][d] row-major
  double* Q = sm + d * d;      // [d][d] row-major
  double* v = Q + d * d;       // [d]
  double* w = v + d;           // [d]
  __shared__ double red[NT_LIN / 32];
  __shared__ double bc;
  const unsigned cyc = (unsigned)P.cnt->cycle + 1u;
  const int nb = (d + 3) / 4;
  for (int t = threadIdx.x; t < d * nb; t += blockDim.x) {
    const int i = t / nb, b = t % nb;
    double z[4];
    normals4d(rng_words(S, (unsigned)i, (unsigned)b, TAG_GR_MAT, cyc, 0u, (unsigned)P.prob_index, 0u), z);
    for (int q = 0; q < 4; ++q)
      if (4 * b + q < d) A[i * d + 4 * b + q] = z[q];
  }
  for (int t = threadIdx.x; t < d * d; t += blockDim.x) Q[t] = (t / d == t % d) ? 1.0 : 0.0;
  __syncthreads();
  auto block_sum = [&](double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int q = 0; q < NT_LIN / 32; ++q) s += red[q];
      bc = s;
    }
    __syncthreads();
    const double r = bc;
    __syncthreads();
    return r;
  };
  for (int j = 0; j + 1 < d; ++j) {
    const int len = d - j;
    const double xt = threadIdx.x < len ? A[(j + threadIdx.x) * d + j] : 0.0;
    const double alpha = sqrt(block_sum(xt * xt));
    if (alpha == 0.0) continue;
    const double x0 = A[j * d + j];
    double vt = xt;
    if (threadIdx.x == 0) vt += copysign(alpha, x0);
    const double vn = sqrt(block_sum(threadIdx.x < len ? vt * vt : 0.0));
    if (threadIdx.x < len) v[threadIdx.x] = vt / vn;
    __syncthreads();
    // A[j:, :] -= 2 v (v^T A[j:, :])
    for (int c = threadIdx.x; c < d; c += blockDim.x) {
      double s = 0.0;
      for (int r = 0; r < len; ++r) s += v[r] * A[(j + r) * d + c];
      w[c] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < len * d; t += blockDim.x) {
      const int r = t / d, c = t % d;
      A[(j + r) * d + c] -= 2.0 * v[r] * w[c];
    }
    __syncthreads();
    // Q[:, j:] -= 2 (Q[:, j:] v) v^T
    for (int r = threadIdx.x; r < d; r += blockDim.x) {
      double s = 0.0;
      for (int k = 0; k < len; ++k) s += Q[r * d + j + k] * v[k];
      w[r] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < d * len; t += blockDim.x) {
      const int r = t / len, k = t % len;
      Q[r * d + j + k] -= 2.0 * w[r] * v[k];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < d * d; t += blockDim.x) {
    const int r = t / d, c = t % d;                       // Q[r][c] -> column-major
    const double sg = A[c * d + c] < 0.0 ? -1.0 : 1.0;
    P.grq[c * d + r] = sg * Q[r * d + c];
  }
}
__global__ void __launch_bounds__(NT_LIN) k_gr_qr(ProbDev P, StepParams S) { gr_qr_body(P, S); }
CHISAO_ALL_KERNEL(k_gr_qr, NT_LIN, gr_qr_body(P, S))

// Largest t >= 0 keeping p + t u inside the box, reduced over the group.
template <int LPS>
__device__ __forceinline__ float ray_exit(float p0, float p1, float u0, float u1, float lo0, float lo1, float hi0,
                                          float hi1, bool v0, bool v1, const Grp<LPS>& g) {
  float t = CUDART_INF_F;
  if (v0 && u0 > 0.f) t = fminf(t, (hi0 - p0) / u0);
  if (v0 && u0 < 0.f) t = fminf(t, (lo0 - p0) / u0);
  if (v1 && u1 > 0.f) t = fminf(t, (hi1 - p1) / u1);
  if (v1 && u1 < 0.f) t = fminf(t, (lo1 - p1) / u1);
#pragma unroll
  for (int o = LPS / 2; o > 0; o >>= 1) t = fminf(t, __shfl_xor_sync(g.mask, t, o, LPS));
  if (!(t < CUDART_INF_F)) t = 0.f;
  return fmaxf(t, 0.f);
}

// Fill free slot r (r-th removed sample in index order) by the chosen strategy.
template <int DP>
__device__ __forceinline__ void reseed_body(const ProbDev& P, const StepParams& S, unsigned b) {
  constexpr int LPS = DP / 2;
  const Grp<LPS> g;
  const int mode = P.cnt->reseed_mode;
  const int K = P.cnt->n_free;
  const int r = (int)(((size_t)b * blockDim.x + threadIdx.x) / LPS);
  if (mode == RESEED_NONE || r >= K) return;
  const int slot = P.l_free[r];
  const int d = P.d, j0 = 2 * g.l;
  const bool v0 = j0 < d, v1 = j0 + 1 < d;
  const unsigned cyc = (unsigned)P.cnt->cycle + 1u, pid = (unsigned)P.prob_index;
  const float lo0 = P.lo[j0], lo1 = P.lo[j0 + 1], hi0 = P.hi[j0], hi1 = P.hi[j0 + 1];
  float c0 = 0.f, c1 = 0.f;
  if (mode == RESEED_RM || mode == RESEED_GR) {
    float u0, u1, p0, p1, uu;
    if (mode == RESEED_RM) {
      const uint4 w = rng_words(S, (unsigned)r, 0u, TAG_RM, cyc, 0u, pid, 0u);
      const unsigned U = (unsigned)P.cnt->n_unfrozen;
      const int parent = P.l_unf[(unsigned)(((unsigned long long)w.x * U) >> 32)];
      float z[2];
      normals_lane<2>(S, (unsigned)r, g.l, TAG_RM_DIR, cyc, 0u, pid, 0u, z);
      const float z0 = v0 ? z[0] : 0.f, z1 = v1 ? z[1] : 0.f;
      const float nz = sqrtf(g.sum(z0 * z0 + z1 * z1));
      u0 = z0 / nz;
      u1 = z1 / nz;
      const float2 pv = *reinterpret_cast<const float2*>(P.x + (size_t)parent * DP + j0);
      p0 = pv.x;
      p1 = pv.y;
      uu = u01f(w.y);
    } else {
      const int Sv = P.cnt->n_surv;
      const int peak = P.l_rank[r % Sv];
      const int col = (r / Sv) % d;
      const float sg = ((r / (Sv * d)) % 2 == 0) ? 1.f : -1.f;
      u0 = v0 ? sg * (float)P.grq[col * d + j0] : 0.f;
      u1 = v1 ? sg * (float)P.grq[col * d + j0 + 1] : 0.f;
      const float2 pv = *reinterpret_cast<const float2*>(P.x + (size_t)peak * DP + j0);
      p0 = pv.x;
      p1 = pv.y;
      const uint4 w = rng_words(S, (unsigned)r, 0u, TAG_GR_T, cyc, 0u, pid, 0u);
      uu = u01f(w.x);
    }
    const float t = uu * ray_exit<LPS>(p0, p1, u0, u1, lo0, lo1, hi0, hi1, v0, v1, g);
    c0 = v0 ? clampf(fmaf(t, u0, p0), lo0, hi0) : 0.f;
    c1 = v1 ? clampf(fmaf(t, u1, p1), lo1, hi1) : 0.f;
  } else {
    const uint4 w = rng_words(S, (unsigned)r, (unsigned)(g.l >> 1), TAG_UNIFORM, cyc, 0u, pid, 0u);
    const float a = u01f((g.l & 1) ? w.z : w.x), b = u01f((g.l & 1) ? w.w : w.y);
    c0 = v0 ? fmaf(a, hi0 - lo0, lo0) : 0.f;
    c1 = v1 ? fmaf(b, hi1 - lo1, lo1) : 0.f;
  }
  *reinterpret_cast<float2*>(P.x + (size_t)slot * DP + j0) = make_float2(c0, c1);
  if (g.l == 0) P.hlen[slot] = 0;
}
template <int DP>
__global__ void __launch_bounds__(128) k_reseed(ProbDev P, StepParams S) { reseed_body<DP>(P, S, blockIdx.x); }
template <int DP>
CHISAO_ALL_KERNEL(k_reseed, 128, reseed_body<DP>(P, S, pos.b))

// ------------------------------------------------------------ Phase 5/6 scales
// Fixed-order sum of the per-block partials, then
//   s = sqrt(mean_j var_j), sigma = c_sigma s, g_rms = sqrt(sum g^2 / (U d)),
//   alpha = alpha_scale s / max(g_rms, 1e-30)   (fixed values when supplied).
// 1024 threads = 8 row groups x 128 columns: row group q sums the partial
// blocks b = q (mod 8) in double-single arithmetic (on the FP32 pipe: one SM's
// FP64 rate would make this single block the slowest kernel of the cycle),
// then the 8 row-group sums are added in order q = 0..7 -- a fixed order, so
// the result does not depend on timing -- and converted to FP64.
constexpr int FIN_NT = 1024, FIN_RG = 8, FIN_COLS = FIN_NT / FIN_RG;
__device__ __forceinline__ void finalize_body(const ProbDev& P, const StepParams& S, int nblocks, int which) {
  const int W = 2 * P.dp + 2;
  extern __shared__ double tot[];                   // [W]
  __shared__ float2 part[FIN_RG][FIN_COLS];
  const int q = threadIdx.x / FIN_COLS, cl = threadIdx.x % FIN_COLS;
  for (int c0 = 0; c0 < W; c0 += FIN_COLS) {
    const int col = c0 + cl;
    float h = 0.f, l = 0.f;
    if (col < W) {
      // FIN_PF partials in flight per thread (the single block is bound by load latency),
      // added in the same order b = q, q + FIN_RG, ...
      constexpr int FIN_PF = 16;
      for (int b0 = q; b0 < nblocks; b0 += FIN_PF * FIN_RG) {
        float2 v[FIN_PF];
#pragma unroll
        for (int u = 0; u < FIN_PF; ++u) {
          const int b = b0 + u * FIN_RG;
          v[u] = b < nblocks ? P.partials[(size_t)b * W + col] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < FIN_PF; ++u)
          if (b0 + u * FIN_RG < nblocks) ff_add(h, l, v[u].x, v[u].y);
      }
    }
    part[q][cl] = make_float2(h, l);
    __syncthreads();
    if (q == 0 && col < W) {
      float sh = 0.f, sl = 0.f;
      for (int r = 0; r < FIN_RG; ++r) ff_add(sh, sl, part[r][cl].x, part[r][cl].y);
      tot[col] = (double)sh + (double)sl;
    }
    __syncthreads();
  }
  // per-coordinate variances by one thread each (warp 0 holds d <= 64 lanes' worth in two passes),
  // summed in a fixed butterfly order
  const double U = tot[2 * P.dp + 1];
  if (threadIdx.x < 32) {
    const double invU = U > 0.0 ? 1.0 / U : 0.0;
    double v = 0.0;
    for (int j = threadIdx.x; j < P.d; j += 32) {
      const double m = tot[j] * invU;
      v += fmax(tot[P.dp + j] * invU - m * m, 0.0);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) tot[0] = v;                 // column 0 is no longer needed
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Counters* c = P.cnt;
    if (U <= 0.0) {
      c->sc_count = 0;
      c->sc_sigma = 0.f;
      c->sc_alpha = 0.f;
      return;
    }
    const double vs = tot[0];
    const double s = sqrt(vs / P.d);
    const double grms = sqrt(tot[2 * P.dp] / (U * P.d));
    const double sigma = S.sigma_fixed > 0.f ? (double)S.sigma_fixed : (double)S.c_sigma * s;
    const double alpha = S.alpha_fixed > 0.f ? (double)S.alpha_fixed : (double)S.alpha_scale * s / fmax(grms, 1e-30);
    c->sc_count = (int)U;
    c->sc_sigma = (float)sigma;
    c->sc_alpha = (float)alpha;
    if (which == 0) {
      c->sigma = (float)sigma;
      c->alpha_hlc = (float)alpha;
    } else {
      c->alpha_anti = (float)alpha;
    }
  }
}

__global__ void __launch_bounds__(FIN_NT) k_finalize_scales(ProbDev P, StepParams S, int nblocks, int which) {
  finalize_body(P, S, nblocks, which);
}

// One block per problem of a group; T is the group's scale-pass table.
__global__ void __launch_bounds__(FIN_NT) k_finalize_grp(GroupTab T, int which) {
  const int q = blockIdx.x;
  finalize_body(T.probs[q], T.sps[q], T.blk_count[q], which);
}

// ------------------------------------------------------------ modes gather
__global__ void __launch_bounds__(NT_LIN) k_gather_modes(ProbDev P, float* xo, float* fo) {
  const long long total = (long long)P.cnt->n_surv * P.d;     // up to 2^27 x 64: 64-bit
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(t / P.d), j = (int)(t % P.d);
    const int i = P.l_surv[r];
    xo[t] = P.x[(size_t)i * P.dp + j];
    if (j == 0) fo[r] = P.f[i];
  }
}

// ------------------------------------------------------------ host launchers
static unsigned lin_blocks(long long n, int nt) {
  long long b = (n + nt - 1) / nt;
  if (b < 1) b = 1;
  return (unsigned)b;
}

cudaError_t launch_cycle_begin(const ProbDev& P, cudaStream_t st) {
  k_cycle_begin<<<lin_blocks(P.nwords, NT_LIN), NT_LIN, 0, st>>>(P);
  return cudaGetLastError();
}
cudaError_t launch_cycle_end(const ProbDev& P, cudaStream_t st) {
  k_cycle_end<<<1, 32, 0, st>>>(P);
  return cudaGetLastError();
}
cudaError_t launch_set_cycle(const ProbDev& P, int completed, cudaStream_t st) {
  k_set_cycle<<<1, 32, 0, st>>>(P, completed);
  return cudaGetLastError();
}

cudaError_t launch_compact_stuck(const ProbDev& P, cudaStream_t st) {
  k_compact_stuck<<<1, NT_ONE, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_lists(const ProbDev& P, cudaStream_t st) {
  k_compact_dedup<<<1, NT_ONE, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_freeze(const ProbDev& P, const StepParams& S, cudaStream_t st) {
  unsigned nb = lin_blocks(P.n, NT_LIN);
  k_fmax<<<nb < 1216 ? nb : 1216, NT_LIN, 0, st>>>(P);
  k_freeze<<<nb, NT_LIN, 0, st>>>(P, S);
  k_compact_stuck<<<1, NT_ONE, 0, st>>>(P);
  return cudaGetLastError();
}

template <int DP>
static void dedup_dp(const ProbDev& P, const StepParams& S, cudaStream_t st) {
  const long long th = (long long)P.n * (DP / 2);
  k_dedup_impl<DP><<<lin_blocks(th, 128), 128, 0, st>>>(P, S);
}

cudaError_t launch_seed(const ProbDev& P, const StepParams& S, int method, cudaStream_t st) {
  k_seed<<<lin_blocks(P.n, NT_LIN), NT_LIN, 0, st>>>(P, S, method);
  return cudaGetLastError();
}

cudaError_t launch_dedup(const ProbDev& P, const StepParams& S, cudaStream_t st) {
  cudaMemsetAsync(P.removed, 0, sizeof(uint32_t) * P.nwords, st);
  const long long slots = (long long)P.hmask + 1;
  k_hash_clear<<<(unsigned)std::min<long long>(lin_blocks(slots, NT_LIN), 1024), NT_LIN, 0, st>>>(P);
  k_hash_spread<<<lin_blocks((long long)P.n * P.d, NT_LIN), NT_LIN, 0, st>>>(P);
  k_hash_axes<<<1, 32, 0, st>>>(P);
  k_hash_insert<<<lin_blocks(P.n, NT_LIN), NT_LIN, 0, st>>>(P, S);
  switch (P.dp) {
    case 4: dedup_dp<4>(P, S, st); break;
    case 8: dedup_dp<8>(P, S, st); break;
    case 16: dedup_dp<16>(P, S, st); break;
    case 32: dedup_dp<32>(P, S, st); break;
    case 64: dedup_dp<64>(P, S, st); break;
    default: return cudaErrorInvalidValue;
  }
  k_compact_dedup<<<1, NT_ONE, 0, st>>>(P);
  return cudaGetLastError();
}

size_t gr_qr_smem(int d) { return sizeof(double) * (2 * (size_t)d * d + 2 * (size_t)d); }

cudaError_t prepare_kernel_attributes() {
  const cudaError_t e = cudaFuncSetAttribute(k_gr_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gr_qr_smem(64));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_gr_qr_all, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gr_qr_smem(64));
}

template <int DP>
static void reseed_dp(const ProbDev& P, const StepParams& S, cudaStream_t st) {
  const long long th = (long long)P.n * (DP / 2);
  k_reseed<DP><<<lin_blocks(th, 128), 128, 0, st>>>(P, S);
}

cudaError_t launch_reseed(const ProbDev& P, const StepParams& S, cudaStream_t st) {
  k_reseed_decide<<<1, 32, 0, st>>>(P, S);
  k_gr_rank<<<lin_blocks(P.n, NT_LIN), NT_LIN, 0, st>>>(P);
  k_gr_qr<<<1, NT_LIN, gr_qr_smem(P.d), st>>>(P, S);
  switch (P.dp) {
    case 4: reseed_dp<4>(P, S, st); break;
    case 8: reseed_dp<8>(P, S, st); break;
    case 16: reseed_dp<16>(P, S, st); break;
    case 32: reseed_dp<32>(P, S, st); break;
    case 64: reseed_dp<64>(P, S, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------ launches over all problems
// Each table lists the problems (or, for the kernels templated on the padded dimension,
// the problems of one dp) with the block count their own launch would use, so every
// problem runs the same blocks as on its own.
static int dp_slot(int dp) {
  int k = 0;
  while ((4 << k) < dp) ++k;
  return k;
}

cudaError_t build_all_tabs(const std::vector<ProbDev>& pd, const std::vector<StepParams>& sp, void** mem,
                           AllTabs* out) {
  const int nq = (int)pd.size();
  std::vector<std::vector<int>> firsts;              // one per table, in the order of `tabs` below
  std::vector<std::vector<int>> qidx;
  auto table = [&](auto blocks_of, const std::vector<int>& members) {
    std::vector<int> f(1, 0);
    for (int q : members) f.push_back(f.back() + (int)blocks_of(pd[q]));
    firsts.push_back(f);
    qidx.push_back(members);
  };
  std::vector<int> all(nq);
  for (int q = 0; q < nq; ++q) all[q] = q;
  table([](const ProbDev& P) { return lin_blocks(P.nwords, NT_LIN); }, all);                              // begin
  table([](const ProbDev& P) { const unsigned nb = lin_blocks(P.n, NT_LIN); return nb < 1216 ? nb : 1216u; }, all);
  table([](const ProbDev& P) { return lin_blocks(P.n, NT_LIN); }, all);                                   // lin
  table([](const ProbDev&) { return 1u; }, all);                                                          // one
  table([](const ProbDev& P) {
    return (unsigned)std::min<long long>(lin_blocks((long long)P.hmask + 1, NT_LIN), 1024); }, all);      // hclear
  table([](const ProbDev& P) { return lin_blocks((long long)P.n * P.d, NT_LIN); }, all);                  // hspread
  for (int k = 0; k < 5; ++k) {
    std::vector<int> m;
    for (int q = 0; q < nq; ++q)
      if (dp_slot(pd[q].dp) == k) m.push_back(q);
    table([](const ProbDev& P) { return lin_blocks((long long)P.n * (P.dp / 2), 128); }, m);              // dp2
  }
  size_t total = 0;
  auto up = [](size_t o) { return (o + 255) / 256 * 256; };
  const size_t off_pd = total;
  total = up(total + nq * sizeof(ProbDev));
  const size_t off_sp = total;
  total = up(total + nq * sizeof(StepParams));
  std::vector<size_t> off_f(firsts.size()), off_q(firsts.size());
  for (size_t t = 0; t < firsts.size(); ++t) {
    off_f[t] = total;
    total = up(total + firsts[t].size() * sizeof(int));
    off_q[t] = total;
    total = up(total + std::max<size_t>(qidx[t].size(), 1) * sizeof(int));
  }
  cudaError_t e;
  if ((e = cudaMalloc(mem, total)) != cudaSuccess) return e;
  char* base = static_cast<char*>(*mem);
  if ((e = cudaMemcpy(base + off_pd, pd.data(), nq * sizeof(ProbDev), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
  if ((e = cudaMemcpy(base + off_sp, sp.data(), nq * sizeof(StepParams), cudaMemcpyHostToDevice)) != cudaSuccess)
    return e;
  AllTab* tabs[] = {&out->begin, &out->fmax, &out->lin, &out->one, &out->hclear, &out->hspread, &out->dp2[0],
                    &out->dp2[1], &out->dp2[2], &out->dp2[3], &out->dp2[4]};
  unsigned* blocks[] = {&out->nb_begin, &out->nb_fmax, &out->nb_lin, &out->nb_one, &out->nb_hclear, &out->nb_hspread,
                        &out->nb_dp2[0], &out->nb_dp2[1], &out->nb_dp2[2], &out->nb_dp2[3], &out->nb_dp2[4]};
  for (size_t t = 0; t < firsts.size(); ++t) {
    if ((e = cudaMemcpy(base + off_f[t], firsts[t].data(), firsts[t].size() * sizeof(int),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
    if (!qidx[t].empty() && (e = cudaMemcpy(base + off_q[t], qidx[t].data(), qidx[t].size() * sizeof(int),
                                            cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
    AllTab& T = *tabs[t];
    T.probs = reinterpret_cast<const ProbDev*>(base + off_pd);
    T.sps = reinterpret_cast<const StepParams*>(base + off_sp);
    T.first = reinterpret_cast<const int*>(base + off_f[t]);
    T.qidx = t >= 6 ? reinterpret_cast<const int*>(base + off_q[t]) : nullptr;
    T.n = (int)qidx[t].size();
    *blocks[t] = (unsigned)firsts[t].back();
  }
  int dmax = 1;
  for (const ProbDev& P : pd) dmax = std::max(dmax, P.d);
  out->qr_smem = gr_qr_smem(dmax);
  return cudaSuccess;
}

cudaError_t launch_cycle_begin_all(const AllTabs& A, cudaStream_t st) {
  k_cycle_begin_all<<<A.nb_begin, NT_LIN, 0, st>>>(A.begin);
  return cudaGetLastError();
}
cudaError_t launch_cycle_end_all(const AllTabs& A, cudaStream_t st) {
  k_cycle_end_all<<<A.nb_one, 32, 0, st>>>(A.one);
  return cudaGetLastError();
}
cudaError_t launch_freeze_all(const AllTabs& A, cudaStream_t st) {
  k_fmax_all<<<A.nb_fmax, NT_LIN, 0, st>>>(A.fmax);
  k_freeze_all<<<A.nb_lin, NT_LIN, 0, st>>>(A.lin);
  k_compact_stuck_all<<<A.nb_one, NT_ONE, 0, st>>>(A.one);
  return cudaGetLastError();
}
template <int DP>
static void dedup_all_dp(const AllTabs& A, int k, cudaStream_t st) {
  if (A.dp2[k].n > 0) k_dedup_impl_all<DP><<<A.nb_dp2[k], 128, 0, st>>>(A.dp2[k]);
}
template <int DP>
static void reseed_all_dp(const AllTabs& A, int k, cudaStream_t st) {
  if (A.dp2[k].n > 0) k_reseed_all<DP><<<A.nb_dp2[k], 128, 0, st>>>(A.dp2[k]);
}
// Phase 3 of every problem (the masks were cleared at the cycle's start).
cudaError_t launch_dedup_all(const AllTabs& A, cudaStream_t st) {
  k_hash_clear_all<<<A.nb_hclear, NT_LIN, 0, st>>>(A.hclear);
  k_hash_spread_all<<<A.nb_hspread, NT_LIN, 0, st>>>(A.hspread);
  k_hash_axes_all<<<A.nb_one, 32, 0, st>>>(A.one);
  k_hash_insert_all<<<A.nb_lin, NT_LIN, 0, st>>>(A.lin);
  dedup_all_dp<4>(A, 0, st);
  dedup_all_dp<8>(A, 1, st);
  dedup_all_dp<16>(A, 2, st);
  dedup_all_dp<32>(A, 3, st);
  dedup_all_dp<64>(A, 4, st);
  k_compact_dedup_all<<<A.nb_one, NT_ONE, 0, st>>>(A.one);
  return cudaGetLastError();
}
cudaError_t launch_reseed_all(const AllTabs& A, cudaStream_t st) {
  k_reseed_decide_all<<<A.nb_one, 32, 0, st>>>(A.one);
  k_gr_rank_all<<<A.nb_lin, NT_LIN, 0, st>>>(A.lin);
  k_gr_qr_all<<<A.nb_one, NT_LIN, A.qr_smem, st>>>(A.one);
  reseed_all_dp<4>(A, 0, st);
  reseed_all_dp<8>(A, 1, st);
  reseed_all_dp<16>(A, 2, st);
  reseed_all_dp<32>(A, 3, st);
  reseed_all_dp<64>(A, 4, st);
  return cudaGetLastError();
}

int scale_blocks(const ProbDev& P) {
  const int gpb = 256 / (P.dp / 4);          // groups per block of k_scales (4 coordinates per lane)
  long long nb = (P.n + gpb - 1) / gpb;
  if (nb > 608) nb = 608;
  if (nb > P.max_part_blocks) nb = P.max_part_blocks;
  if (nb < 1) nb = 1;
  return (int)nb;
}

cudaError_t launch_finalize_grp(const GroupTab& T, int members, int dp, int which, cudaStream_t st) {
  k_finalize_grp<<<(unsigned)members, FIN_NT, sizeof(double) * (2 * dp + 2), st>>>(T, which);
  return cudaGetLastError();
}

cudaError_t launch_finalize_scales(const ProbDev& P, const StepParams& S, int which, cudaStream_t st) {
  k_finalize_scales<<<1, FIN_NT, sizeof(double) * (2 * P.dp + 2), st>>>(P, S, scale_blocks(P), which);
  return cudaGetLastError();
}

cudaError_t launch_gather_modes(const ProbDev& P, float* xo, float* fo, cudaStream_t st) {
  k_gather_modes<<<lin_blocks((long long)P.n * P.d, NT_LIN) < 2048 ? lin_blocks((long long)P.n * P.d, NT_LIN) : 2048,
                   NT_LIN, 0, st>>>(P, xo, fo);
  return cudaGetLastError();
}

}  // namespace chisao

// C ABI of the ChiSao population step (declared in include/chisao.h).
//
// Host responsibilities only: argument validation, the device-memory layout,
// FP64 preparation of the objective parameters (mixture constants, triangular
// inverses, A = Q^T diag(lam) Q), enqueueing the per-cycle kernel sequence of
// Algorithm 1 and capturing it in CUDA graphs.  Every phase itself runs in the
// kernels of phase_kernels.cu and obj_kernels.cuh.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/chisao.h"
#include "host.h"

using namespace chisao;

namespace {

constexpr int MAX_PART_BLOCKS = 608;
constexpr size_t ALIGN = 256;
constexpr long long MAX_N = 1ll << 27;

struct ProbHost {
  int d = 0, dp = 0, kind = 0, K = 0;
  long long n = 0;
  ProbDev dev{};
  StepParams sp{};
  float* gather_x = nullptr;
  float* gather_f = nullptr;
  uint8_t* tc_weights = nullptr;     // tensor-core operand tiles (full-covariance mixtures)
  float* tc_part = nullptr;          // partial results of component-split launches
  int* tc_ticket = nullptr;          // their per-tile arrival counters (zero between launches)
  bool tc = false;                   // the cycle runs around a batched evaluator (tensor cores or external)
  ExtBuf ext{};                      // its buffers
  chisao_batch_eval_fn ext_eval = nullptr;   // CHISAO_OBJ_EXTERNAL: the caller's evaluator
  void* ext_user = nullptr;
  mutable int32_t ext_status = 0;    // its last non-zero return value, for the error message
};

// Bump allocator over the arena; with a null base it only measures.
struct Bump {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + ALIGN - 1) / ALIGN * ALIGN;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Problems of one objective kind and padded dimension whose Phases 1, 5 and 6 run as
// one grouped launch each (exact gradients, several problems in the context).
struct Group {
  int kind = 0, dp = 0;
  int tile = 0;                      // tile shape of the diagonal mixture's kernels (the tuner's choice)
  std::vector<int> members;          // problem indices
  unsigned blocks = 0;               // blocks of one per-sample launch over all members
  unsigned blocks_sc = 0;            // blocks of the grouped scale pass
  GroupTab tab{}, tab_sc{};          // device tables (one allocation, `mem`)
  void* mem = nullptr;
};

int pad_dim(int d) {
  int dp = 4;
  while (dp < d) dp <<= 1;
  return dp;
}

}  // namespace

struct chisao_ctx {
  chisao_params params{};
  std::vector<ProbHost> probs;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  bool own_arena = false;
  int cycles_done = 0;
  cudaGraphExec_t g_mid = nullptr, g_last = nullptr;
  // several problems: each cycle forks onto branch streams (problems spread over them,
  // largest first, to the least-loaded branch) and joins back, so a captured cycle is a
  // graph whose per-problem chains run concurrently
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> joined;
  cudaEvent_t forked = nullptr;
  std::vector<int> branch_of;              // problem -> branch
  std::vector<Group> groups;               // grouped Phase 1 / 5 / 6 launches (empty: per problem)
  bool groups_enabled = true;              // chisao_autotune's choice
  AllTabs all{};                           // grouped launches of the per-problem steps
  void* all_mem = nullptr;
  std::string err;
};

namespace {

chisao_status fail(chisao_ctx* c, chisao_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

chisao_status cuda_fail(chisao_ctx* c, cudaError_t e, const char* what) {
  for (const ProbHost& ph : c->probs)
    if (ph.ext_status != 0) {
      const int32_t r = ph.ext_status;
      ph.ext_status = 0;
      return fail(c, CHISAO_ERR_CUDA, std::string(what) + ": the external objective's evaluator returned " +
                                          std::to_string(r));
    }
  return fail(c, CHISAO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);    \
  } while (0)

chisao_status validate_params(const chisao_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return CHISAO_ERR_ARG; }
  if (p->n_osc < 1) { why = "n_osc must be >= 1"; return CHISAO_ERR_ARG; }
  if (p->n_conv < 0 || p->n_anti < 0 || p->n_cloud < 0) { why = "step counts must be >= 0"; return CHISAO_ERR_ARG; }
  if (p->M < 1 || p->M > 65535) { why = "M must be in [1, 65535]"; return CHISAO_ERR_ARG; }
  if (p->m < 1 || p->m > CHISAO_MAX_MEMORY) { why = "m must be in [1, 10]"; return CHISAO_ERR_ARG; }
  if (p->T_ls < 1 || p->T_ls > 126) { why = "T_ls must be in [1, 126]"; return CHISAO_ERR_ARG; }
  if (p->n_cloud > 255) { why = "n_cloud must be <= 255"; return CHISAO_ERR_ARG; }
  if (p->grad_mode < 0 || p->grad_mode > 3) { why = "unknown grad_mode"; return CHISAO_ERR_ARG; }
  if (p->n_refine < 0) { why = "n_refine must be >= 0"; return CHISAO_ERR_ARG; }
  if (p->hlc_value_only != 0 && p->hlc_value_only != 1) { why = "hlc_value_only must be 0 or 1"; return CHISAO_ERR_ARG; }
  if (p->hlc_value_only && p->grad_mode == CHISAO_GRAD_ADJOINT_TC) {
    why = "the value-only smoothing estimator is not available with the tensor-core mode";
    return CHISAO_ERR_ARG;
  }
  if (!(p->eps_grad > 0) || !(p->eps_dup > 0)) { why = "eps_grad and eps_dup must be > 0"; return CHISAO_ERR_ARG; }
  if (!(p->delta > 0 && p->delta < 1)) { why = "delta must be in (0, 1)"; return CHISAO_ERR_ARG; }
  if (!(p->h > 0) || !(p->h_rel > 0) || !(p->c1 > 0 && p->c1 < 1)) { why = "h, h_rel > 0 and c1 in (0,1) required"; return CHISAO_ERR_ARG; }
  if (!std::isfinite(p->mu) || !std::isfinite(p->alpha) || !std::isfinite(p->sigma)) { why = "mu, alpha, sigma must be finite"; return CHISAO_ERR_ARG; }
  if (p->rm_min_unfrozen < 1 || p->gr_patience < 1) { why = "rm_min_unfrozen and gr_patience must be >= 1"; return CHISAO_ERR_ARG; }
  return CHISAO_OK;
}

bool is_bench_kind(int kind) { return kind >= CHISAO_OBJ_RASTRIGIN && kind <= CHISAO_OBJ_BUKIN6; }

chisao_status validate_problem(const chisao_problem* pr, std::string& why) {
  if (pr->d < 1 || pr->d > CHISAO_MAX_DIM) { why = "d must be in [1, 64]"; return CHISAO_ERR_ARG; }
  if (pr->n < 1 || pr->n > MAX_N) { why = "n must be in [1, 2^27]"; return CHISAO_ERR_ARG; }
  if (!pr->lo || !pr->hi || !pr->x0) { why = "lo, hi and x0 are required"; return CHISAO_ERR_ARG; }
  for (int j = 0; j < pr->d; ++j)
    if (!(std::isfinite(pr->lo[j]) && std::isfinite(pr->hi[j]) && pr->lo[j] < pr->hi[j])) {
      why = "box needs finite lo < hi";
      return CHISAO_ERR_ARG;
    }
  const chisao_objective& o = pr->objective;
  if (!(std::isfinite(o.noise_sigma) && o.noise_sigma >= 0)) { why = "noise_sigma must be finite and >= 0"; return CHISAO_ERR_ARG; }
  if (o.kind == CHISAO_OBJ_MIXTURE_DIAG || o.kind == CHISAO_OBJ_MIXTURE_FULL) {
    if (o.n_comp < 1 || o.n_comp > 65536) { why = "mixture needs 1 <= K <= 65536"; return CHISAO_ERR_ARG; }
    if (!o.weights || !o.means) { why = "mixture needs weights and means"; return CHISAO_ERR_ARG; }
    for (int k = 0; k < o.n_comp; ++k)
      if (!(o.weights[k] > 0)) { why = "mixture weights must be > 0"; return CHISAO_ERR_ARG; }
    if (o.kind == CHISAO_OBJ_MIXTURE_DIAG) {
      if (!o.sigmas) { why = "diagonal mixture needs sigmas"; return CHISAO_ERR_ARG; }
      for (long long t = 0; t < (long long)o.n_comp * pr->d; ++t)
        if (!(o.sigmas[t] > 0)) { why = "sigmas must be > 0"; return CHISAO_ERR_ARG; }
    } else {
      if (!o.chol) { why = "full mixture needs chol"; return CHISAO_ERR_ARG; }
      for (int k = 0; k < o.n_comp; ++k)
        for (int j = 0; j < pr->d; ++j)
          if (!(o.chol[((size_t)k * pr->d + j) * pr->d + j] > 0)) { why = "Cholesky diagonals must be > 0"; return CHISAO_ERR_ARG; }
    }
  } else if (o.kind == CHISAO_OBJ_QUADRATIC) {
    if (!o.center || !o.Q || !o.lam) { why = "quadratic needs center, Q and lam"; return CHISAO_ERR_ARG; }
  } else if (is_bench_kind(o.kind)) {
    if (o.kind == CHISAO_OBJ_BUKIN6 && pr->d != 2) { why = "Bukin N.6 needs d = 2"; return CHISAO_ERR_ARG; }
  } else if (o.kind == CHISAO_OBJ_EXTERNAL) {
    if (!o.eval) { why = "an external objective needs its evaluator"; return CHISAO_ERR_ARG; }
    if (o.noise_sigma != 0) { why = "an external objective adds its own noise (noise_sigma must be 0)"; return CHISAO_ERR_ARG; }
  } else {
    why = "unknown objective kind";
    return CHISAO_ERR_ARG;
  }
  return CHISAO_OK;
}

// Objective kind against the gradient mode and the Phase 5 variant.
chisao_status validate_mode(const chisao_problem* pr, const chisao_params* p, std::string& why) {
  const int kind = pr->objective.kind;
  if (p->grad_mode == CHISAO_GRAD_ADJOINT_TC && kind != CHISAO_OBJ_MIXTURE_FULL) {
    why = "the tensor-core mode needs full-covariance mixtures";
    return CHISAO_ERR_ARG;
  }
  if (kind == CHISAO_OBJ_EXTERNAL && (p->grad_mode != CHISAO_GRAD_ADJOINT || p->hlc_value_only)) {
    why = "an external objective supplies exact gradients: grad_mode ADJOINT, hlc_value_only 0";
    return CHISAO_ERR_ARG;
  }
  return CHISAO_OK;
}

// The quadratic's symmetric A as the blocks its binary32 product reads (objectives.cuh:
// sym_times): with L = dp / 4 lanes per sample, lane l at step k = 0 .. L/2 reads the 4 x 4
// block A[l][(l + k) mod L] as four float4 columns; entry ((k * 4 + c) * L + l) * 4 + v holds
// A[4 l + v][4 ((l + k) mod L) + c], so the lanes of a group read one contiguous line per
// (k, c).  The blocks with 0 < k < L/2 also stand for their transposes.
size_t quad_sym_elems(int dp) { return (size_t)(dp / 8 + 1) * 4 * dp; }

void quad_sym_table(const std::vector<double>& A, int dp, double* out) {
  const int L = dp / 4;
  for (int k = 0; k <= L / 2; ++k)
    for (int c = 0; c < 4; ++c)
      for (int l = 0; l < L; ++l)
        for (int v = 0; v < 4; ++v)
          out[(((size_t)k * 4 + c) * L + l) * 4 + v] = A[(size_t)(4 * l + v) * dp + 4 * ((l + k) % L) + c];
}

size_t obj_elems(const chisao_problem& pr, int dp, size_t* n0, size_t* n1, size_t* n2, size_t* n3) {
  const size_t K = (size_t)pr.objective.n_comp;
  switch (pr.objective.kind) {
    case CHISAO_OBJ_MIXTURE_DIAG: *n0 = K * dp; *n1 = K * dp; *n2 = K; *n3 = 0; break;
    case CHISAO_OBJ_MIXTURE_FULL: *n0 = K * dp; *n1 = K * dp * dp; *n2 = K; *n3 = K * dp * dp; break;
    case CHISAO_OBJ_QUADRATIC: *n0 = dp; *n1 = (size_t)dp * dp; *n2 = quad_sym_elems(dp); *n3 = 0; break;
    default: *n0 = *n1 = *n2 = *n3 = 0; break;                 // benchmark functions: no constants
  }
  return *n0 + *n1 + *n2 + *n3;
}

// Carve one problem's buffers (measure-only when b.base is null).
void layout_problem(Bump& b, const chisao_problem& pr, const chisao_params& prm, ProbHost& ph) {
  const int d = pr.d, dp = pad_dim(d);
  const size_t n = (size_t)pr.n, nw = (n + 31) / 32;
  ProbDev& P = ph.dev;
  P.x = b.take<float>(n * dp);
  P.g = b.take<float>(n * dp);
  P.f = b.take<float>(n);
  P.hs = b.take<float>(n * MMAX * dp);
  P.hy = b.take<float>(n * MMAX * dp);
  P.hrho = b.take<float>(n * MMAX);
  P.hlen = b.take<int>(n);
  P.stuck = b.take<uint32_t>(nw);
  P.removed = b.take<uint32_t>(nw);
  P.l_stuck = b.take<int>(n);
  P.l_free = b.take<int>(n);
  P.l_unf = b.take<int>(n);
  P.l_surv = b.take<int>(n);
  P.l_rank = b.take<int>(n);
  P.lo = b.take<float>(dp);
  P.hi = b.take<float>(dp);
  P.cnt = b.take<Counters>(1);
  P.partials = b.take<float2>((size_t)MAX_PART_BLOCKS * (2 * dp + 2));
  P.max_part_blocks = MAX_PART_BLOCKS;
  P.grq = b.take<double>((size_t)d * d);
  size_t slots = 1;
  while (slots < 2 * n) slots <<= 1;
  P.hkey = b.take<unsigned long long>(slots);
  P.hbest = b.take<unsigned long long>(slots);
  P.hhead = b.take<int>(slots);
  P.hnext = b.take<int>(n);
  P.hmask = (int)(slots - 1);
  P.hspread = b.take<unsigned>(2 * (size_t)dp);
  P.haxes = b.take<int>(4);
  size_t n0, n1, n2, n3;
  obj_elems(pr, dp, &n0, &n1, &n2, &n3);
  P.obj.f32.p0 = b.take<float>(n0);
  P.obj.f32.p1 = b.take<float>(n1);
  P.obj.f32.p2 = n2 ? b.take<float>(n2) : nullptr;
  P.obj.f32.p3 = n3 ? b.take<float>(n3) : nullptr;
  P.obj.f64.p0 = b.take<double>(n0);
  P.obj.f64.p1 = b.take<double>(n1);
  P.obj.f64.p2 = n2 ? b.take<double>(n2) : nullptr;
  P.obj.f64.p3 = n3 ? b.take<double>(n3) : nullptr;
  ph.gather_x = b.take<float>(n * d);
  ph.gather_f = b.take<float>(n);
  if (pr.objective.kind == CHISAO_OBJ_MIXTURE_FULL) {
    ph.tc_weights = b.take<uint8_t>(tc_weight_bytes(pr.objective.n_comp));
    ph.tc_part = b.take<float>(tc_split_floats());
    ph.tc_ticket = b.take<int>(tc_split_tickets());
  }
  ph.tc = prm.grad_mode == CHISAO_GRAD_ADJOINT_TC || pr.objective.kind == CHISAO_OBJ_EXTERNAL;
  if (ph.tc) {
    ExtBuf& E = ph.ext;
    E.p = b.take<float>(n * dp);
    E.xt = b.take<float>(n * dp);
    E.ft = b.take<float>(n);
    E.gt = b.take<float>(n * dp);
    E.a0 = b.take<float>(n);
    E.list0 = b.take<int>(n);
    E.mlist[0] = b.take<int>(n);
    E.mlist[1] = b.take<int>(n);
    E.cnt = b.take<int>(2 * ((size_t)ls_rounds(prm.T_ls) + 1));
    E.iota = b.take<int>(2 * LS_BATCH * n);
    E.fm = b.take<float>(2 * LS_BATCH * n);
    const size_t xrows = (size_t)std::max(prm.M, 2 * LS_BATCH) * n;
    E.xp = b.take<float>(xrows * dp);
    E.gp = b.take<float>(xrows * dp);
    E.vel = b.take<float>(n * dp);
    E.head = b.take<int>(n);
  }
}

// FP64 objective constants on the host, padded to dp (zeros in the padding).
void prepare_objective(const chisao_problem& pr, int dp, std::vector<double>& a0, std::vector<double>& a1,
                       std::vector<double>& a2, std::vector<double>& a3, std::vector<double>& linv_all) {
  const int d = pr.d;
  const chisao_objective& o = pr.objective;
  size_t n0, n1, n2, n3;
  obj_elems(pr, dp, &n0, &n1, &n2, &n3);
  a0.assign(n0, 0.0);
  a1.assign(n1, 0.0);
  a2.assign(n2, 0.0);
  a3.assign(n3, 0.0);
  const double half_log2pi = 0.5 * std::log(2.0 * M_PI);
  if (o.kind == CHISAO_OBJ_MIXTURE_DIAG) {
    for (int k = 0; k < o.n_comp; ++k) {
      double ls = 0.0;
      for (int j = 0; j < d; ++j) {
        const double s = o.sigmas[(size_t)k * d + j];
        a0[(size_t)k * dp + j] = o.means[(size_t)k * d + j];
        a1[(size_t)k * dp + j] = 1.0 / (s * s);
        ls += std::log(s);
      }
      a2[k] = std::log(o.weights[k]) - ls - d * half_log2pi;
    }
  } else if (o.kind == CHISAO_OBJ_MIXTURE_FULL) {
    std::vector<double> inv((size_t)d * d);
    linv_all.assign((size_t)o.n_comp * d * d, 0.0);
    for (int k = 0; k < o.n_comp; ++k) {
      const double* L = o.chol + (size_t)k * d * d;
      // inverse of the lower-triangular L by forward substitution, column by column
      std::fill(inv.begin(), inv.end(), 0.0);
      for (int c = 0; c < d; ++c) {
        for (int i = c; i < d; ++i) {
          double s = (i == c) ? 1.0 : 0.0;
          for (int j = c; j < i; ++j) s -= L[(size_t)i * d + j] * inv[(size_t)j * d + c];
          inv[(size_t)i * d + c] = s / L[(size_t)i * d + i];
        }
      }
      double ld = 0.0;
      for (int j = 0; j < d; ++j) {
        ld += std::log(L[(size_t)j * d + j]);
        a0[(size_t)k * dp + j] = o.means[(size_t)k * d + j];
      }
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          a1[((size_t)k * dp + i) * dp + j] = inv[(size_t)i * d + j];
          linv_all[((size_t)k * d + i) * d + j] = inv[(size_t)i * d + j];
          a3[((size_t)k * dp + j) * dp + i] = inv[(size_t)i * d + j];
        }
      a2[k] = std::log(o.weights[k]) - ld - d * half_log2pi;
    }
  } else if (o.kind == CHISAO_OBJ_QUADRATIC) {
    for (int j = 0; j < d; ++j) a0[j] = o.center[j];
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b) {
        double s = 0.0;
        for (int i = 0; i < d; ++i) s += o.Q[(size_t)i * d + a] * o.lam[i] * o.Q[(size_t)i * d + b];
        a1[(size_t)a * dp + b] = s;
      }
    quad_sym_table(a1, dp, a2.data());
  }
}

StepParams make_step_params(const chisao_params& p, int d) {
  StepParams s{};
  s.n_conv = p.n_conv > 0 ? p.n_conv : (d > 1 ? std::max(10, (int)std::ceil(3.0 * std::log2((double)d))) : 10);
  s.n_anti = p.n_anti;
  s.hlc_value_only = p.hlc_value_only;
  s.n_cloud = p.n_cloud;
  s.M = p.M;
  s.m = p.m;
  s.T_ls = p.T_ls;
  s.grad_mode = p.grad_mode;
  s.rm_min = p.rm_min_unfrozen;
  s.gr_patience = p.gr_patience;
  s.eps_grad = (float)p.eps_grad;
  s.eps_dup = (float)p.eps_dup;
  s.log_delta = (float)std::log(p.delta);
  s.mu = (float)p.mu;
  s.alpha_fixed = (float)p.alpha;
  s.sigma_fixed = (float)p.sigma;
  s.c_sigma = (float)p.c_sigma;
  s.alpha_scale = (float)p.alpha_scale;
  s.h = p.h;
  s.h_rel = p.h_rel;
  s.c1 = p.c1;
  s.curv_eps = p.curv_eps;
  s.seed_lo = (unsigned)(p.seed & 0xffffffffu);
  s.seed_hi = (unsigned)(p.seed >> 32);
  s.n_refine = p.n_refine;
  return s;
}

cudaError_t launch_objective(int which, const ProbHost& ph, int gm, int arg, const EvalArgs* ea, cudaStream_t st) {
  switch (ph.kind) {
    case CHISAO_OBJ_MIXTURE_DIAG: return launch_obj_mixdiag(which, gm, ph.dev, ph.sp, arg, ea, st);
    case CHISAO_OBJ_QUADRATIC: return launch_obj_quad(which, gm, ph.dev, ph.sp, arg, ea, st);
    case CHISAO_OBJ_MIXTURE_FULL: return launch_obj_mixfull(which, gm, ph.dev, ph.sp, arg, ea, st);
    case CHISAO_OBJ_EXTERNAL: return cudaErrorNotSupported;      // no per-sample device objective
    default: return launch_obj_bench(which, gm, ph.dev, ph.sp, arg, ea, st);
  }
}

__global__ void k_reset_problem(ProbDev P) {
  if (threadIdx.x != 0) return;
  Counters* c = P.cnt;
  memset(c, 0, sizeof(Counters));
  c->gr_enabled = 1;
  c->gr_prev_surv = -1;
}

// Phases 4-6 of one problem (reseed, HLC with its scale pass, anti with its scale pass).
cudaError_t enqueue_explore(const ProbHost& ph, cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_reseed(ph.dev, ph.sp, st)) != cudaSuccess) return e;
  // Phase 1 left the gradients of every unmoved sample in g: only reseeded slots need new ones
  if ((e = launch_objective(OKID_SCALES, ph, ph.sp.grad_mode, 1, nullptr, st)) != cudaSuccess) return e;
  if ((e = launch_finalize_scales(ph.dev, ph.sp, 0, st)) != cudaSuccess) return e;
  if ((e = launch_objective(OKID_HLC, ph, ph.sp.grad_mode, 0, nullptr, st)) != cudaSuccess) return e;
  if ((e = launch_objective(OKID_SCALES, ph, ph.sp.grad_mode, 0, nullptr, st)) != cudaSuccess) return e;
  if ((e = launch_finalize_scales(ph.dev, ph.sp, 1, st)) != cudaSuccess) return e;
  return launch_objective(OKID_ANTI, ph, ph.sp.grad_mode, 0, nullptr, st);
}

// ---- batched objectives (the tensor-core mixture, or the caller's evaluator) around per-sample kernels
cudaError_t tc_eval_rows(const ProbHost& ph, const float* x, float* f, float* g, int rows, const int* idx,
                         const int* count, cudaStream_t st) {
  if (ph.kind == CHISAO_OBJ_EXTERNAL) {
    const int32_t r = ph.ext_eval(ph.ext_user, x, ph.dp, rows, idx, count, f, g, ph.dp, st);
    if (r != 0) {
      ph.ext_status = r;
      return cudaErrorUnknown;
    }
    return launch_zero_padding(g, rows, ph.d, ph.dp, st);   // the evaluator writes d coordinates only
  }
  return tc_launch_mixfull(x, ph.dp, rows, ph.d, ph.K, ph.tc_weights, f, g, ph.dp, &ph.dev.cnt->err, st,
                           ph.tc_part, ph.tc_ticket, idx, count);
}

// n_iter L-BFGS iterations (Phase 1).  Per iteration: the direction kernel writes
// the first trial point of every moving sample; round 0 evaluates them and accepts
// or hands each failing sample on with its next LS_BATCH trial points; each later
// round evaluates all pending trial points in one call (rows 0 .. 4 count - 1 of
// its buffer, through the identity row list) and accepts the first passing trial.
cudaError_t enqueue_phase1_tc(const ProbHost& ph, int n_iter, bool fresh, cudaStream_t st) {
  const ProbDev& P = ph.dev;
  const ExtBuf& E = ph.ext;
  const int R = ls_rounds(ph.sp.T_ls);
  const size_t brows = (size_t)LS_BATCH * P.n;          // rows of one trial-point buffer
  cudaError_t e;
  if (fresh && (e = tc_eval_rows(ph, P.x, P.f, P.g, P.n, nullptr, nullptr, st)) != cudaSuccess) return e;
  for (int it = 0; it < n_iter; ++it) {
    if ((e = cudaMemsetAsync(E.cnt, 0, sizeof(int) * 2 * (R + 1), st)) != cudaSuccess) return e;
    if ((e = launch_ext(EXT_DIR, P, ph.sp, E, (fresh && it == 0) ? 1 : 0, st)) != cudaSuccess) return e;
    if ((e = tc_eval_rows(ph, E.xt, E.ft, E.gt, P.n, E.list0, E.cnt, st)) != cudaSuccess) return e;
    if ((e = launch_ext(EXT_ACCEPT, P, ph.sp, E, 0, st)) != cudaSuccess) return e;
    for (int r = 1; r < R; ++r) {
      const size_t o = (size_t)((r - 1) & 1) * brows;   // buffer written by the previous round
      if ((e = tc_eval_rows(ph, E.xp + o * ph.dp, E.fm + o, E.gp + o * ph.dp, (int)brows, E.iota,
                            E.cnt + (R + 1) + r, st)) != cudaSuccess)
        return e;
      if ((e = launch_ext(EXT_ACCEPT_MULTI, P, ph.sp, E, r, st)) != cudaSuccess) return e;
    }
  }
  return n_iter > 0 ? launch_ext(EXT_HIST_ROTATE, P, ph.sp, E, 0, st) : cudaSuccess;   // newest pair to slot 0
}

// Phase 5 (scale pass + HLC) with all M perturbations evaluated in one launch.
cudaError_t enqueue_hlc_tc(const ProbHost& ph, cudaStream_t st) {
  const ProbDev& P = ph.dev;
  const ExtBuf& E = ph.ext;
  cudaError_t e;
  if ((e = tc_eval_rows(ph, P.x, nullptr, P.g, P.n, nullptr, nullptr, st)) != cudaSuccess) return e;
  if ((e = launch_ext(EXT_SCALES, P, ph.sp, E, 0, st)) != cudaSuccess) return e;
  if ((e = launch_finalize_scales(P, ph.sp, 0, st)) != cudaSuccess) return e;
  for (int t = 0; t < ph.sp.n_cloud; ++t) {
    if ((e = launch_ext(EXT_HLC_POINTS, P, ph.sp, E, t, st)) != cudaSuccess) return e;
    if ((e = tc_eval_rows(ph, E.xp, nullptr, E.gp, ph.sp.M * P.n, nullptr, nullptr, st)) != cudaSuccess) return e;
    if ((e = launch_ext(EXT_HLC_STEP, P, ph.sp, E, t, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Phase 6 (scale pass + momentum steps).
cudaError_t enqueue_anti_tc(const ProbHost& ph, cudaStream_t st) {
  const ProbDev& P = ph.dev;
  const ExtBuf& E = ph.ext;
  cudaError_t e;
  if ((e = tc_eval_rows(ph, P.x, nullptr, P.g, P.n, nullptr, nullptr, st)) != cudaSuccess) return e;
  if ((e = launch_ext(EXT_SCALES, P, ph.sp, E, 0, st)) != cudaSuccess) return e;
  if ((e = launch_finalize_scales(P, ph.sp, 1, st)) != cudaSuccess) return e;
  for (int t = 0; t < ph.sp.n_anti; ++t) {
    if (t > 0 && (e = tc_eval_rows(ph, P.x, nullptr, P.g, P.n, nullptr, nullptr, st)) != cudaSuccess) return e;
    if ((e = launch_ext(EXT_ANTI_STEP, P, ph.sp, E, t, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// FP32 polish of the survivors with the exact objective (after the last cycle).
cudaError_t enqueue_refine(const ProbHost& ph, int n_iter, cudaStream_t st) {
  if (n_iter <= 0) return cudaSuccess;
  return launch_objective(OKID_REFINE, ph, GRAD_ADJOINT, n_iter, nullptr, st);
}

cudaError_t enqueue_cycle_tc(const ProbHost& ph, bool last, cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_cycle_begin(ph.dev, st)) != cudaSuccess) return e;
  if ((e = enqueue_phase1_tc(ph, ph.sp.n_conv, true, st)) != cudaSuccess) return e;
  if ((e = launch_freeze(ph.dev, ph.sp, st)) != cudaSuccess) return e;
  if ((e = launch_dedup(ph.dev, ph.sp, st)) != cudaSuccess) return e;
  if (!last) {
    if ((e = launch_reseed(ph.dev, ph.sp, st)) != cudaSuccess) return e;
    if ((e = enqueue_hlc_tc(ph, st)) != cudaSuccess) return e;
    if ((e = enqueue_anti_tc(ph, st)) != cudaSuccess) return e;
  } else if (ph.kind == CHISAO_OBJ_MIXTURE_FULL && (e = enqueue_refine(ph, ph.sp.n_refine, st)) != cudaSuccess) {
    return e;                        // the FP32 polish of tensor-core modes (an external objective is exact)
  }
  return launch_cycle_end(ph.dev, st);
}

// One oscillation cycle (Algorithm 1) of one problem.
cudaError_t enqueue_problem_cycle(const ProbHost& ph, bool last, cudaStream_t st) {
  if (ph.tc) return enqueue_cycle_tc(ph, last, st);
  cudaError_t e;
  if ((e = launch_cycle_begin(ph.dev, st)) != cudaSuccess) return e;                          // release all
  if ((e = launch_objective(OKID_PHASE1, ph, ph.sp.grad_mode, ph.sp.n_conv, nullptr, st)) != cudaSuccess)
    return e;                                                                                  // Phase 1
  if ((e = launch_freeze(ph.dev, ph.sp, st)) != cudaSuccess) return e;                        // Phase 2
  if ((e = launch_dedup(ph.dev, ph.sp, st)) != cudaSuccess) return e;                         // Phase 3
  if (!last && (e = enqueue_explore(ph, st)) != cudaSuccess) return e;                        // Phases 4-6
  return launch_cycle_end(ph.dev, st);
}

cudaError_t launch_grouped(int which, const Group& gr, cudaStream_t st, int arg = 0) {
  const GroupTab& T = which == OKID_SCALES ? gr.tab_sc : gr.tab;
  const unsigned blocks = which == OKID_SCALES ? gr.blocks_sc : gr.blocks;
  switch (gr.kind) {
    case CHISAO_OBJ_MIXTURE_DIAG: return launch_grp_mixdiag_tile(which, gr.dp, gr.tile, T, blocks, st, arg);
    case CHISAO_OBJ_MIXTURE_FULL: return launch_grp_mixfull(which, gr.dp, T, blocks, st, arg);
    case CHISAO_OBJ_QUADRATIC: return launch_grp_quad(which, gr.dp, T, blocks, st, arg);
    default: return launch_grp_bench(which, gr.dp, T, blocks, st, arg);
  }
}

// Phases 5 and 6 of a group: scale pass, finalization, HLC, scale pass, finalization, anti.
cudaError_t enqueue_explore_group(const Group& gr, cudaStream_t st) {
  cudaError_t e;
  const int k = (int)gr.members.size();
  if ((e = launch_grouped(OKID_SCALES, gr, st, 1)) != cudaSuccess) return e;      // Phase 1's gradients reused
  if ((e = launch_finalize_grp(gr.tab_sc, k, gr.dp, 0, st)) != cudaSuccess) return e;
  if ((e = launch_grouped(OKID_HLC, gr, st)) != cudaSuccess) return e;
  if ((e = launch_grouped(OKID_SCALES, gr, st)) != cudaSuccess) return e;
  if ((e = launch_finalize_grp(gr.tab_sc, k, gr.dp, 1, st)) != cudaSuccess) return e;
  return launch_grouped(OKID_ANTI, gr, st);
}

// Fork the branch streams from the context stream, run f(branch index) on each, join back.
template <class F>
cudaError_t forked(chisao_ctx* c, F&& f) {
  cudaError_t e;
  if ((e = cudaEventRecord(c->forked, c->stream)) != cudaSuccess) return e;
  for (cudaStream_t s : c->branch)
    if ((e = cudaStreamWaitEvent(s, c->forked, 0)) != cudaSuccess) return e;
  if ((e = f()) != cudaSuccess) return e;
  for (size_t b = 0; b < c->branch.size(); ++b) {
    if ((e = cudaEventRecord(c->joined[b], c->branch[b])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->stream, c->joined[b], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One cycle with grouped launches: the objective-independent steps (release, freeze,
// dedup, reseed, cycle end) of all problems run as one launch per kernel on the context
// stream; Phase 1, and then the scale passes with Phases 5 and 6, run as one chain of
// launches per group (the groups on separate branches), with joins in between, since
// every phase needs the previous one of the same problem.
cudaError_t enqueue_cycle_grouped(chisao_ctx* c, bool last) {
  auto per_group = [&](auto&& body) {
    return forked(c, [&]() -> cudaError_t {
      for (size_t k = 0; k < c->groups.size(); ++k) {
        const cudaError_t e = body(c->groups[k], c->branch[k % c->branch.size()]);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    });
  };
  cudaError_t e;
  // the objective-independent steps of all problems are one launch per kernel on the
  // context stream; the per-group objective phases run on the branches
  if ((e = launch_cycle_begin_all(c->all, c->stream)) != cudaSuccess) return e;
  if ((e = per_group([](const Group& gr, cudaStream_t s) { return launch_grouped(OKID_PHASE1, gr, s); })) !=
      cudaSuccess)
    return e;                                                                               // Phase 1
  if ((e = launch_freeze_all(c->all, c->stream)) != cudaSuccess) return e;                // Phase 2
  if ((e = launch_dedup_all(c->all, c->stream)) != cudaSuccess) return e;                 // Phase 3
  if (!last && (e = launch_reseed_all(c->all, c->stream)) != cudaSuccess) return e;       // Phase 4
  if (!last && (e = per_group(enqueue_explore_group)) != cudaSuccess) return e;            // Phases 5-6
  return launch_cycle_end_all(c->all, c->stream);
}

// One oscillation cycle of every problem: independent problems on the branch streams.
cudaError_t enqueue_cycle(chisao_ctx* c, bool last) {
  cudaError_t e;
  if (!c->groups.empty() && c->groups_enabled) return enqueue_cycle_grouped(c, last);
  if (c->branch.empty()) {
    for (const ProbHost& ph : c->probs)
      if ((e = enqueue_problem_cycle(ph, last, c->stream)) != cudaSuccess) return e;
    return cudaSuccess;
  }
  if ((e = cudaEventRecord(c->forked, c->stream)) != cudaSuccess) return e;
  for (cudaStream_t s : c->branch)
    if ((e = cudaStreamWaitEvent(s, c->forked, 0)) != cudaSuccess) return e;
  for (size_t q = 0; q < c->probs.size(); ++q)
    if ((e = enqueue_problem_cycle(c->probs[q], last, c->branch[c->branch_of[q]])) != cudaSuccess) return e;
  for (size_t b = 0; b < c->branch.size(); ++b) {
    if ((e = cudaEventRecord(c->joined[b], c->branch[b])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(c->stream, c->joined[b], 0)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void free_branches(chisao_ctx* c) {
  for (cudaStream_t s : c->branch) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  for (cudaEvent_t ev : c->joined) cudaEventDestroy(ev);
  if (c->forked) cudaEventDestroy(c->forked);
  c->branch.clear();
  c->joined.clear();
  c->forked = nullptr;
  c->branch_of.clear();
}

// Branch streams for a context of several problems (nb_req of them, at most one per
// problem); each problem goes, largest first, to the branch with the least work so far
// (work ~ samples x padded dimension).
cudaError_t make_branches(chisao_ctx* c, int nb_req = 32) {
  const int nq = (int)c->probs.size();
  if (nq < 2) return cudaSuccess;
  const int nb = std::max(1, std::min(nq, nb_req));
  cudaError_t e;
  if ((e = cudaEventCreateWithFlags(&c->forked, cudaEventDisableTiming)) != cudaSuccess) return e;
  for (int b = 0; b < nb; ++b) {
    cudaStream_t s;
    cudaEvent_t ev;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return e;
    c->branch.push_back(s);
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
    c->joined.push_back(ev);
  }
  std::vector<int> order(nq);
  for (int q = 0; q < nq; ++q) order[q] = q;
  auto work = [&](int q) { return (double)c->probs[q].n * c->probs[q].dp; };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) > work(y); });
  std::vector<double> load(nb, 0.0);
  c->branch_of.assign(nq, 0);
  for (int q : order) {
    const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    c->branch_of[q] = b;
    load[b] += work(q);
  }
  return cudaSuccess;
}

// Grouped launches when the context holds several problems with exact gradients (none
// on the batched-evaluator path): problems of one (kind, dp) form a group whose Phase 1,
// HLC and anti-convergence each run as one launch covering all its samples.
cudaError_t make_groups(chisao_ctx* c) {
  const int nq = (int)c->probs.size();
  if (nq < 2 || c->params.grad_mode != CHISAO_GRAD_ADJOINT) return cudaSuccess;
  for (const ProbHost& ph : c->probs)
    if (ph.tc) return cudaSuccess;
  for (int q = 0; q < nq; ++q) {
    const ProbHost& ph = c->probs[q];
    Group* gr = nullptr;
    for (Group& x : c->groups)
      if (x.kind == ph.kind && x.dp == ph.dp) gr = &x;
    if (!gr) {
      c->groups.emplace_back();
      gr = &c->groups.back();
      gr->kind = ph.kind;
      gr->dp = ph.dp;
    }
    gr->members.push_back(q);
  }
  for (Group& gr : c->groups) {
    const size_t k = gr.members.size();
    // two block maps over the same problem tables: NT_OBJ-thread blocks over the samples, and
    // each problem's scale-pass grid
    std::vector<int> first(k), count(k), owner, first_sc(k), count_sc(k), owner_sc;
    std::vector<ProbDev> pd(k);
    std::vector<StepParams> sp(k);
    for (size_t j = 0; j < k; ++j) {
      const ProbHost& ph = c->probs[gr.members[j]];
      pd[j] = ph.dev;
      sp[j] = ph.sp;
      first[j] = (int)owner.size();
      count[j] = (int)obj_blocks(ph.n, ph.dp);
      owner.insert(owner.end(), count[j], (int)j);
      first_sc[j] = (int)owner_sc.size();
      count_sc[j] = scale_blocks(ph.dev);
      owner_sc.insert(owner_sc.end(), count_sc[j], (int)j);
    }
    gr.blocks = (unsigned)owner.size();
    gr.blocks_sc = (unsigned)owner_sc.size();
    auto up = [](size_t off) { return (off + ALIGN - 1) / ALIGN * ALIGN; };
    struct Part { const void* src; size_t bytes; size_t off; };
    std::vector<Part> parts = {{pd.data(), k * sizeof(ProbDev), 0}, {sp.data(), k * sizeof(StepParams), 0},
                               {first.data(), k * sizeof(int), 0}, {count.data(), k * sizeof(int), 0},
                               {owner.data(), owner.size() * sizeof(int), 0},
                               {first_sc.data(), k * sizeof(int), 0}, {count_sc.data(), k * sizeof(int), 0},
                               {owner_sc.data(), owner_sc.size() * sizeof(int), 0}};
    size_t total = 0;
    for (Part& p : parts) {
      p.off = total;
      total = up(total + p.bytes);
    }
    cudaError_t e;
    if ((e = cudaMalloc(&gr.mem, total)) != cudaSuccess) return e;
    char* base = static_cast<char*>(gr.mem);
    for (const Part& p : parts)
      if ((e = cudaMemcpy(base + p.off, p.src, p.bytes, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    auto at = [&](int t) { return reinterpret_cast<const int*>(base + parts[t].off); };
    gr.tab.probs = gr.tab_sc.probs = reinterpret_cast<const ProbDev*>(base + parts[0].off);
    gr.tab.sps = gr.tab_sc.sps = reinterpret_cast<const StepParams*>(base + parts[1].off);
    gr.tab.blk_first = at(2);
    gr.tab.blk_count = at(3);
    gr.tab.blk_prob = at(4);
    gr.tab_sc.blk_first = at(5);
    gr.tab_sc.blk_count = at(6);
    gr.tab_sc.blk_prob = at(7);
  }
  std::vector<ProbDev> pd(nq);
  std::vector<StepParams> sp(nq);
  for (int q = 0; q < nq; ++q) {
    pd[q] = c->probs[q].dev;
    sp[q] = c->probs[q].sp;
  }
  return build_all_tabs(pd, sp, &c->all_mem, &c->all);
}

chisao_status check_prob(chisao_ctx* c, int32_t prob) {
  if (!c) return CHISAO_ERR_ARG;
  if (prob < 0 || prob >= (int32_t)c->probs.size()) return fail(c, CHISAO_ERR_ARG, "problem index out of range");
  return CHISAO_OK;
}

}  // namespace

extern "C" {

void chisao_default_params(chisao_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->n_osc = 3;
  p->n_conv = 0;
  p->n_anti = 5;
  p->n_cloud = 3;
  p->M = 8;
  p->m = 10;
  p->T_ls = 20;
  p->grad_mode = CHISAO_GRAD_FD64;
  p->eps_grad = 1e-6;
  p->eps_dup = 1e-3;
  p->delta = 0.1;
  p->mu = 0.9;
  p->alpha = 0.0;
  p->sigma = 0.0;
  p->c_sigma = 0.1;
  p->alpha_scale = 0.1;
  p->h = 1e-5;
  p->h_rel = std::pow(2.0, -23.0 / 3.0);
  p->c1 = 1e-4;
  p->curv_eps = 1e-10;
  p->seed = 0;
  p->rm_min_unfrozen = 5;
  p->gr_patience = 2;
  p->use_graph = 1;
  p->n_refine = 10;
}

chisao_status chisao_arena_bytes(const chisao_problem* probs, int32_t n_probs, const chisao_params* params,
                                 size_t* bytes) {
  std::string why;
  if (!probs || n_probs < 1 || n_probs > 65536 || !bytes) return CHISAO_ERR_ARG;
  if (validate_params(params, why) != CHISAO_OK) return CHISAO_ERR_ARG;
  Bump b;
  for (int q = 0; q < n_probs; ++q) {
    if (validate_problem(&probs[q], why) != CHISAO_OK) return CHISAO_ERR_ARG;
    ProbHost ph;
    if (validate_mode(&probs[q], params, why) != CHISAO_OK) return CHISAO_ERR_ARG;
    layout_problem(b, probs[q], *params, ph);
  }
  *bytes = (b.off + ALIGN - 1) / ALIGN * ALIGN;
  return CHISAO_OK;
}

chisao_status chisao_create(const chisao_problem* probs, int32_t n_probs, const chisao_params* params, void* arena,
                            size_t arena_bytes, void* cuda_stream, chisao_ctx** out) {
  if (!out) return CHISAO_ERR_ARG;
  *out = nullptr;
  std::string why;
  if (!probs || n_probs < 1 || n_probs > 65536) return CHISAO_ERR_ARG;
  if (validate_params(params, why) != CHISAO_OK) {
    fprintf(stderr, "chisao_create: %s\n", why.c_str());
    return CHISAO_ERR_ARG;
  }
  for (int q = 0; q < n_probs; ++q)
    if (validate_problem(&probs[q], why) != CHISAO_OK || validate_mode(&probs[q], params, why) != CHISAO_OK) {
      fprintf(stderr, "chisao_create: problem %d: %s\n", q, why.c_str());
      return CHISAO_ERR_ARG;
    }
  size_t need = 0;
  chisao_arena_bytes(probs, n_probs, params, &need);
  if (arena && (arena_bytes < need || (reinterpret_cast<uintptr_t>(arena) % ALIGN) != 0)) return CHISAO_ERR_OOM;

  chisao_ctx* c = new chisao_ctx();
  c->params = *params;
  if (prepare_kernel_attributes() != cudaSuccess || tc_prepare_attributes() != cudaSuccess) {
    delete c;
    return CHISAO_ERR_CUDA;
  }
  if (cuda_stream) {
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return CHISAO_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (arena) {
    c->arena = reinterpret_cast<char*>(arena);
    c->arena_bytes = arena_bytes;
  } else {
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      chisao_destroy(c);
      return CHISAO_ERR_OOM;
    }
    c->arena = reinterpret_cast<char*>(p);
    c->arena_bytes = need;
    c->own_arena = true;
  }
  Bump b;
  b.base = c->arena;
  c->probs.resize(n_probs);
  std::vector<double> a0, a1, a2, a3, linv_all, logw;
  std::vector<uint8_t> tcw;
  std::vector<float> f0, f1, f2, f3, box;
  auto to32 = [](const std::vector<double>& v, std::vector<float>& o) {
    o.resize(v.size());
    for (size_t t = 0; t < v.size(); ++t) o[t] = (float)v[t];
  };
  chisao_status st = CHISAO_OK;
  for (int q = 0; q < n_probs && st == CHISAO_OK; ++q) {
    const chisao_problem& pr = probs[q];
    ProbHost& ph = c->probs[q];
    ph.d = pr.d;
    ph.dp = pad_dim(pr.d);
    ph.n = pr.n;
    ph.kind = pr.objective.kind;
    ph.K = pr.objective.n_comp;
    ph.ext_eval = pr.objective.eval;
    ph.ext_user = pr.objective.user;
    layout_problem(b, pr, *params, ph);
    ProbDev& P = ph.dev;
    P.d = ph.d;
    P.dp = ph.dp;
    P.n = (int)ph.n;
    P.nwords = (int)((ph.n + 31) / 32);
    P.prob_index = q;
    P.m = params->m;
    P.obj.kind = is_bench_kind(ph.kind) ? OBJ_BENCH : ph.kind;
    P.obj.f32.fn = P.obj.f64.fn = is_bench_kind(ph.kind) ? ph.kind - CHISAO_OBJ_RASTRIGIN : 0;
    P.obj.prob_index = q;
    P.obj.noise_sigma = (float)pr.objective.noise_sigma;
    P.obj.f32.K = P.obj.f64.K = (ph.kind == CHISAO_OBJ_MIXTURE_DIAG || ph.kind == CHISAO_OBJ_MIXTURE_FULL) ? ph.K : 0;
    P.obj.f32.d = P.obj.f64.d = ph.d;
    P.obj.f32.dp = P.obj.f64.dp = ph.dp;
    ph.sp = make_step_params(*params, ph.d);
    prepare_objective(pr, ph.dp, a0, a1, a2, a3, linv_all);
    if (ph.kind == CHISAO_OBJ_MIXTURE_FULL) {
      logw.resize(ph.K);
      for (int k = 0; k < ph.K; ++k) logw[k] = std::log(pr.objective.weights[k]);
      tc_build_weights(ph.K, ph.d, linv_all.data(), pr.objective.means, logw.data(), tcw);
      if (cudaMemcpy(ph.tc_weights, tcw.data(), tcw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemset(ph.tc_ticket, 0, tc_split_tickets() * sizeof(int)) != cudaSuccess)
        st = cuda_fail(c, cudaGetLastError(), "tensor-core weight upload");
    }
    if (ph.tc && (cudaMemsetAsync(ph.ext.head, 0, sizeof(int) * (size_t)P.n, c->stream) != cudaSuccess ||
                  launch_ext(EXT_IOTA, P, ph.sp, ph.ext, 0, c->stream) != cudaSuccess))
      st = cuda_fail(c, cudaGetLastError(), "row list of the line-search rounds");
    to32(a0, f0); to32(a1, f1); to32(a2, f2); to32(a3, f3);
    auto up = [&](const void* dst, const void* src, size_t bytes) {
      if (bytes && cudaMemcpy(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        st = cuda_fail(c, cudaGetLastError(), "objective upload");
    };
    up(P.obj.f64.p0, a0.data(), a0.size() * 8);
    up(P.obj.f64.p1, a1.data(), a1.size() * 8);
    if (P.obj.f64.p2) up(P.obj.f64.p2, a2.data(), a2.size() * 8);
    if (P.obj.f64.p3) up(P.obj.f64.p3, a3.data(), a3.size() * 8);
    up(P.obj.f32.p0, f0.data(), f0.size() * 4);
    up(P.obj.f32.p1, f1.data(), f1.size() * 4);
    if (P.obj.f32.p2) up(P.obj.f32.p2, f2.data(), f2.size() * 4);
    if (P.obj.f32.p3) up(P.obj.f32.p3, f3.data(), f3.size() * 4);
    box.assign(ph.dp, 0.f);
    for (int j = 0; j < ph.d; ++j) box[j] = (float)pr.lo[j];
    up(P.lo, box.data(), box.size() * 4);
    for (int j = 0; j < ph.d; ++j) box[j] = (float)pr.hi[j];
    up(P.hi, box.data(), box.size() * 4);
  }
  if (st == CHISAO_OK && make_branches(c) != cudaSuccess) st = cuda_fail(c, cudaGetLastError(), "branch streams");
  if (st == CHISAO_OK && make_groups(c) != cudaSuccess) st = cuda_fail(c, cudaGetLastError(), "grouped launch tables");
  if (st != CHISAO_OK) {
    chisao_destroy(c);
    return st;
  }
  for (int q = 0; q < n_probs; ++q) {
    if ((st = chisao_load_population(c, q, probs[q].x0)) != CHISAO_OK) {
      fprintf(stderr, "chisao_create: %s\n", c->err.c_str());
      chisao_destroy(c);
      return st;
    }
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    chisao_destroy(c);
    return CHISAO_ERR_CUDA;
  }
  *out = c;
  return CHISAO_OK;
}

chisao_status chisao_init(const chisao_problem* probs, int32_t n_probs, const chisao_params* params,
                          void* cuda_stream, chisao_ctx** out) {
  return chisao_create(probs, n_probs, params, nullptr, 0, cuda_stream, out);
}

chisao_status chisao_load_population(chisao_ctx* c, int32_t prob, const float* x_host) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  if (!x_host) return fail(c, CHISAO_ERR_ARG, "x_host is NULL");
  ProbHost& ph = c->probs[prob];
  ProbDev& P = ph.dev;
  const size_t n = (size_t)ph.n;
  CK(cudaMemsetAsync(P.x, 0, n * ph.dp * sizeof(float), c->stream));
  CK(cudaMemcpy2DAsync(P.x, ph.dp * sizeof(float), x_host, ph.d * sizeof(float), ph.d * sizeof(float), n,
                       cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(P.g, 0, n * ph.dp * sizeof(float), c->stream));
  CK(cudaMemsetAsync(P.f, 0, n * sizeof(float), c->stream));
  CK(cudaMemsetAsync(P.hlen, 0, n * sizeof(int), c->stream));
  CK(cudaMemsetAsync(P.stuck, 0, P.nwords * sizeof(uint32_t), c->stream));
  CK(cudaMemsetAsync(P.removed, 0, P.nwords * sizeof(uint32_t), c->stream));
  k_reset_problem<<<1, 32, 0, c->stream>>>(P);
  CK(cudaGetLastError());
  c->cycles_done = 0;
  return CHISAO_OK;
}

chisao_status chisao_seed(chisao_ctx* c, int32_t prob, int32_t method) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  if (method != CHISAO_SEED_UNIFORM && method != CHISAO_SEED_CARRY_TIGER)
    return fail(c, CHISAO_ERR_ARG, "unknown seeding method");
  ProbHost& ph = c->probs[prob];
  ProbDev& P = ph.dev;
  const size_t n = (size_t)ph.n;
  CK(cudaMemsetAsync(P.x, 0, n * ph.dp * sizeof(float), c->stream));     // the padding coordinates
  CK(launch_seed(P, ph.sp, method, c->stream));
  CK(cudaMemsetAsync(P.g, 0, n * ph.dp * sizeof(float), c->stream));
  CK(cudaMemsetAsync(P.f, 0, n * sizeof(float), c->stream));
  CK(cudaMemsetAsync(P.hlen, 0, n * sizeof(int), c->stream));
  CK(cudaMemsetAsync(P.stuck, 0, P.nwords * sizeof(uint32_t), c->stream));
  CK(cudaMemsetAsync(P.removed, 0, P.nwords * sizeof(uint32_t), c->stream));
  k_reset_problem<<<1, 32, 0, c->stream>>>(P);
  CK(cudaGetLastError());
  c->cycles_done = 0;
  return CHISAO_OK;
}

chisao_status chisao_step(chisao_ctx* c) {
  if (!c) return CHISAO_ERR_ARG;
  if (c->cycles_done >= c->params.n_osc) return fail(c, CHISAO_ERR_STATE, "all n_osc cycles have run");
  const bool last = c->cycles_done + 1 >= c->params.n_osc;
  if (c->params.use_graph) {
    cudaGraphExec_t& ge = last ? c->g_last : c->g_mid;
    if (!ge) {
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      const cudaError_t e = enqueue_cycle(c, last);
      const cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
      if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(c, e, "cycle capture");
      }
      if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
      const cudaError_t e3 = cudaGraphInstantiate(&ge, graph, 0);
      cudaGraphDestroy(graph);
      if (e3 != cudaSuccess) {
        ge = nullptr;
        return cuda_fail(c, e3, "cudaGraphInstantiate");
      }
    }
    CK(cudaGraphLaunch(ge, c->stream));
  } else {
    const cudaError_t e = enqueue_cycle(c, last);
    if (e != cudaSuccess) return cuda_fail(c, e, "cycle launch");
  }
  c->cycles_done += 1;
  return CHISAO_OK;
}

chisao_status chisao_modes(chisao_ctx* c, int32_t prob, float* x_out, float* f_out, int64_t cap, int64_t* count) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  if (!count || cap < 0 || (cap > 0 && !x_out)) return fail(c, CHISAO_ERR_ARG, "bad output arguments");
  ProbHost& ph = c->probs[prob];
  Counters cnt;
  CK(cudaMemcpyAsync(&cnt, ph.dev.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *count = cnt.n_surv;
  if (cnt.n_surv > cap) return fail(c, CHISAO_ERR_CAPACITY, "output capacity below the number of modes");
  if (cnt.n_surv == 0) return CHISAO_OK;
  CK(launch_gather_modes(ph.dev, ph.gather_x, ph.gather_f, c->stream));
  CK(cudaMemcpyAsync(x_out, ph.gather_x, sizeof(float) * cnt.n_surv * ph.d, cudaMemcpyDeviceToHost, c->stream));
  if (f_out) CK(cudaMemcpyAsync(f_out, ph.gather_f, sizeof(float) * cnt.n_surv, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return CHISAO_OK;
}

chisao_status chisao_measure_fma_peak(int32_t precision, void* cuda_stream, double* flops) {
  if (!flops || (precision != 0 && precision != 1)) return CHISAO_ERR_ARG;
  return measure_fma_peak(precision, flops, reinterpret_cast<cudaStream_t>(cuda_stream)) == cudaSuccess
             ? CHISAO_OK
             : CHISAO_ERR_CUDA;
}

chisao_status chisao_measure_mma_rate(int32_t n, int32_t threads, int32_t tmem_a, void* cuda_stream,
                                      double* clk_per_mma) {
  const int nmax = threads == 1 ? 256 : threads == 2 ? 128 : 64;   // each issuer's accumulator width
  if (!clk_per_mma || n < 16 || n > nmax || n % 16 || threads < 1 || threads > 4 || tmem_a < 0 ||
      tmem_a > threads)
    return CHISAO_ERR_ARG;
  return tc_measure_mma_rate(n, threads, tmem_a, clk_per_mma, reinterpret_cast<cudaStream_t>(cuda_stream)) ==
                 cudaSuccess
             ? CHISAO_OK
             : CHISAO_ERR_CUDA;
}

chisao_status chisao_autotune(chisao_ctx* c, int32_t cycles_per_trial, chisao_tuning* out) {
  if (!c) return CHISAO_ERR_ARG;
  if (!out || cycles_per_trial < 1 || cycles_per_trial > 100) return fail(c, CHISAO_ERR_ARG, "bad arguments");
  memset(out, 0, sizeof(*out));
  out->n_branch = (int32_t)c->branch.size();
  out->grouped = (!c->groups.empty() && c->groups_enabled) ? 1 : 0;
  const int nq = (int)c->probs.size();
  if (nq < 2) return CHISAO_OK;
  for (const ProbHost& ph : c->probs)                 // a caller's evaluator may not be capture-safe
    if (ph.kind == CHISAO_OBJ_EXTERNAL) return CHISAO_OK;
  void* backup = nullptr;
  if (cudaMalloc(&backup, c->arena_bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CHISAO_ERR_OOM, "no device memory for the state snapshot");
  }
  const int saved_cycles = c->cycles_done;
  const int def_nb = (int)c->branch.size();
  const bool def_g = c->groups_enabled;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemcpyAsync(backup, c->arena, c->arena_bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto restore = [&]() {
    return cudaMemcpyAsync(c->arena, backup, c->arena_bytes, cudaMemcpyDeviceToDevice, c->stream);
  };
  auto apply = [&](int nb, bool grouped) -> cudaError_t {
    cudaError_t r = cudaStreamSynchronize(c->stream);
    if (r != cudaSuccess) return r;
    free_branches(c);
    c->groups_enabled = grouped;
    return make_branches(c, nb);
  };
  // one trial: restore, capture a non-final cycle, run it once untimed, then time it
  auto trial = [&](float* ms) -> cudaError_t {
    cudaError_t r;
    if ((r = restore()) != cudaSuccess) return r;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t ge = nullptr;
    if ((r = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return r;
    const cudaError_t rc = enqueue_cycle(c, false);
    r = cudaStreamEndCapture(c->stream, &graph);
    if (rc != cudaSuccess || r != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return rc != cudaSuccess ? rc : r;
    }
    r = cudaGraphInstantiate(&ge, graph, 0);
    cudaGraphDestroy(graph);
    if (r != cudaSuccess) return r;
    if ((r = cudaGraphLaunch(ge, c->stream)) == cudaSuccess && (r = cudaEventRecord(e0, c->stream)) == cudaSuccess) {
      for (int k = 0; k < cycles_per_trial && r == cudaSuccess; ++k) r = cudaGraphLaunch(ge, c->stream);
      if (r == cudaSuccess) r = cudaEventRecord(e1, c->stream);
      if (r == cudaSuccess) r = cudaEventSynchronize(e1);
      if (r == cudaSuccess) r = cudaEventElapsedTime(ms, e0, e1);
    }
    cudaGraphExecDestroy(ge);
    *ms /= (float)cycles_per_trial;
    return r;
  };
  int best_nb = def_nb, trials = 0;
  bool best_g = def_g;
  float best = 3.0e38f, def_ms = 0.f;
  const int nbs[4] = {8, 16, 32, 64};
  for (int gi = 0; gi < (c->groups.empty() ? 1 : 2) && e == cudaSuccess; ++gi) {
    const bool g = c->groups.empty() ? false : gi == 0;
    int last_nb = -1;
    for (int t = 0; t < 4 && e == cudaSuccess; ++t) {
      const int nb = std::min(nbs[t], nq);
      if (nb == last_nb) continue;                   // fewer problems than the candidate
      last_nb = nb;
      float ms = 0.f;
      if ((e = apply(nb, g)) != cudaSuccess || (e = trial(&ms)) != cudaSuccess) break;
      ++trials;
      if (nb == def_nb && g == def_g) def_ms = ms;
      if (ms < best) {
        best = ms;
        best_nb = nb;
        best_g = g;
      }
    }
  }
  // the tile shape of each group of diagonal mixtures (components per step), one group at
  // a time with the chosen launch shape (every tile gives the same results)
  if (e == cudaSuccess && best_g) {
    e = apply(best_nb, best_g);
    for (Group& gr : c->groups) {
      if (e != cudaSuccess || gr.kind != CHISAO_OBJ_MIXTURE_DIAG) continue;
      int best_tile = gr.tile;
      for (int tile = 0; tile < MIXDIAG_TILES && e == cudaSuccess; ++tile) {
        if (tile == best_tile) continue;
        const int keep = gr.tile;
        gr.tile = tile;
        float ms = 0.f;
        if ((e = trial(&ms)) != cudaSuccess) break;
        ++trials;
        if (ms < best) {
          best = ms;
          best_tile = tile;
        } else {
          gr.tile = keep;
        }
      }
      gr.tile = best_tile;
    }
  }
  for (const Group& gr : c->groups) {
    int k = 0;
    while ((4 << k) < gr.dp) ++k;
    if (gr.kind == CHISAO_OBJ_MIXTURE_DIAG && k < 5) out->ck[k] = MIXDIAG_TILE_CK[gr.tile];
  }
  // the chosen configuration, the saved state, and graphs recaptured at the next step
  const cudaError_t ea = apply(best_nb, best_g);
  if (e == cudaSuccess) e = ea;
  if (e == cudaSuccess) e = restore();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (c->g_mid) cudaGraphExecDestroy(c->g_mid);
  if (c->g_last) cudaGraphExecDestroy(c->g_last);
  c->g_mid = c->g_last = nullptr;
  c->cycles_done = saved_cycles;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(backup);
  if (e != cudaSuccess) return cuda_fail(c, e, "autotune");
  out->n_branch = best_nb;
  out->grouped = best_g ? 1 : 0;
  out->trials = trials;
  out->ms_per_cycle = best;
  out->ms_default = def_ms;
  return CHISAO_OK;
}

chisao_status chisao_widths(chisao_ctx* c, int32_t prob, float* w_out, float* cov_out, int64_t cap,
                            int64_t* count) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  if (!count || cap < 0 || (cap > 0 && !w_out)) return fail(c, CHISAO_ERR_ARG, "bad output arguments");
  ProbHost& ph = c->probs[prob];
  Counters cnt;
  CK(cudaMemcpyAsync(&cnt, ph.dev.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *count = cnt.n_surv;
  if (cnt.n_surv > cap) return fail(c, CHISAO_ERR_CAPACITY, "output capacity below the number of modes");
  if (cnt.n_surv == 0) return CHISAO_OK;
  const size_t S = (size_t)cnt.n_surv, d = (size_t)ph.d;
  float* cov = nullptr;
  if (cov_out && cudaMalloc(&cov, sizeof(float) * S * d * d) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CHISAO_ERR_OOM, "no device memory for the covariance rows");
  }
  cudaError_t e = launch_widths(ph.dev, cnt.n_surv, ph.gather_x, cov, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w_out, ph.gather_x, sizeof(float) * S * d, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess && cov) e = cudaMemcpyAsync(cov_out, cov, sizeof(float) * S * d * d, cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (cov) cudaFree(cov);
  CK(e);
  return CHISAO_OK;
}

chisao_status chisao_get_counters(chisao_ctx* c, int32_t prob, chisao_counters* out) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  if (!out) return fail(c, CHISAO_ERR_ARG, "out is NULL");
  Counters cnt;
  CK(cudaMemcpyAsync(&cnt, c->probs[prob].dev.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  memset(out, 0, sizeof(*out));
  out->evals = cnt.evals;
  out->grads = cnt.grads;
  out->ls_trials = cnt.ls_trials;
  out->ls_fail = cnt.ls_fail;
  out->cycles = cnt.cycle;
  out->n_stuck = cnt.n_stuck;
  out->k_lost = cnt.n_removed;
  out->n_unfrozen = cnt.n_unfrozen;
  out->last_reseed = cnt.reseed_mode;
  out->gr_enabled = cnt.gr_enabled;
  out->f_max = cnt.fmax;
  out->sigma = cnt.sigma;
  out->alpha_hlc = cnt.alpha_hlc;
  out->alpha_anti = cnt.alpha_anti;
  out->device_error = cnt.err;
  if (cnt.err != 0) {
    CK(cudaMemsetAsync(&c->probs[prob].dev.cnt->err, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return fail(c, CHISAO_ERR_TIMEOUT, "a device-side wait ran out of its time budget (flag " +
                                           std::to_string(cnt.err) + ", now cleared)");
  }
  return CHISAO_OK;
}

chisao_status chisao_stats(chisao_ctx* c, int32_t prob, chisao_counters* out) {
  return chisao_get_counters(c, prob, out);
}

chisao_status chisao_selftest_wait(chisao_ctx* c, int32_t prob, int64_t budget_ns) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  if (budget_ns < 1 || budget_ns > 10000000000ll) return fail(c, CHISAO_ERR_ARG, "budget_ns out of range");
  CK(tc_wait_selftest(budget_ns, &c->probs[prob].dev.cnt->err, c->stream));
  return CHISAO_OK;
}

chisao_status chisao_eval(chisao_ctx* c, int32_t prob, const float* x_dev, int64_t n, float* f_dev, float* g_dev,
                          int32_t grad_mode) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  if (n < 0 || n > MAX_N || (n > 0 && !x_dev)) return fail(c, CHISAO_ERR_ARG, "bad points");
  if (grad_mode < 0 || grad_mode > 3) return fail(c, CHISAO_ERR_ARG, "unknown grad_mode");
  if (n == 0 || (!f_dev && !g_dev)) return CHISAO_OK;
  const ProbHost& ph = c->probs[prob];
  if (ph.kind == CHISAO_OBJ_EXTERNAL) {
    if (grad_mode != CHISAO_GRAD_ADJOINT) return fail(c, CHISAO_ERR_ARG, "an external objective supplies exact gradients only");
    const int32_t r = ph.ext_eval(ph.ext_user, x_dev, ph.d, n, nullptr, nullptr, f_dev, g_dev, ph.d, c->stream);
    if (r != 0) return fail(c, CHISAO_ERR_CUDA, "the external objective's evaluator returned " + std::to_string(r));
    return CHISAO_OK;
  }
  if (grad_mode == CHISAO_GRAD_ADJOINT_TC) {
    if (ph.kind != CHISAO_OBJ_MIXTURE_FULL) return fail(c, CHISAO_ERR_ARG, "tensor-core mode needs a full-covariance mixture");
    CK(tc_launch_mixfull(x_dev, ph.d, (int)n, ph.d, ph.K, ph.tc_weights, f_dev, g_dev, ph.d, &ph.dev.cnt->err,
                         c->stream, ph.tc_part, ph.tc_ticket));
    return CHISAO_OK;
  }
  EvalArgs ea{x_dev, (int)n, f_dev, g_dev};
  CK(launch_objective(OKID_EVAL, c->probs[prob], grad_mode, 0, &ea, c->stream));
  return CHISAO_OK;
}

const char* chisao_last_error(const chisao_ctx* c) { return c ? c->err.c_str() : "null context"; }

void chisao_destroy(chisao_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->g_mid) cudaGraphExecDestroy(c->g_mid);
  if (c->g_last) cudaGraphExecDestroy(c->g_last);
  free_branches(c);
  for (Group& gr : c->groups)
    if (gr.mem) cudaFree(gr.mem);
  if (c->all_mem) cudaFree(c->all_mem);
  if (c->own_arena && c->arena) cudaFree(c->arena);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

chisao_status chisao_layout(chisao_ctx* c, int32_t prob, int32_t* dp, int32_t* m_max) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  if (dp) *dp = c->probs[prob].dp;
  if (m_max) *m_max = MMAX;
  return CHISAO_OK;
}

static chisao_status field_ptr(chisao_ctx* c, int32_t prob, int32_t field, void** ptr, size_t* bytes) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  ProbHost& ph = c->probs[prob];
  ProbDev& P = ph.dev;
  const size_t n = (size_t)ph.n;
  switch (field) {
    case CHISAO_FIELD_X: *ptr = P.x; *bytes = n * ph.dp * 4; break;
    case CHISAO_FIELD_G: *ptr = P.g; *bytes = n * ph.dp * 4; break;
    case CHISAO_FIELD_F: *ptr = P.f; *bytes = n * 4; break;
    case CHISAO_FIELD_HS: *ptr = P.hs; *bytes = n * MMAX * ph.dp * 4; break;
    case CHISAO_FIELD_HY: *ptr = P.hy; *bytes = n * MMAX * ph.dp * 4; break;
    case CHISAO_FIELD_HRHO: *ptr = P.hrho; *bytes = n * MMAX * 4; break;
    case CHISAO_FIELD_HLEN: *ptr = P.hlen; *bytes = n * 4; break;
    case CHISAO_FIELD_STUCK: *ptr = P.stuck; *bytes = (size_t)P.nwords * 4; break;
    case CHISAO_FIELD_REMOVED: *ptr = P.removed; *bytes = (size_t)P.nwords * 4; break;
    default: return fail(c, CHISAO_ERR_ARG, "unknown field");
  }
  return CHISAO_OK;
}

chisao_status chisao_state_get(chisao_ctx* c, int32_t prob, int32_t field, void* host, size_t bytes) {
  void* p;
  size_t want;
  chisao_status s = field_ptr(c, prob, field, &p, &want);
  if (s != CHISAO_OK) return s;
  if (!host || bytes != want) return fail(c, CHISAO_ERR_ARG, "state_get: size mismatch");
  CK(cudaMemcpyAsync(host, p, bytes, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return CHISAO_OK;
}

chisao_status chisao_state_set(chisao_ctx* c, int32_t prob, int32_t field, const void* host, size_t bytes) {
  void* p;
  size_t want;
  chisao_status s = field_ptr(c, prob, field, &p, &want);
  if (s != CHISAO_OK) return s;
  if (!host || bytes != want) return fail(c, CHISAO_ERR_ARG, "state_set: size mismatch");
  CK(cudaMemcpyAsync(p, host, bytes, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return CHISAO_OK;
}

chisao_status chisao_run_phase(chisao_ctx* c, int32_t prob, int32_t phase, int32_t arg) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  const ProbHost& ph = c->probs[prob];
  cudaStream_t st = c->stream;
  switch (phase) {
    case CHISAO_PHASE_LBFGS:
      if (ph.tc)
        CK(enqueue_phase1_tc(ph, arg < 0 ? -arg : arg, arg >= 0, st));
      else
        CK(launch_objective(OKID_PHASE1, ph, ph.sp.grad_mode, arg, nullptr, st));
      break;
    case CHISAO_PHASE_REFINE:
      CK(enqueue_refine(ph, arg, st));
      break;
    case CHISAO_PHASE_FREEZE:
      CK(launch_cycle_begin(ph.dev, st));
      CK(launch_freeze(ph.dev, ph.sp, st));
      break;
    case CHISAO_PHASE_DEDUP:
      CK(launch_compact_stuck(ph.dev, st));
      CK(launch_dedup(ph.dev, ph.sp, st));
      break;
    case CHISAO_PHASE_LISTS:
      CK(launch_lists(ph.dev, st));
      break;
    case CHISAO_PHASE_RESEED:
      CK(launch_set_cycle(ph.dev, arg - 1, st));
      CK(launch_reseed(ph.dev, ph.sp, st));
      break;
    case CHISAO_PHASE_HLC:
      CK(launch_set_cycle(ph.dev, arg - 1, st));
      if (ph.tc) {
        CK(enqueue_hlc_tc(ph, st));
        break;
      }
      CK(launch_objective(OKID_SCALES, ph, ph.sp.grad_mode, 0, nullptr, st));
      CK(launch_finalize_scales(ph.dev, ph.sp, 0, st));
      CK(launch_objective(OKID_HLC, ph, ph.sp.grad_mode, 0, nullptr, st));
      break;
    case CHISAO_PHASE_ANTI:
      if (ph.tc) {
        CK(enqueue_anti_tc(ph, st));
        break;
      }
      CK(launch_objective(OKID_SCALES, ph, ph.sp.grad_mode, 0, nullptr, st));
      CK(launch_finalize_scales(ph.dev, ph.sp, 1, st));
      CK(launch_objective(OKID_ANTI, ph, ph.sp.grad_mode, 0, nullptr, st));
      break;
    case CHISAO_PHASE_DIRECTION:
      CK(launch_objective(OKID_DIRECTION, ph, ph.sp.grad_mode, 0, nullptr, st));
      break;
    default:
      return fail(c, CHISAO_ERR_ARG, "unknown phase");
  }
  return CHISAO_OK;
}

chisao_status chisao_set_tile(chisao_ctx* c, int32_t dp, int32_t ck) {
  if (!c) return CHISAO_ERR_ARG;
  int tile = -1;
  for (int t = 0; t < MIXDIAG_TILES; ++t)
    if (MIXDIAG_TILE_CK[t] == ck) tile = t;
  if (tile < 0) return fail(c, CHISAO_ERR_ARG, "components per step must be 2, 4 or 8");
  bool found = false;
  for (Group& gr : c->groups)
    if (gr.kind == CHISAO_OBJ_MIXTURE_DIAG && gr.dp == dp) {
      gr.tile = tile;
      found = true;
    }
  if (!found) return fail(c, CHISAO_ERR_ARG, "no grouped diagonal mixtures of that padded dimension");
  CK(cudaStreamSynchronize(c->stream));
  if (c->g_mid) cudaGraphExecDestroy(c->g_mid);       // recaptured at the next step
  if (c->g_last) cudaGraphExecDestroy(c->g_last);
  c->g_mid = c->g_last = nullptr;
  return CHISAO_OK;
}

chisao_status chisao_set_gr_state(chisao_ctx* c, int32_t prob, int32_t enabled, int32_t noprog, int32_t prev_surv) {
  chisao_status s = check_prob(c, prob);
  if (s != CHISAO_OK) return s;
  CK(cudaStreamSynchronize(c->stream));
  Counters cnt;
  Counters* dptr = c->probs[prob].dev.cnt;
  CK(cudaMemcpy(&cnt, dptr, sizeof(cnt), cudaMemcpyDeviceToHost));
  cnt.gr_enabled = enabled;
  cnt.gr_noprog = noprog;
  cnt.gr_prev_surv = prev_surv;
  CK(cudaMemcpy(dptr, &cnt, sizeof(cnt), cudaMemcpyHostToDevice));
  return CHISAO_OK;
}

}  // extern "C"

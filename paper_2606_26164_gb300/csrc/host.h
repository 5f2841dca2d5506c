// Internal host-side declarations shared by the C ABI and the kernel files.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "dev_common.cuh"

namespace chisao {

// objective-dependent kernels (one translation unit per objective kind)
// The scale-pass finalization of every problem of a group (T: its scale-pass table).
cudaError_t launch_finalize_grp(const GroupTab& T, int members, int dp, int which, cudaStream_t st);
// Measured FMA throughput (FLOP/s, 2 per FMA) in binary32 (f64 = 0) or binary64.
cudaError_t measure_fma_peak(int f64, double* flops, cudaStream_t st);
// Zero the padding coordinates d .. dp-1 of rows x dp gradient rows.
cudaError_t launch_zero_padding(float* g, long long rows, int d, int dp, cudaStream_t st);
// Blocks of a per-sample objective kernel over n samples of padded dimension dp.
unsigned obj_blocks(long long n, int dp);
// Grouped launches of Phase 1 / 5 / 6 (OKID_PHASE1, OKID_HLC, OKID_ANTI) with exact gradients
// over the problems of one group (same objective kind and padded dimension dp).
cudaError_t launch_grp_mixdiag(int which, int dp, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0);
// the same at a tile shape: 0 = 4 components per step (launch_grp_mixdiag), 1 = 2, 2 = 8
constexpr int MIXDIAG_TILES = 3;
constexpr int MIXDIAG_TILE_CK[MIXDIAG_TILES] = {4, 2, 8};
cudaError_t launch_grp_mixdiag_tile(int which, int dp, int tile, const GroupTab& T, unsigned blocks,
                                    cudaStream_t st, int arg = 0);
cudaError_t launch_grp_mixfull(int which, int dp, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0);
cudaError_t launch_grp_quad(int which, int dp, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0);
cudaError_t launch_grp_bench(int which, int dp, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0);
cudaError_t launch_grp_bench_4(int which, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0);
cudaError_t launch_grp_bench_8(int which, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0);
cudaError_t launch_grp_bench_16(int which, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0);
cudaError_t launch_grp_bench_32(int which, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0);
cudaError_t launch_grp_bench_64(int which, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg = 0);
cudaError_t launch_obj_mixdiag(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                               const EvalArgs* ea, cudaStream_t st);
cudaError_t launch_obj_mixfull(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                               const EvalArgs* ea, cudaStream_t st);
cudaError_t launch_obj_quad(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                            const EvalArgs* ea, cudaStream_t st);
cudaError_t launch_obj_bench(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                             const EvalArgs* ea, cudaStream_t st);
cudaError_t launch_obj_bench_4(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                                 const EvalArgs* ea, cudaStream_t st);
cudaError_t launch_obj_bench_8(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                                 const EvalArgs* ea, cudaStream_t st);
cudaError_t launch_obj_bench_16(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                                 const EvalArgs* ea, cudaStream_t st);
cudaError_t launch_obj_bench_32(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                                 const EvalArgs* ea, cudaStream_t st);
cudaError_t launch_obj_bench_64(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                                 const EvalArgs* ea, cudaStream_t st);

// objective-independent kernels
cudaError_t launch_cycle_begin(const ProbDev& P, cudaStream_t st);
cudaError_t launch_cycle_end(const ProbDev& P, cudaStream_t st);
cudaError_t launch_set_cycle(const ProbDev& P, int completed, cudaStream_t st);
cudaError_t launch_freeze(const ProbDev& P, const StepParams& S, cudaStream_t st);
cudaError_t launch_compact_stuck(const ProbDev& P, cudaStream_t st);
cudaError_t launch_lists(const ProbDev& P, cudaStream_t st);
cudaError_t launch_seed(const ProbDev& P, const StepParams& S, int method, cudaStream_t st);
cudaError_t launch_dedup(const ProbDev& P, const StepParams& S, cudaStream_t st);
cudaError_t launch_reseed(const ProbDev& P, const StepParams& S, cudaStream_t st);
cudaError_t launch_finalize_scales(const ProbDev& P, const StepParams& S, int which, cudaStream_t st);
cudaError_t launch_gather_modes(const ProbDev& P, float* xo, float* fo, cudaStream_t st);
cudaError_t prepare_kernel_attributes();

// Phases 1, 5 and 6 around a batched evaluator (ext_kernels.cu)
// Laplace widths of the first n_surv survivors (l_surv order): w[r][j] = sqrt(H_jj),
// cov[r][j][:] = H e_j when cov is not null (H the sample's L-BFGS inverse-Hessian
// estimate); rows is the host's count of survivors (the grid size).
cudaError_t launch_widths(const ProbDev& P, int rows, float* w, float* cov, cudaStream_t st);
cudaError_t launch_ext(int which, const ProbDev& P, const StepParams& S, const ExtBuf& E, int arg,
                       cudaStream_t st);

// tensor-core (tcgen05, BF16) full-covariance mixture objective
cudaError_t tc_prepare_attributes();
// A bounded wait that runs out (budget_ns of the global timer) and raises *err = 2.
cudaError_t tc_wait_selftest(long long budget_ns, int* err, cudaStream_t st);
// Clocks per tcgen05.mma (M = 128, K = 16, width n) with `threads` issuers together.
cudaError_t tc_measure_mma_rate(int n, int threads, int tmem_a, double* clk_per_mma, cudaStream_t st);
size_t tc_weight_bytes(int K);     // operand tiles of all component groups
size_t tc_split_floats();          // partial results of a component-split launch
size_t tc_split_tickets();         // its per-tile arrival counters
void tc_build_weights(int K, int d, const double* linv, const double* mu, const double* logw,
                      std::vector<uint8_t>& out);
// n: rows (or the capacity when count is given); idx/count: optional row list and device count;
// part/ticket: the component-split scratch (null: every CTA takes a whole tile)
cudaError_t tc_launch_mixfull(const float* x, int ldx, int n, int d, int K, const uint8_t* weights,
                              float* f, float* g, int ldg, int* err, cudaStream_t st, float* part,
                              int* ticket, const int* idx = nullptr, const int* count = nullptr);
int scale_blocks(const ProbDev& P);
size_t gr_qr_smem(int d);

// Launch tables of the objective-independent kernels of a cycle over all problems of a
// context (phase_kernels.cu): one grouped launch per kernel instead of one per problem,
// each problem running the blocks its own launch would.
struct AllTabs {
  AllTab begin, fmax, lin, one, hclear, hspread;   // one entry per problem
  AllTab dp2[5];                                   // problems of padded dimension 4 << k
  unsigned nb_begin = 0, nb_fmax = 0, nb_lin = 0, nb_one = 0, nb_hclear = 0, nb_hspread = 0, nb_dp2[5] = {};
  size_t qr_smem = 0;                              // the Golden Rooster QR's shared memory
};
// Builds the tables in one device allocation *mem (the caller frees it).
cudaError_t build_all_tabs(const std::vector<ProbDev>& pd, const std::vector<StepParams>& sp, void** mem,
                           AllTabs* out);
cudaError_t launch_cycle_begin_all(const AllTabs& A, cudaStream_t st);
cudaError_t launch_cycle_end_all(const AllTabs& A, cudaStream_t st);
cudaError_t launch_freeze_all(const AllTabs& A, cudaStream_t st);   // Phase 2: f_max, stick mask, stuck list
cudaError_t launch_dedup_all(const AllTabs& A, cudaStream_t st);    // Phase 3 and the sample lists
cudaError_t launch_reseed_all(const AllTabs& A, cudaStream_t st);   // Phase 4

}  // namespace chisao

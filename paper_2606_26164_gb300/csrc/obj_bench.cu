// The benchmark functions' kernels, one translation unit per padded dimension.
#include "host.h"

namespace chisao {

cudaError_t launch_obj_bench(int which, int gm, const ProbDev& P, const StepParams& S, int arg, const EvalArgs* ea,
                             cudaStream_t st) {
  switch (P.dp) {
    case 4: return launch_obj_bench_4(which, gm, P, S, arg, ea, st);
    case 8: return launch_obj_bench_8(which, gm, P, S, arg, ea, st);
    case 16: return launch_obj_bench_16(which, gm, P, S, arg, ea, st);
    case 32: return launch_obj_bench_32(which, gm, P, S, arg, ea, st);
    case 64: return launch_obj_bench_64(which, gm, P, S, arg, ea, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_grp_bench(int which, int dp, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg) {
  switch (dp) {
    case 4: return launch_grp_bench_4(which, T, blocks, st, arg);
    case 8: return launch_grp_bench_8(which, T, blocks, st, arg);
    case 16: return launch_grp_bench_16(which, T, blocks, st, arg);
    case 32: return launch_grp_bench_32(which, T, blocks, st, arg);
    case 64: return launch_grp_bench_64(which, T, blocks, st, arg);
  }
  return cudaErrorInvalidValue;
}

}  // namespace chisao

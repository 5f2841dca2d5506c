// Instantiation of the objective-dependent kernels for the benchmark functions at one
// padded dimension (the five dimensions compile in parallel).
#include "host.h"
#include "obj_kernels.cuh"

namespace chisao {

cudaError_t launch_obj_bench_64(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                                 const EvalArgs* ea, cudaStream_t st) {
  return launch_obj_dp<OBJ_BENCH, 64>(which, gm, P, S, arg, ea, st);
}

cudaError_t launch_grp_bench_64(int which, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg) {
  return launch_grp_dp<OBJ_BENCH, 64>(which, T, blocks, st, arg);
}

}  // namespace chisao

// Instantiation of the objective-dependent kernels for one objective kind
// (one translation unit per kind keeps the parallel build short).
#include "host.h"
#include "obj_kernels.cuh"

namespace chisao {

cudaError_t launch_obj_mixfull(int which, int gm, const ProbDev& P, const StepParams& S, int arg, const EvalArgs* ea,
                         cudaStream_t st) {
  return launch_obj<OBJ_MIXTURE_FULL>(which, gm, P, S, arg, ea, st);
}

cudaError_t launch_grp_mixfull(int which, int dp, const GroupTab& T, unsigned blocks, cudaStream_t st, int arg) {
  return launch_grp<OBJ_MIXTURE_FULL>(which, dp, T, blocks, st, arg);
}

}  // namespace chisao

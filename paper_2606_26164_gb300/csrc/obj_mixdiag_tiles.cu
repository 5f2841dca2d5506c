// Grouped launches of the diagonal mixture at the other component steps (2 and 8 per
// step; obj_mixdiag.cu has the default 4), in their own translation unit so the build
// compiles them in parallel.  The tuner of batched contexts picks one per group.
#include "host.h"
#include "obj_kernels.cuh"

namespace chisao {

cudaError_t launch_grp_mixdiag_tile(int which, int dp, int tile, const GroupTab& T, unsigned blocks,
                                    cudaStream_t st, int arg) {
  switch (tile) {
    case 0: return launch_grp_mixdiag(which, dp, T, blocks, st, arg);
    case 1: return launch_grp<OBJ_MIXDIAG_C2>(which, dp, T, blocks, st, arg);
    case 2: return launch_grp<OBJ_MIXDIAG_C8>(which, dp, T, blocks, st, arg);
  }
  return cudaErrorInvalidValue;
}

}  // namespace chisao

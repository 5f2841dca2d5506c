// Internal host-side declarations shared by the C ABI and the kernel files.
#pragma once
#include <cuda_runtime.h>

#include "dev_common.cuh"

namespace chisao {

// objective-dependent kernels (one translation unit per objective kind)
cudaError_t launch_obj_mixdiag(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                               const EvalArgs* ea, cudaStream_t st);
cudaError_t launch_obj_mixfull(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                               const EvalArgs* ea, cudaStream_t st);
cudaError_t launch_obj_quad(int which, int gm, const ProbDev& P, const StepParams& S, int arg,
                            const EvalArgs* ea, cudaStream_t st);

// objective-independent kernels
cudaError_t launch_cycle_begin(const ProbDev& P, cudaStream_t st);
cudaError_t launch_cycle_end(const ProbDev& P, cudaStream_t st);
cudaError_t launch_set_cycle(const ProbDev& P, int completed, cudaStream_t st);
cudaError_t launch_freeze(const ProbDev& P, const StepParams& S, cudaStream_t st);
cudaError_t launch_compact_stuck(const ProbDev& P, cudaStream_t st);
cudaError_t launch_lists(const ProbDev& P, cudaStream_t st);
cudaError_t launch_dedup(const ProbDev& P, const StepParams& S, cudaStream_t st);
cudaError_t launch_reseed(const ProbDev& P, const StepParams& S, cudaStream_t st);
cudaError_t launch_finalize_scales(const ProbDev& P, const StepParams& S, int which, cudaStream_t st);
cudaError_t launch_gather_modes(const ProbDev& P, float* xo, float* fo, cudaStream_t st);
cudaError_t prepare_kernel_attributes();
int scale_blocks(const ProbDev& P);
size_t gr_qr_smem(int d);

}  // namespace chisao

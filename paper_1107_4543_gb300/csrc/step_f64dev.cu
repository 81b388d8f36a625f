// LBM_F64DEV instantiation of the deviation-storage step kernel
// (step_impl.cuh): FP64 deviations, FP64 collision with fused multiply-adds.
#include "step_impl.cuh"

namespace lbm {

cudaError_t launch_step_dev_f64dev(const Lattice &L, const void *src, void *dst, cudaStream_t st,
                                   int block, int variant) {
  return launch_step_dev_t<double>(L, src, dst, st, block, variant);
}

}  // namespace lbm

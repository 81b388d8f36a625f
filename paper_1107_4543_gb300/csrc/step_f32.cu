// Step kernels for one storage type (float); see step_impl.cuh.
#define LBM_TABLE_DEV  // this unit holds its type's constant table
#include "step_impl.cuh"

namespace lbm {

cudaError_t launch_step_dev_f32(const Lattice &L, const void *src, void *dst, cudaStream_t st,
                              int block, int variant) {
  return launch_step_dev_t<float>(L, src, dst, st, block, variant);
}

cudaError_t launch_step_batch_f32(const BatchList &bl, int parity, cudaStream_t st, int block,
                                  int variant, const int *limits, int k) {
  return launch_step_batch_t<float>(bl, parity, st, block, variant, limits, k);
}

cudaError_t upload_batch_consts_f32(const BatchEntry *ents, int n, int pbase, void *stage,
                                    cudaStream_t st) {
  return upload_consts_t<float>(ents, n, pbase, stage, st);
}

cudaError_t launch_batch_resident_f32(const BatchEntry *ents, const int *idx, int nres,
                                      int nents, size_t smem, int parity, long steps,
                                      const int *limits, cudaStream_t st) {
  return launch_resident_t<float>(ents, idx, nres, nents, smem, parity, steps, limits, st);
}

unsigned bounds_word_step_f32(bool reset) { return bounds::read_word(reset); }

}  // namespace lbm

// Step kernels for one storage type (__half); see step_impl.cuh.
#define LBM_TABLE_PAIRS  // this unit holds its type's constant table
#include "step_impl.cuh"

namespace lbm {

cudaError_t launch_step_dev_f16(const Lattice &L, const void *src, void *dst, cudaStream_t st,
                              int block, int variant) {
  return launch_step_dev_t<__half>(L, src, dst, st, block, variant);
}

cudaError_t launch_step_batch_f16(const BatchList &bl, int parity, cudaStream_t st, int block,
                                  int variant, const int *limits, int k) {
  return launch_step_batch_t<__half>(bl, parity, st, block, variant, limits, k);
}

cudaError_t upload_batch_consts_f16(const BatchEntry *ents, int n, int pbase, void *stage,
                                   cudaStream_t st) {
  return upload_consts_t<__half>(ents, n, pbase, stage, st);
}

cudaError_t launch_batch_resident_f16(const BatchEntry *ents, const int *idx, int nres,
                                      int nents, size_t smem, int parity, long steps,
                                      const int *limits, cudaStream_t st) {
  return launch_resident_t<__half>(ents, idx, nres, nents, smem, parity, steps, limits, st);
}

unsigned bounds_word_step_f16(bool reset) { return bounds::read_word(reset); }

}  // namespace lbm

// Internal declarations shared by the translation units of liblbm.so.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "collide.cuh"
#include "d2q9_pull.cuh"

namespace lbm {

// NVTX range for the lifetime of a scope: step chunks, batch steps, host I/O
// and serving generations show up by name in a profiler's timeline
// (header-only NVTX; without a profiler attached the calls do nothing).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};


// Make device d current for the lifetime of a scope (restored afterwards).
struct DevGuard {
  int prev = -1, want;
  explicit DevGuard(int d) : want(d) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != d) cudaSetDevice(d);
  }
  ~DevGuard() {
    if (prev >= 0 && prev != want) cudaSetDevice(prev);
  }
  DevGuard(const DevGuard &) = delete;
  DevGuard &operator=(const DevGuard &) = delete;
};

// Everything a step launch needs about one lattice.
struct Lattice {
  Geom g;
  int dtype;
  int V;             // nodes per vector (vec_nodes)
  int variant;       // launch variant of the step kernel (tuner)
  int esize;         // bytes per stored population
  void *buf[2];      // double buffer (each 9 planes)
  int cur;           // buffer holding the current state
  DevParams dp;      // deviation types stored in 32 or 16 bits
  DevParams64 dp64;  // LBM_F64DEV
  F64Params fp;      // LBM_F64
};

// Per-lattice work list entry of the batched step (device memory).
struct BatchEntry {
  Geom g;
  DevParams dp;
  void *buf[2];
  int off;           // buffer index holding the state when the batch began
};

// One block of a batch's plain grid: every lattice starts on a block
// boundary, and each block carries its lattice's geometry and buffers, so a
// warp finds its work with one load and no search; the relaxation
// parameters (needed only by the collision) come from the lattice's entry.
struct BlockRec {
  Geom g;
  void *buf[2];
  long long task_base;  // lattice task of the block's warp 0
  int lat;              // lattice index in the entry list
  int off;              // as BatchEntry::off
};

// Device work list of one storage type's batch members: per-lattice
// entries and the plain grid's block records (the persistent grids stride
// over the same records).
struct BatchList {
  const BatchEntry *ents;
  int n;
  int pbase = -1;  // first slot of the type's constant table, or -1 (entries)
  const BlockRec *blocks;  // the plain grid's blocks
  long long nblocks;       // sum over lattices of ceil(tasks / warps per block)
  long long ntasks;        // sum of the lattices' tasks
};

// launch helpers (step_f32.cu, step_f16.cu, step_bf16.cu, step_f64.cu).
// `variant` selects the register cap of the deviation step kernels
// (0, 1, 2: at least 1, 2, 3 resident 256-thread blocks per SM).
constexpr int kStepVariants = 3;
// batched launches add kStepVariants persistent variants (the same register
// caps, a grid of MINB blocks per SM striding over the block records)
constexpr int kBatchVariants = 2 * kStepVariants;
cudaError_t launch_step_dev_f32(const Lattice &L, const void *src, void *dst, cudaStream_t st,
                                int block, int variant);
cudaError_t launch_step_dev_f16(const Lattice &L, const void *src, void *dst, cudaStream_t st,
                                int block, int variant);
cudaError_t launch_step_dev_bf16(const Lattice &L, const void *src, void *dst, cudaStream_t st,
                                 int block, int variant);
cudaError_t launch_step_dev_f64dev(const Lattice &L, const void *src, void *dst, cudaStream_t st,
                                   int block, int variant);
cudaError_t launch_step_batch_f32(const BatchList &bl, int parity, cudaStream_t st, int block,
                                  int variant, const int *limits, int k);
cudaError_t launch_step_batch_f16(const BatchList &bl, int parity, cudaStream_t st, int block,
                                  int variant, const int *limits, int k);
cudaError_t launch_step_batch_bf16(const BatchList &bl, int parity, cudaStream_t st, int block,
                                   int variant, const int *limits, int k);
// Constant-memory tables of the batched step's per-lattice collision
// constants, one per storage type and device (step_impl.cuh): the 16-bit
// types keep PC_COUNT broadcast floats per lattice (kPairSlots lattices,
// 61,440 bytes of the 64 KB constant bank), FP32 whole DevParams records
// (kDevSlots lattices, 64,000 bytes).  upload_batch_consts writes slots
// pbase .. pbase + n - 1 from the entries' parameters through `stage`
// (n * const_slot_bytes(dtype) bytes of device memory) in the order of
// stream st.
constexpr int kPairSlots = 960;
constexpr int kDevSlots = 640;
inline int const_slots(int dtype) {
  return dtype == LBM_F32DEV ? kDevSlots
                             : (dtype == LBM_F16DEV || dtype == LBM_BF16DEV ? kPairSlots : 0);
}
inline size_t const_slot_bytes(int dtype) {
  return dtype == LBM_F32DEV ? sizeof(DevParams) : PC_COUNT * sizeof(float);
}
cudaError_t upload_batch_consts_f32(const BatchEntry *ents, int n, int pbase, void *stage,
                                    cudaStream_t st);
cudaError_t upload_batch_consts_f16(const BatchEntry *ents, int n, int pbase, void *stage,
                                    cudaStream_t st);
cudaError_t upload_batch_consts_bf16(const BatchEntry *ents, int n, int pbase, void *stage,
                                     cudaStream_t st);
inline cudaError_t upload_batch_consts(int dtype, const BatchEntry *ents, int n, int pbase,
                                       void *stage, cudaStream_t st) {
  switch (dtype) {
    case LBM_F32DEV: return upload_batch_consts_f32(ents, n, pbase, stage, st);
    case LBM_F16DEV: return upload_batch_consts_f16(ents, n, pbase, stage, st);
    case LBM_BF16DEV: return upload_batch_consts_bf16(ents, n, pbase, stage, st);
    default: return cudaSuccess;
  }
}
cudaError_t launch_step_f64(const Lattice &L, const void *src, void *dst,
                            cudaStream_t st, int block, int grid_cap);

inline cudaError_t launch_step_dev(const Lattice &L, const void *src, void *dst,
                                   cudaStream_t st, int block, int variant) {
  switch (L.dtype) {
    case LBM_F32DEV: return launch_step_dev_f32(L, src, dst, st, block, variant);
    case LBM_F16DEV: return launch_step_dev_f16(L, src, dst, st, block, variant);
    case LBM_BF16DEV: return launch_step_dev_bf16(L, src, dst, st, block, variant);
    case LBM_F64DEV: return launch_step_dev_f64dev(L, src, dst, st, block, variant);
    default: return cudaErrorInvalidValue;
  }
}

inline cudaError_t launch_step_batch(int dtype, const BatchList &bl, int parity, cudaStream_t st,
                                     int block, int variant, const int *limits = nullptr,
                                     int k = 0) {
  switch (dtype) {
    case LBM_F32DEV: return launch_step_batch_f32(bl, parity, st, block, variant, limits, k);
    case LBM_F16DEV: return launch_step_batch_f16(bl, parity, st, block, variant, limits, k);
    case LBM_BF16DEV: return launch_step_batch_bf16(bl, parity, st, block, variant, limits, k);
    default: return cudaErrorInvalidValue;
  }
}

// Batch members small enough to stay in shared memory for all the steps of
// a launch (k_batch_resident, resident.cuh): both step buffers of 9 compact
// planes.  resident_limit: the device's shared memory per block, lowered by
// the environment variable LBM_RESIDENT_BYTES (0 turns resident members off).
inline size_t resident_bytes(int nx, int ny, int esize) {
  return (size_t)2 * 9 * (size_t)nx * (size_t)ny * (size_t)esize;
}
size_t resident_limit(int device);
cudaError_t launch_batch_resident_f32(const BatchEntry *ents, const int *idx, int nres,
                                      int nents, size_t smem, int parity, long steps,
                                      const int *limits, cudaStream_t st);
cudaError_t launch_batch_resident_f16(const BatchEntry *ents, const int *idx, int nres,
                                      int nents, size_t smem, int parity, long steps,
                                      const int *limits, cudaStream_t st);
cudaError_t launch_batch_resident_bf16(const BatchEntry *ents, const int *idx, int nres,
                                      int nents, size_t smem, int parity, long steps,
                                      const int *limits, cudaStream_t st);
inline cudaError_t launch_batch_resident(int dtype, const BatchEntry *ents, const int *idx,
                                         int nres, int nents, size_t smem, int parity,
                                         long steps, const int *limits, cudaStream_t st) {
  switch (dtype) {
    case LBM_F32DEV:
      return launch_batch_resident_f32(ents, idx, nres, nents, smem, parity, steps, limits, st);
    case LBM_F16DEV:
      return launch_batch_resident_f16(ents, idx, nres, nents, smem, parity, steps, limits, st);
    case LBM_BF16DEV:
      return launch_batch_resident_bf16(ents, idx, nres, nents, smem, parity, steps, limits,
                                        st);
    default: return cudaErrorInvalidValue;
  }
}

// Nodes per vector of a storage type (host side of d2q9_pull.cuh's Elem).
inline int vec_nodes(int dtype) {
  return dtype == LBM_F64 || dtype == LBM_F64DEV ? 2
         : dtype == LBM_F32DEV ? 4
         : dtype == LBM_F16DEV ? LBM_VF16 : LBM_VBF16;
}

// aux kernels (aux.cu)
struct AuxView {
  Geom g;
  int dtype;
  void *buf;          // current buffer
  double rho0, jx0, jy0;
  double f0[9];       // base populations f^eq(rho0, j0) (deviation types)
  double scale;       // stored = f' * scale (FP16), 1 otherwise
};
// FP16 storage scale for a largest |f'| of maxabs (host and device alike):
// 2^(14 - ceil(log2 maxabs)), clamped to 2^-100 .. 2^100, so stored values
// stay near 2^14 -- 11-bit mantissas with 4x headroom below the largest
// finite FP16 and no subnormals down to 2^-10 of the largest; 1 for a zero
// or non-finite maxabs
__host__ __device__ inline double fp16_scale(double maxabs) {
  if (!(maxabs > 0.0) || isinf(maxabs)) return 1.0;
  int e = 0;
  const double f = frexp(maxabs, &e);  // maxabs = f 2^e, f in [0.5, 1)
  int k = 14 - (f == 0.5 ? e - 1 : e);  // 14 - ceil(log2 maxabs)
  k = k < -100 ? -100 : (k > 100 ? 100 : k);
  return ldexp(1.0, k);
}

cudaError_t launch_init_eq(const AuxView &a, const double *rho, const double *ux,
                           const double *uy, int analytic_kind, const double *params,
                           cudaStream_t st, unsigned int *bad = nullptr);
cudaError_t launch_maxdev_eq(const AuxView &a, const double *rho, const double *ux,
                             const double *uy, int analytic_kind, const double *params,
                             unsigned int *max_bits, cudaStream_t st);
cudaError_t launch_moments(const AuxView &a, double *rho, double *ux, double *uy,
                           cudaStream_t st);
// deviation storage types: equilibrium deviations formed from the
// O(perturbation) differences to the reference state (io_dev.cu)
cudaError_t launch_init_dev(const AuxView &a, const double *rho, const double *ux,
                            const double *uy, cudaStream_t st, unsigned int *bad);
cudaError_t launch_maxdev_dev(const AuxView &a, const double *rho, const double *ux,
                              const double *uy, unsigned int *max_bits, cudaStream_t st);
cudaError_t launch_moments_dev(const AuxView &a, double *rho, double *ux, double *uy,
                               cudaStream_t st);
// batched field I/O of a batch's deviation-storage members (one launch for
// all members): block b covers nodes [start, start + count) of `member`
struct IoBlock {
  int member;
  int count;
  long long start;
};
constexpr int kIoBlockNodes = 1024;
// FP16 members of a pipelined solve: the largest |f'| of each member's
// equilibrium from the staged fields (max_bits: float bits, zeroed first),
// then each member's storage scale (fp16_scale of that, or of floor[k] if
// larger) written into both drift/I-O views, the member's batch entry
// (ent[k]) and scale_out[k]
cudaError_t launch_batch_fp16_scales(AuxView *views0, AuxView *views1, BatchEntry *const *ent,
                                     const IoBlock *blocks, long long nblocks,
                                     const long long *poff, long long total, const double *stage,
                                     unsigned int *max_bits, const double *floor_,
                                     double *scale_out, int members, cudaStream_t st);
cudaError_t launch_batch_init_dev(const AuxView *views, const IoBlock *blocks, long long nblocks,
                                  const long long *poff, long long total, const double *stage,
                                  unsigned int *bad, int members, cudaStream_t st);
cudaError_t launch_batch_moments_dev(const AuxView *views, const IoBlock *blocks,
                                     long long nblocks, const long long *poff, long long total,
                                     double *stage, int members, cudaStream_t st);

// debug build (-DLBM_DEBUG_BOUNDS): each translation unit's index-check word
// (bounds.cuh), optionally cleared; 0 without the flag
unsigned bounds_word_vn(bool reset);
unsigned bounds_word_opt(bool reset);
unsigned bounds_word_step_f32(bool reset);
unsigned bounds_word_step_f16(bool reset);
unsigned bounds_word_step_bf16(bool reset);
unsigned bounds_word_io(bool reset);
cudaError_t launch_bounds_selftest(unsigned int *one, cudaStream_t st);
cudaError_t launch_force_node(const AuxView &a, int x, int y, const double fs[9],
                              cudaStream_t st);
cudaError_t launch_force_node_tab(const AuxView &a, int x, int y, const double *fs_dev,
                                  cudaStream_t st);
cudaError_t launch_get_pop(const AuxView &a, double *f, cudaStream_t st);
cudaError_t launch_set_pop(const AuxView &a, const double *f, cudaStream_t st);
cudaError_t launch_maxdev_pop(const AuxView &a, const double *f, unsigned int *max_bits,
                              cudaStream_t st);
int drift_blocks();
cudaError_t launch_drift(const AuxView &a, double *partials, double *out,
                         cudaStream_t st);
int batch_drift_partials(int n);
cudaError_t launch_add_u32(unsigned int *acc, const unsigned int *add, int n, cudaStream_t st);
cudaError_t launch_batch_drift(const AuxView *views_dev, int n, double *partials, double *out,
                               cudaStream_t st);

// base populations f^eq(rho0, j0) on the host, in the canonical FP64 order
void host_feq_j(double rho, double jx, double jy, double out[9]);

// batch launch-variant control (batch.cu), for the server
void batch_pin_variant(lbm_batch_ctx *b, int variant);
// One generation of a server batch: member k advances min(steps[k], n)
// steps (n launches; a member's warps return once it is done).  The batch
// can only be destroyed afterwards.
int batch_step_ragged(lbm_batch_ctx *b, const long *steps, long n);
int batch_variant(const lbm_batch_ctx *b);
long long batch_nodes(const lbm_batch_ctx *b);

// lattice handles (lbm_api.cu): the constructor behind lbm_create, with
// halo rows for the slabs of a split lattice, and what the slab driver
// (slabs.cu) reads of a handle
int create_lattice(int nx, int ny, const double S[9], double rho0, const double u0[2],
                   int storage_dtype, bool halo, lbm_handle *out);
Lattice &lattice_of(lbm_handle h);
int block_of(lbm_handle h);
bool is_slab(lbm_handle h);
cudaStream_t stream_of(lbm_handle h);
int device_of(lbm_handle h);
void advance_one(lbm_handle h);  // after one step launched by the slab driver

// device memory through the configurable allocator
void *dev_alloc(size_t bytes);
void dev_free(void *p);

void set_error(const std::string &msg);
int sm_count();

}  // namespace lbm

// Fused pull-stream + MRT collide step for the deviation storage types
// (FP32, FP16 scaled, BF16; FP32 collision), single lattice and batched.
// Template implementation; step_f32.cu, step_f16.cu and step_bf16.cu each
// instantiate one storage type (parallel compilation).
//
// One time step of section 2.1 (Eq. blbs) per launch: each warp task pulls
// the 9 populations of 32 x V nodes with 16-byte loads, collides them in
// registers (collide_dev) and stores them with 16-byte stores.  Per node
// the kernel moves 9 reads + 9 writes of one stored population (72 B in
// FP32, 36 B in FP16/BF16): an HBM-bound stream with ~110 FP32 operations
// per node.
#pragma once
#include <type_traits>

#include "bounds.cuh"
#include "lbm_internal.h"

namespace lbm {

// collision parameters of a storage type: FP32 constants (hi + lo pairs
// for FP32 storage) for the 32- and 16-bit types, FP64 ones for LBM_F64DEV
template <typename T> struct ParamsOf { using type = DevParams; };
template <> struct ParamsOf<double> { using type = DevParams64; };

// The batched step's per-lattice collision constants in constant memory:
// each batch owns a range of the slots of its storage type's table (one
// table per translation unit and device) and refreshes it from its entries
// before it steps.  The 16-bit types keep the PC_COUNT broadcast constants
// of the pair collision (PairConst order).  Read at a block-uniform index,
// the constants take the constant cache's path instead of global loads
// held in registers across the task: spills of the FP16 step at 80
// registers 148 -> 84 bytes, the 512-lattice FP16 batch 5.76 -> 6.14 TB/s.
// FP32 keeps the lattice's DevParams itself (hi + lo constants, read by
// collide_dev through a reference into the table).  A translation unit holds
// one full-size table (the constant bank has 64 KB): step_f32.cu defines
// LBM_TABLE_DEV, step_f16.cu and step_bf16.cu LBM_TABLE_PAIRS, before they
// include this file; the other table shrinks to one element there.
#if defined(LBM_TABLE_DEV)
constexpr int kDevTable = kDevSlots, kPairTable = 1;
#elif defined(LBM_TABLE_PAIRS)
constexpr int kDevTable = 1, kPairTable = kPairSlots;
#else
constexpr int kDevTable = 1, kPairTable = 1;
#endif
static __constant__ float c_pairs[kPairTable * PC_COUNT];
static __constant__ DevParams c_dev[kDevTable];

struct ConstPairs {
  int base;  // first constant of the lattice: slot * PC_COUNT
  __device__ __forceinline__ F2 operator()(PairConst c) const { return f2s(c_pairs[base + c]); }
};

// 16-bit storage: unpack / collide / repack the packed populations two
// nodes at a time (9 x V floats per lane would not fit the register
// budget); the word's two nodes collide together, one per lane of the
// packed FP32 pair instructions.  FP16 is stored scaled and collided in the
// scaled units.
template <typename T, typename K>
__device__ __forceinline__ void collide_packed(uint32_t (&w)[9][Elem<T>::V / 2], const K &P) {
  constexpr bool SCALED = std::is_same<T, __half>::value;
#pragma unroll
  for (int k = 0; k < Elem<T>::V / 2; ++k) {
    F2 f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      float t[2];
      Elem<T>::unpack2(w[i][k], t);
      f[i] = f2(t[0], t[1]);
    }
    collide_pair<SCALED>(f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7], f[8], P);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      float t[2];
      f2split(f[i], t[0], t[1]);
      w[i][k] = Elem<T>::pack2(t[0], t[1]);
    }
  }
}

// The collision constants of a 16-bit task: a DevParams, or the lattice's
// slot of the constant table
__device__ __forceinline__ ParamPairs pairs_of(const DevParams &P) { return ParamPairs{P}; }
__device__ __forceinline__ const ConstPairs &pairs_of(const ConstPairs &P) { return P; }

// P: the lattice's ParamsOf<T>::type, or (16-bit types) a ConstPairs
template <typename T, typename PS>
__device__ __forceinline__ void step_task(const T *__restrict__ src, T *__restrict__ dst,
                                          const Geom &g, const PS &P, long long task, int lane) {
  constexpr int V = Elem<T>::V;
  // FP16 is stored scaled and collided in the scaled units; FP32 carries
  // hi + lo constants (see collide_dev)
  constexpr bool SCALED = std::is_same<T, __half>::value;
  constexpr bool PRECISE = std::is_same<T, float>::value;
  LanePos p = lane_pos<V>(g, task, lane);
  if (!bounds::ok(!p.active || (p.y >= 0 && p.y < g.ny && p.x0 >= 0 && p.x0 + V <= g.pitch),
                  bounds::BATCH_LANE))
    p.active = false;
  if constexpr (sizeof(T) == 2) {
    uint32_t w[9][V / 2];
    pull9_packed<T>(src, g, p, w);
    collide_packed<T>(w, pairs_of(P));
    store9_packed<T>(dst, g, p, w);
  } else if constexpr (std::is_same<T, double>::value) {
    double f[9][V];
    pull9<T, false>(src, g, p, 1.0, f);
#pragma unroll
    for (int e = 0; e < V; ++e)
      collide_dev64(f[0][e], f[1][e], f[2][e], f[3][e], f[4][e], f[5][e], f[6][e], f[7][e],
                    f[8][e], P);
    store9<T, false>(dst, g, p, 1.0, f);
  } else {
    float f[9][V];
    pull9<T, false>(src, g, p, 1.0f, f);
#pragma unroll
    for (int e = 0; e < V; ++e)
      collide_dev<PRECISE, SCALED>(f[0][e], f[1][e], f[2][e], f[3][e], f[4][e], f[5][e], f[6][e],
                                   f[7][e], f[8][e], P);
    store9<T, false>(dst, g, p, 1.0f, f);
  }
}

// MINB: minimum resident 256-thread blocks per SM asked of the compiler,
// i.e. a register cap (1: none, 2: 128, 3: 80 registers) and so the warps
// an SM holds (8, 16, 24); the kernels are launched with smaller blocks
// (64 threads) that fill the same warp slots.  The launch variants of the
// tuner are MINB = 1, 2, 3.
template <typename T, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_step_dev(const T *__restrict__ src, T *__restrict__ dst, Geom g,
           typename ParamsOf<T>::type P, long long ntasks) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long task = warp0; task < ntasks; task += nwarps)
    step_task<T>(src, dst, g, P, task, lane);
}

// Batched, plain grid: every lattice starts on a block boundary and block b
// reads its lattice's geometry and buffers from blocks[b] (one load before
// the pull can start; a search over the lattices' task offsets, or a
// lattice index followed by the lattice's entry, cost 10-15% of the
// bandwidth on batches of small lattices).  Warps past the lattice's last
// task return.  limits (may be null): lattice l takes part only while
// k < limits[l], so members of one launch sequence can stop after different
// step counts.  CP (16-bit types): lattice l's collision constants are slot
// pbase + l of the constant table, else its entry's DevParams.
template <typename T, bool CP>
__device__ __forceinline__ void batch_block(const BatchEntry *__restrict__ ents,
                                            const BlockRec *__restrict__ blocks, int nents,
                                            int parity, const int *__restrict__ limits, int k,
                                            int pbase) {
  const int lane = threadIdx.x & 31;
  const BlockRec &B = blocks[blockIdx.x];
  // The records are read once per launch, so a step's 4.9 GB of streaming
  // has evicted them from L2 by the next launch, and a warp's record miss
  // to DRAM precedes its pull: each block prefetches into L2 the record of
  // the block about one wave of resident blocks later (measured +1.7%
  // FP32, +2.9% FP16, +1.8% BF16 on the 512-lattice batch; any distance
  // from 1024 to 2048 blocks alike; 152 SMs hold 1824 of the 64-thread
  // blocks at the 80-register cap, 2128 at 72; a compile-time distance
  // keeps the register budget, a launch parameter cost 20 bytes more of
  // spills)
  constexpr unsigned kPrefetch = 1536;
  if (threadIdx.x == 0 && blockIdx.x + kPrefetch < gridDim.x) {
    const char *q = reinterpret_cast<const char *>(blocks + blockIdx.x + kPrefetch);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(q));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(q + sizeof(BlockRec) - 1));
  }
  const long long task = B.task_base + (threadIdx.x >> 5);
  if (task >= B.g.tasks) return;                         // warp-uniform
  if (!bounds::ok(B.lat >= 0 && B.lat < nents, bounds::BATCH_REC)) return;
  if (limits != nullptr && k >= limits[B.lat]) return;   // block-uniform
  const int from = parity ^ B.off;
  const T *src = static_cast<const T *>(B.buf[from]);
  T *dst = static_cast<T *>(B.buf[from ^ 1]);
  if constexpr (CP && sizeof(T) == 2) {
    step_task<T>(src, dst, B.g, ConstPairs{(pbase + B.lat) * PC_COUNT}, task, lane);
  } else if constexpr (CP) {
    static_assert(sizeof(T) == 4, "constant tables: FP32 and the 16-bit types");
    step_task<T>(src, dst, B.g, c_dev[pbase + B.lat], task, lane);
  } else {
    step_task<T>(src, dst, B.g, ents[B.lat].dp, task, lane);
  }
}

template <typename T, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_step_batch(const BatchEntry *__restrict__ ents, const BlockRec *__restrict__ blocks,
             int nents, int parity, const int *__restrict__ limits, int k) {
  batch_block<T, false>(ents, blocks, nents, parity, limits, k, -1);
}

// The batched step with the constant table.  Register caps by variant: no
// cap, 128, and for variant 2 80 (FP32) or 72 (16-bit types; 28 warps per
// SM instead of 24).  Without the constants held in registers the 16-bit
// task spills less at 72 than at 80 (ptxas: FP16 64 / 56 bytes stored /
// loaded against 84 / 80, BF16 100 / 88 against 104 / 104), and the
// 512-lattice batch streams at 0.962 / 0.920 of the measured copy rate
// against 0.925 / 0.894 (FP16 / BF16; 64 registers, 32 warps: 0.882 /
// 0.747).  FP32 spills nothing at 80 (8 bytes with the constants from the
// entries) and streams at 1.033 against 1.026 (72 registers: 1.030).  The
// cap is written out in the attribute: nvcc takes a plain expression of
// MINB and T there.
template <typename T, int MINB>
__global__ void __maxnreg__(MINB >= 3 ? (sizeof(T) == 4 ? 80 : 72) : (MINB == 2 ? 128 : 255))
k_step_batch_table(const BatchEntry *__restrict__ ents, const BlockRec *__restrict__ blocks,
                   int nents, int parity, const int *__restrict__ limits, int k, int pbase) {
  batch_block<T, true>(ents, blocks, nents, parity, limits, k, pbase);
}

static inline long long n_tasks(const Geom &g) { return g.tasks; }

// Persistent batched variant: a grid of MINB blocks per SM strides over the
// plain grid's block records (block b takes records b, b + grid, ...), so
// at any time the grid works on a window of consecutive records, as the
// plain grid does.  Each warp keeps its current record in shared memory and
// fetches the next one (one word per lane, a single register) while it
// steps the current task, so the record's latency is hidden behind the
// step instead of opening every block.
template <typename T, int MINB>
__global__ void __launch_bounds__(256, MINB)
k_step_batch_stride(const BatchEntry *__restrict__ ents, const BlockRec *__restrict__ blocks,
                    long long nblocks, int nents, int parity, const int *__restrict__ limits,
                    int k) {
  constexpr int NW = sizeof(BlockRec) / 4;
  static_assert(sizeof(BlockRec) % 4 == 0 && NW <= 32, "a record must fit one word per lane");
  __shared__ BlockRec rec[2][8];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  long long b = blockIdx.x;
  if (b >= nblocks) return;  // block-uniform
  if (lane < NW)
    reinterpret_cast<uint32_t *>(&rec[0][w])[lane] =
        __ldg(reinterpret_cast<const uint32_t *>(blocks + b) + lane);
  __syncwarp();
  int s = 0;
  for (;;) {
    const long long nb = b + gridDim.x;
    uint32_t next = 0;
    if (nb < nblocks && lane < NW) next = __ldg(reinterpret_cast<const uint32_t *>(blocks + nb) + lane);
    const BlockRec &B = rec[s][w];
    const long long task = B.task_base + w;
    if (task < B.g.tasks && bounds::ok(B.lat >= 0 && B.lat < nents, bounds::BATCH_REC) &&
        !(limits != nullptr && k >= limits[B.lat])) {  // warp-uniform
      const int from = parity ^ B.off;
      step_task<T>(static_cast<const T *>(B.buf[from]), static_cast<T *>(B.buf[from ^ 1]), B.g,
                   ents[B.lat].dp, task, lane);
    }
    if (nb >= nblocks) break;
    __syncwarp();
    if (lane < NW) reinterpret_cast<uint32_t *>(&rec[s ^ 1][w])[lane] = next;
    __syncwarp();
    s ^= 1;
    b = nb;
  }
}

template <typename T>
cudaError_t launch_step_dev_t(const Lattice &L, const void *src, void *dst, cudaStream_t st,
                              int block, int variant) {
  const long long nt = n_tasks(L.g);
  const int wpb = block / 32;
  long long grid = (nt + wpb - 1) / wpb;
  if (grid < 1) grid = 1;
  const T *s = static_cast<const T *>(src);
  T *d = static_cast<T *>(dst);
  const typename ParamsOf<T>::type *P;
  if constexpr (std::is_same<T, double>::value) P = &L.dp64;
  else P = &L.dp;
  switch (variant) {
    case 0: k_step_dev<T, 1><<<(unsigned)grid, block, 0, st>>>(s, d, L.g, *P, nt); break;
    case 1: k_step_dev<T, 2><<<(unsigned)grid, block, 0, st>>>(s, d, L.g, *P, nt); break;
    default: k_step_dev<T, 3><<<(unsigned)grid, block, 0, st>>>(s, d, L.g, *P, nt); break;
  }
  return cudaGetLastError();
}

}  // namespace lbm

// small batch members held in shared memory (uses the collisions above)
#include "resident.cuh"

namespace lbm {

// Slots pbase .. pbase + n - 1 of the constant table from the entries'
// parameters, through stage (n * PC_COUNT floats of device memory), in the
// order of stream st.
static __global__ void k_fill_pairs(const BatchEntry *__restrict__ ents, int n,
                                    float *__restrict__ stage) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n * PC_COUNT) stage[i] = pair_const(ents[i / PC_COUNT].dp, i % PC_COUNT);
}

static __global__ void k_fill_dev(const BatchEntry *__restrict__ ents, int n,
                                  DevParams *__restrict__ stage) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) stage[i] = ents[i].dp;
}

template <typename T>
cudaError_t upload_consts_t(const BatchEntry *ents, int n, int pbase, void *stage,
                            cudaStream_t st) {
  constexpr bool PAIRS = sizeof(T) == 2;
  static_assert(PAIRS || sizeof(T) == 4, "constant tables: FP32 and the 16-bit types");
  constexpr int slots = PAIRS ? kPairTable : kDevTable;
  static_assert(slots == (PAIRS ? kPairSlots : kDevSlots),
                "this translation unit does not hold the type's constant table");
  if (n < 1) return cudaSuccess;
  if (pbase < 0 || n > slots - pbase || stage == nullptr) return cudaErrorInvalidValue;
  cudaError_t e;
  if constexpr (PAIRS) {
    const int nv = n * PC_COUNT;
    k_fill_pairs<<<(nv + 255) / 256, 256, 0, st>>>(ents, n, static_cast<float *>(stage));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbolAsync(c_pairs, stage, (size_t)nv * sizeof(float),
                                   (size_t)pbase * PC_COUNT * sizeof(float),
                                   cudaMemcpyDeviceToDevice, st);
  } else {
    k_fill_dev<<<(n + 255) / 256, 256, 0, st>>>(ents, n, static_cast<DevParams *>(stage));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbolAsync(c_dev, stage, (size_t)n * sizeof(DevParams),
                                   (size_t)pbase * sizeof(DevParams), cudaMemcpyDeviceToDevice,
                                   st);
  }
}

template <typename T>
cudaError_t launch_step_batch_t(const BatchList &bl, int parity, cudaStream_t st, int block,
                                int variant, const int *limits, int k) {
  if (bl.nblocks < 1 || bl.ntasks < 1) return cudaSuccess;
  if (variant >= kStepVariants) {
    // persistent: the resident blocks (MINB x 256 threads per SM) striding
    // over the records
    const int minb = variant - kStepVariants + 1;
    long long pgrid = (long long)sm_count() * minb * (256 / block);
    if (pgrid > bl.nblocks) pgrid = bl.nblocks;
    switch (minb) {
      case 1:
        k_step_batch_stride<T, 1><<<(unsigned)pgrid, block, 0, st>>>(
            bl.ents, bl.blocks, bl.nblocks, bl.n, parity, limits, k);
        break;
      case 2:
        k_step_batch_stride<T, 2><<<(unsigned)pgrid, block, 0, st>>>(
            bl.ents, bl.blocks, bl.nblocks, bl.n, parity, limits, k);
        break;
      default:
        k_step_batch_stride<T, 3><<<(unsigned)pgrid, block, 0, st>>>(
            bl.ents, bl.blocks, bl.nblocks, bl.n, parity, limits, k);
        break;
    }
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)bl.nblocks;
  if constexpr (sizeof(T) <= 4) {
    if (bl.pbase >= 0) {
      switch (variant) {
        case 0:
          k_step_batch_table<T, 1><<<grid, block, 0, st>>>(bl.ents, bl.blocks, bl.n, parity,
                                                           limits, k, bl.pbase);
          break;
        case 1:
          k_step_batch_table<T, 2><<<grid, block, 0, st>>>(bl.ents, bl.blocks, bl.n, parity,
                                                           limits, k, bl.pbase);
          break;
        default:
          k_step_batch_table<T, 3><<<grid, block, 0, st>>>(bl.ents, bl.blocks, bl.n, parity,
                                                           limits, k, bl.pbase);
          break;
      }
      return cudaGetLastError();
    }
  }
  switch (variant) {
    case 0:
      k_step_batch<T, 1><<<grid, block, 0, st>>>(bl.ents, bl.blocks, bl.n, parity, limits, k);
      break;
    case 1:
      k_step_batch<T, 2><<<grid, block, 0, st>>>(bl.ents, bl.blocks, bl.n, parity, limits, k);
      break;
    default:
      k_step_batch<T, 3><<<grid, block, 0, st>>>(bl.ents, bl.blocks, bl.n, parity, limits, k);
      break;
  }
  return cudaGetLastError();
}

}  // namespace lbm

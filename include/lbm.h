/*
 * lbm.h -- C ABI of the GB300 (sm_103a) D2Q9 multi-relaxation-time lattice
 * Boltzmann library (liblbm.so).
 *
 * The scheme is the one of Xu & Sagaut, "Optimal low-dispersion
 * low-dissipation LBM schemes for computational aeroacoustics"
 * (arXiv 1107.4543):
 *   - evolution f_i(x + c_i, t + 1) = f_i + Lambda_ij (f_j^eq - f_j)
 *     (section 2.1, Eq. blbs) on a periodic nx x ny lattice, dt = dx = 1;
 *   - Lambda = M^-1 S M, conserved moments rho, jx, jy kept, the others
 *     relaxed m_i <- m_i - s_i (m_i - m_i^eq) (section 2.1,
 *     Eqs. eq_conservative, eq_noconservative, q-macro);
 *   - D2Q9 equilibrium moments {rho, jx, jy, -2rho + 3|j|^2/rho,
 *     rho - 3|j|^2/rho, -jx, -jy, (jx^2 - jy^2)/rho, jx jy/rho} and
 *     S = diag(0,0,0,s_e,s_eps,s_q,s_q,s_nu,s_nu) (section 2.3).
 * The paper prints neither the velocity order nor M; this library uses
 * c_0..c_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1)
 * and the Lallemand-Luo D2Q9 moment matrix.
 *
 * Conventions (all entry points):
 *   - return LBM_OK (0) on success, LBM_PENDING (> 0) for an unfinished
 *     request, or a negative LBM_E* code; lbm_strerror() names a code and
 *     lbm_last_error() gives the calling thread's last detailed message;
 *   - host arrays are owned by the caller and are row-major ny x nx
 *     (index y * nx + x) float64, populations 9 x ny x nx (index
 *     (i * ny + y) * nx + x);
 *   - device memory of a lattice is owned by its handle; arguments named
 *     *_dev are device pointers owned by the caller;
 *   - a handle is not thread-safe; the server (lbm_server_*) is;
 *   - every call runs on the GPU that was current at lbm_create; work is
 *     enqueued on the handle's stream (lbm_set_stream), and the calls that
 *     return host data synchronize that stream.
 * No entry point falls back to the CPU: without a usable GPU they fail
 * with LBM_ECUDA.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ codes */
#define LBM_OK 0
#define LBM_PENDING 1
#define LBM_EINVAL (-1)    /* bad argument (sizes, rates, null pointer)    */
#define LBM_ENOMEM (-2)    /* device or host allocation failed / budget    */
#define LBM_ECUDA (-3)     /* a CUDA call failed                           */
#define LBM_EUNSTABLE (-4) /* non-finite populations detected              */
#define LBM_ETIMEOUT (-5)  /* a bounded wait ran out                       */
#define LBM_ENOTFOUND (-6) /* unknown request id                           */
#define LBM_ECLOSED (-7)   /* server shutting down                         */

/* storage types of the populations.  The *DEV types store the deviation
 * f' = f - f^eq(rho0, u0); the 32- and 16-bit ones collide in FP32,
 * LBM_F64DEV in FP64 with fused multiply-adds.  LBM_F64 stores the full
 * populations and computes in FP64 with the operation order of a plain
 * matrix-vector implementation of section 2.1 (bit-identical to a plain
 * FP64 implementation); LBM_F64DEV is the faster FP64 path, within 1e-12
 * relative of an extended-precision implementation of the same scheme.
 * Batches and the server take the 32- and 16-bit types. */
#define LBM_F64 0
#define LBM_F32DEV 1
#define LBM_F16DEV 2  /* FP16, scaled by a power of two fixed at init */
#define LBM_BF16DEV 3
#define LBM_F64DEV 4

typedef struct lbm_ctx *lbm_handle;

/* lbm_create -- allocate a periodic nx x ny lattice (section 2.1).
 *   S[9]   relaxation rates in Lallemand-Luo order
 *          (rho, e, eps, jx, qx, jy, qy, pxx, pxy), e.g. the original
 *          scheme's (0, 1.64, 1.54, 0, 1.9, 0, 1.9, 1/tau, 1/tau) of
 *          section 2.3; the library maps them to the paper's order
 *          (rho, jx, jy, e, eps, qx, qy, pxx, pxy).  Entries of the conserved
 *          slots (rho, jx, jy) are ignored but must be finite; the others
 *          must lie in (0, 2].  The two q entries may differ, as may the two
 *          p entries.
 *   rho0, u0[2]  reference state: the base f^eq(rho0, u0) of the
 *          deviation storage types and the initial uniform state.
 *   storage_dtype  LBM_F64 / LBM_F32DEV / LBM_F16DEV / LBM_BF16DEV /
 *                  LBM_F64DEV.
 * The lattice starts as the uniform equilibrium f^eq(rho0, u0).
 * Errors: LBM_EINVAL (nx or ny < 2, rates out of range, rho0 <= 0, null
 * out), LBM_ENOMEM, LBM_ECUDA (no GPU).  *out is set only on success. */
int lbm_create(int nx, int ny, const double S[9], double rho0,
               const double u0[2], int storage_dtype, lbm_handle *out);

/* lbm_init_field -- set f = f^eq(rho, u) at every node from host fields
 * rho, ux, uy (ny x nx each); t is reset to 0.  Initialisation by the
 * equilibrium of the prescribed macroscopic fields (section 5.2 gives only
 * rho and u).  For LBM_F16DEV the power-of-two storage scale is chosen here
 * from the largest |f'|.  Copies host->device and synchronizes.
 * Errors: LBM_EINVAL (null pointer, rho <= 0 somewhere), LBM_ECUDA. */
int lbm_init_field(lbm_handle h, const double *rho, const double *ux,
                   const double *uy);

/* lbm_init_field_dev -- as lbm_init_field with device fields (float64,
 * ny x nx, row-major, caller-owned); enqueued, no host copy.  For
 * LBM_F16DEV it synchronizes once to read the largest |f'|. */
int lbm_init_field_dev(lbm_handle h, const double *rho_dev,
                       const double *ux_dev, const double *uy_dev);

/* lbm_init_analytic -- f = f^eq(rho, u) of an analytic field computed on
 * the device (no host arrays):
 *   kind LBM_INIT_GAUSSIAN: rho = rho0 + p[0] exp(-ln2 |x - (p[2],p[3])|^2
 *        / p[1]^2) with the minimum-image distance, u = u0 (section 5.2);
 *   kind LBM_INIT_PLANE: rho = rho0 + p[0] cos(2 pi p[1] x / nx),
 *        ux = u0x + p[0] cos(...) / (sqrt(3) rho0), uy = u0y (a right-running
 *        acoustic wave with p[1] wavelengths in the period). */
#define LBM_INIT_GAUSSIAN 1
#define LBM_INIT_PLANE 2
int lbm_init_analytic(lbm_handle h, int kind, const double params[8]);

/* lbm_step -- enqueue n >= 0 time steps (one fused pull-stream + collide
 * kernel per step, replayed from a captured CUDA graph in chunks) on the
 * handle's stream and return without waiting.  Errors: LBM_EINVAL (n < 0),
 * LBM_ECUDA (launch failure). */
int lbm_step(lbm_handle h, long n);

/* lbm_set_source -- the acoustic point source of section 5.1: before the
 * collision of every later lbm_step, node (x, y) is set to the equilibrium
 * at rest with density rho0 + amplitude * sin(2 pi t / period), t the
 * lattice time at the start of that step (0 after init).  amplitude = 0
 * removes the source.  Runs of 64 steps from an even step replay a captured
 * graph of (forced node, step) pairs after the host uploads that run's 64
 * forcing values; other steps are launched one by one (same results).  FP16
 * storage: a source set before lbm_init_field / lbm_set_populations enters
 * the choice of the storage scale (its node deviates by up to 4/9 of the
 * amplitude).  Errors: LBM_EINVAL (node outside the lattice, period <= 0,
 * batch member, or an FP16 state whose scale leaves no room for the
 * amplitude). */
int lbm_set_source(lbm_handle h, int x, int y, double amplitude, double period);

/* lbm_tune -- (runtime; no counterpart in the paper) time the launch
 * variants of the step kernel on this lattice
 * (LBM_TUNE_VARIANTS register caps of the deviation-storage kernel) and keep
 * the fastest for later steps.  Trial launches read the current state and
 * write only the idle buffer, so the lattice's state does not change.
 * times_ms (may be NULL) receives each variant's average launch time,
 * chosen (may be NULL) the variant kept.  lbm_step tunes lattices of at
 * least 2^20 nodes on their first step unless the environment sets
 * LBM_AUTOTUNE=0; choices are shared by lattices of the same type and size
 * within the process.  LBM_F64 has one variant (times -1).  Synchronizes. */
#define LBM_TUNE_VARIANTS 3
int lbm_tune(lbm_handle h, double *times_ms, int *chosen);
/* Use launch variant `variant` (0 .. LBM_TUNE_VARIANTS-1) for later steps,
 * without timing (no automatic tuning afterwards).  Every variant computes
 * the same result; they differ only in speed.  lbm_get_variant reports the
 * variant in use once chosen (by tuning, the tuning file, lbm_set_variant or
 * a small lattice's first step), -1 before; LBM_F64 reports 0.
 * With LBM_TUNE_CACHE=<path> in the environment the choices of lbm_step's
 * automatic tuning and of the batches' are also read from and appended to
 * that file (one line per choice, keyed by GPU model, storage type and
 * size), so later processes skip the timing runs. */
int lbm_set_variant(lbm_handle h, int variant);
int lbm_get_variant(lbm_handle h, int *variant);

/* lbm_moments -- rho, ux, uy (host, ny x nx) at the current time: the
 * moments of the pre-collision populations, u = j / rho.  Synchronizes. */
int lbm_moments(lbm_handle h, double *rho, double *ux, double *uy);

/* lbm_moments_dev -- as lbm_moments into caller-owned device arrays;
 * enqueued, does not synchronize. */
int lbm_moments_dev(lbm_handle h, double *rho_dev, double *ux_dev,
                    double *uy_dev);

/* lbm_destroy -- synchronize the handle's stream and free its memory. */
int lbm_destroy(lbm_handle h);

/* ---------------------------------------------------------- extensions */
/* Full populations f (host, 9 x ny x nx, float64) at the current time:
 * checkpoint (get) and restore / arbitrary initial state (set).  For the
 * deviation types the base f^eq(rho0, u0) is added / subtracted in FP64;
 * set() on LBM_F16DEV re-chooses the storage scale.  Both synchronize. */
int lbm_get_populations(lbm_handle h, double *f);
int lbm_set_populations(lbm_handle h, const double *f);

/* Use `stream` (a cudaStream_t, e.g. torch.cuda.current_stream()) for all
 * further work of the handle; NULL restores the handle's own stream (so the
 * legacy default stream cannot be selected: pass a created stream).
 * Synchronizes the previous stream first. */
int lbm_set_stream(lbm_handle h, void *stream);

/* Wait for the handle's stream. */
int lbm_sync(lbm_handle h);

/* Global sums over the lattice in FP64, by a deterministic two-stage
 * reduction on the device: out[0] = sum rho', out[1] = sum jx',
 * out[2] = sum jy' (deviations from rho0, rho0 u0), out[3] = number of
 * non-finite stored populations.  Each node's sums are taken over the
 * populations' deviations from the base f^eq(rho0, j0) (stored as such by
 * the deviation types; formed exactly from FP64 populations near the base),
 * so they round at the size of the perturbation.  The collision conserves mass and
 * momentum exactly in exact arithmetic (section 2.1,
 * Eq. eq_conservative), so out[0..2] measure rounding drift.
 * Synchronizes; returns LBM_EUNSTABLE when out[3] > 0. */
int lbm_drift(lbm_handle h, double out[4]);

/* lbm_drift_pop_noalloc -- the sums of lbm_drift over a caller-owned array
 * of full FP64 populations, without allocating any device memory.  The
 * paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory -- e.g. a host application whose own allocator
 * already owns the GPU's memory, or a loop under a fixed memory budget where
 * a cudaMalloc (with its implicit synchronisation and failure modes) is not
 * acceptable.
 *   f_dev   device array of 9 x ny x nx doubles (index (i*ny + y)*nx + x),
 *           owned by the caller, unchanged
 *   rho0, jx0, jy0  reference state: its equilibrium populations
 *           f^eq(rho0, j0) are subtracted from every node's populations
 *           before the sums, as lbm_drift does
 *   out     host array of 4 doubles, owned by the caller: sum rho',
 *           sum jx', sum jy', number of non-finite populations
 *   stream  cudaStream_t to run on (NULL: the legacy default stream);
 *           the call synchronizes it before returning.
 * Its scratch is a fixed device array inside the library of
 * (8192 + 1) x 4 doubles (256 KiB + 32 B), held by every GPU that loads the
 * library until the process exits; hence ny <= 8192 (LBM_EINVAL with a
 * message otherwise).  The first call on a device looks up that array's
 * device address (once per device); make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's
 * contents (each call writes every slot it reads): calls that overlap on
 * the GPU race, so serialize them.  Returns LBM_EUNSTABLE when out[3] > 0. */
int lbm_drift_pop_noalloc(const double *f_dev, int nx, int ny, double rho0,
                          double jx0, double jy0, double out[4], void *stream);

/* Static description of a lattice. */
typedef struct {
  int nx, ny;
  int pitch;          /* elements per stored row (>= nx)                */
  int dtype;          /* LBM_F64 ... LBM_F64DEV                          */
  int elem_bytes;     /* bytes per stored population                     */
  long t;             /* time steps taken since the last init/set        */
  double qscale;      /* LBM_F16DEV: stored value = f' * qscale          */
  double S_paper[9];  /* rates in the paper's moment order               */
  size_t device_bytes;/* device memory held by the handle                */
} lbm_info_t;
int lbm_info(lbm_handle h, lbm_info_t *out);

/* (runtime; no counterpart in the paper) Device allocator used for all
 * later allocations of lattices, batches,
 * servers and cost evaluations (e.g. a caching allocator).  alloc returns
 * NULL on failure, else memory aligned to 256 bytes (as cudaMalloc's;
 * lbm_create refuses lattice buffers that are not, LBM_EINVAL).  Passing NULL functions restores cudaMalloc / cudaFree.
 * Not thread-safe with respect to concurrent lbm_create calls.  The
 * staging that lbm_vn_eigs keeps for the life of the process uses
 * cudaMalloc / cudaHostAlloc directly, so that it never outlives the
 * allocator that made it. */
/* (runtime; no counterpart in the paper) Page-locked host memory for the
 * host arrays of the I/O calls (lbm_batch_solve_packed's fields and
 * moments above all): an anonymous mapping advised for transparent huge
 * pages -- arrays of at least a quarter huge page start on a huge-page
 * boundary and fill whole huge pages -- touched, then registered with the
 * CUDA driver, so that a copy walks few page translations.  Returns NULL
 * (message in lbm_last_error) when the mapping or the registration fails.
 * lbm_host_free releases one such array (LBM_EINVAL for any other
 * pointer; NULL is a no-op). */
void *lbm_host_alloc(size_t bytes);
int lbm_host_free(void *p);

typedef void *(*lbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbm_free_fn)(void *ptr, void *ctx);
int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void *ctx);

const char *lbm_strerror(int code);
const char *lbm_last_error(void);

/* (runtime; no counterpart in the paper) Index checks of the debug build
 * (compiled with -DLBM_DEBUG_BOUNDS: paper_1107_4543_gb300/build.py
 * build(debug=True) makes _build_debug/liblbm.so).  The von Neumann QR, the
 * optimizer's polynomial-matrix slots and tables, the batched step's block
 * records and lane positions and the batched init / moments blocks check
 * their indices; a failed check sets a bit of a device word and the access
 * goes to the array's first element instead (no trap, the context stays
 * usable).  lbm_debug_bounds ORs the words of every translation unit of the
 * current device into *word (bits: see csrc/bounds.cuh) and, if reset,
 * clears them; lbm_debug_bounds_selftest runs one checked access past its
 * bound (bit 31).  Without the flag both return LBM_EINVAL (*word = 0). */
int lbm_debug_bounds(unsigned int *word, int reset);
int lbm_debug_bounds_selftest(void);

/* ------------------------------------------------- von Neumann analysis */
/* lbm_vn_eigs -- eigenvalues of the von Neumann amplification matrix of
 * section 4.1, G(k) = diag(exp(-i k.c_j)) M^-1 Psi M, with Psi the
 * linearized relaxation of section 2.3 about rho = 1 and the mean flow
 * (U, V), for n cases on the GPU (one thread per case, FP64: Householder
 * Hessenberg reduction and shifted QR).  Host arrays, caller-owned:
 *   kx, ky, U, V  n each;  S  9 n, case c's rates in Lallemand-Luo order at
 *   S[9c .. 9c+8];  eig  18 n, the 9 eigenvalues of case c as (re, im)
 *   pairs at eig[18c ..], in no particular order.
 * lambda = exp(-i omega): damping per step -ln|lambda|, phase speed
 * -arg(lambda)/|k|.  *unconverged (may be NULL) counts eigenvalues whose QR
 * iteration reached its limit of 60 sweeps (returns LBM_ETIMEOUT then).
 * Synchronizes.  The cases go in up to 8 chunks on their own streams, so
 * the host's packing and unpacking overlap the copies and the kernels;
 * page-locked host and device staging sized for the largest call so far
 * is kept for the life of the process, and concurrent calls are
 * serialized. */
int lbm_vn_eigs(int n, const double *kx, const double *ky, const double *U,
                const double *V, const double *S, double *eig,
                int *unconverged);

/* -------------------------------------- free-parameter optimization */
/* The cost functions of section 3.2 and their minimization (section 4.2).
 * For a wave direction theta and mean flow (U, V) the recursive algorithm
 * of section 2.2 (Eqs. R-A, R-B, R-D, R-E) gives dW/dt = B_n W for the
 * conserved W = (rho, jx, jy), B_n = sum_{l<n} dt^l k^(l+1) b^l(theta).
 * The costs integrate ||M_eps||_F^2, M_eps = B_n - B (the exact linearized
 * matrix B as selected by `reference`), over dt k in [0, pi] and theta in
 * [0, 2 pi): F^o, F^e, calligraphic F (Eqs. Minimization-A/B/C) for zero
 * mean flow; for mean flows G^o, G^e, calligraphic G (Eqs. approximation-D/E,
 * Minimization-F) also over the flow direction in [0, 2 pi) and the speed
 * in [0, u0].  The odd / even parts keep the odd / even powers of dt k.
 * Readings (each reproduces the cost values printed in Tables 1-3 to 1e-9):
 * the speed integral runs over [0, 0.2] (the paper's stated u0); Table 2
 * measures B_n against the inviscid (Euler) matrix, Table 3 against
 * convection plus shear dissipation (B - Bbulk of section 3.2.3), zero-flow
 * costs against convection plus the exact dissipation. */
#define LBM_COST_F 0       /* zero mean flow */
#define LBM_COST_G 1       /* mean flows, integrated over direction and speed */
#define LBM_PART_ALL 0
#define LBM_PART_ODD 1     /* dispersion: odd powers of dt k */
#define LBM_PART_EVEN 2    /* dissipation: even powers of dt k */
#define LBM_REF_NS 0       /* convection + exact dissipation */
#define LBM_REF_EULER 1    /* convection only */
#define LBM_REF_NS_BULK 2  /* convection + shear dissipation (B - Bbulk) */
typedef struct {
  int kind;         /* LBM_COST_F or LBM_COST_G */
  int order;        /* truncation order n of B_n, 1..6 */
  int part;         /* LBM_PART_* */
  int reference;    /* LBM_REF_* */
  double u0;        /* LBM_COST_G: speeds in [0, u0] */
  int fixed_speed;  /* LBM_COST_G: nonzero = the single speed u0 */
} lbm_cost_spec;
/* lbm_opt_cost -- the cost of n candidates.  sigmas: 4 n host doubles,
 * candidate c's (sigma_e, sigma_eps, sigma_q, sigma_nu) at sigmas[4c],
 * sigma = 1/s - 1/2 >= 0 (s in (0, 2]); out: n host doubles.  One warp per
 * quadrature point on the GPU, FP64, quadratures exact for the integrands;
 * results reproducible bit for bit.  Synchronizes; allocates device memory
 * for the call.  LBM_EINVAL on a bad spec or a negative / non-finite sigma. */
int lbm_opt_cost(const lbm_cost_spec *spec, int n, const double *sigmas, double *out);
/* lbm_opt_minimize -- minimize the cost over the sigmas selected by
 * free_mask (bit i = sigma i of the order above) within [lo[i], hi[i]]
 * (0 <= lo < hi), the others held at sigmas_in: a grid scan (0 and a
 * log-spaced grid per free sigma, evaluated as one batch), then Nelder-Mead
 * in the scaled free sigmas, restarted until the cost stops improving.
 * Writes the minimizer to sigmas_out, its cost to *cost_out and the number
 * of cost evaluations to *evals (both may be NULL). */
int lbm_opt_minimize(const lbm_cost_spec *spec, const double sigmas_in[4],
                     unsigned free_mask, const double lo[4], const double hi[4],
                     double sigmas_out[4], double *cost_out, int *evals);

/* ------------------------------------------------------------- batches */
/* Many independent lattices advanced together (runtime around the step of
 * section 2.1, which the paper states for one lattice): every time step is ONE
 * kernel launch per storage type over a work list of all members (each
 * lattice starts on a block boundary; one record per block gives its
 * lattice, geometry and buffers), and chunks of 64 steps are replayed from a
 * captured CUDA graph; members small enough for one block's shared memory
 * are instead held there for all the steps of a call (lbm_batch_resident),
 * with the same arithmetic.  Members must be deviation-storage lattices
 * (LBM_F32DEV, LBM_F16DEV or LBM_BF16DEV) created on the current device,
 * none of them in another batch; they keep their own memory, rates and
 * reference state, and each advances with exactly the arithmetic of
 * lbm_step.  While in the batch a member's work runs on the batch stream
 * (its first member's); lbm_moments, lbm_get_populations and lbm_drift on a
 * member work as usual between batch steps, while lbm_step, init and
 * set_populations on a member are rejected (LBM_EINVAL).  lbm_batch_destroy
 * releases the members, which stay valid. */
typedef struct lbm_batch_ctx *lbm_batch;
int lbm_batch_create(int n, const lbm_handle *members, lbm_batch *out);
int lbm_batch_step(lbm_batch b, long n);
/* Host I/O for the whole batch with one synchronization: the arrays hold
 * one pointer per member (member order), each to a host ny x nx float64
 * array as for lbm_init_field / lbm_moments.  The copies run on a copy
 * stream of the batch, overlapped with the batch stream's kernels of the
 * neighbouring members; the call returns when all of them are done and the
 * host arrays may be reused.  lbm_batch_init_fields sets f = f^eq(rho, u)
 * for every member (t reset to 0; FP16 members re-choose their storage
 * scale) and keeps the batch usable; LBM_EINVAL if any member's field has
 * non-finite values or rho <= 0.  lbm_batch_moments returns every member's
 * rho, ux, uy.  Page-locked host memory gives the full link rate. */
int lbm_batch_init_fields(lbm_batch b, const double *const *rho,
                          const double *const *ux, const double *const *uy);
int lbm_batch_moments(lbm_batch b, double *const *rho, double *const *ux,
                      double *const *uy);
/* members: number of members; nodes: their total node count, sum of nx*ny
 * (either pointer may be NULL). */
int lbm_batch_size(lbm_batch b, int *members, long long *nodes);
/* The same host I/O with packed arrays: rho, ux, uy each hold `nodes`
 * float64 values (lbm_batch_size), member k's ny x nx row-major field
 * starting at the sum of nx*ny of members 0..k-1.  The copies go in groups
 * of consecutive members of about 2^23 nodes, so a batch of many small
 * lattices still moves its fields in few large copies (many small host
 * copies run well below the link rate on some hosts).  The first call
 * allocates a device staging buffer of 3 x nodes doubles, kept until
 * lbm_batch_destroy.  Results equal those of the per-member calls bit for
 * bit. */
int lbm_batch_init_packed(lbm_batch b, const double *rho, const double *ux,
                          const double *uy);
int lbm_batch_moments_packed(lbm_batch b, double *rho, double *ux, double *uy);

/* (runtime; no counterpart in the paper) One whole solve of every member,
 * queued without waiting: upload the packed fields (layout of
 * lbm_batch_init_packed), set every member to f^eq(rho, u) (section 2.3),
 * advance n time steps (section 2.1, Eq. blbs), take every member's drift
 * sums (as lbm_batch_drift) and download the packed moments (as
 * lbm_batch_moments_packed).  Returns once the work is queued.  Successive
 * solves of a batch overlap: solve k's upload and solve k-1's download run
 * on two copy streams of the batch while solve k-1 and solve k step, through
 * two device staging slots (4 x 3 x nodes doubles in all, allocated on the
 * first call and kept until lbm_batch_destroy).  Results equal those of
 * lbm_batch_init_packed + lbm_batch_step + lbm_batch_drift +
 * lbm_batch_moments_packed bit for bit.
 *   rho_in, ux_in, uy_in    host arrays of the batch's node count (packed
 *                           member after member, each ny x nx row-major),
 *                           read by the upload; page-locked for overlap
 *   rho_out, ux_out, uy_out host arrays of the same size, written by the
 *                           download; page-locked (a copy into pageable
 *                           memory blocks the call until it lands, which
 *                           leaves nothing to overlap)
 *   drift_out               host array of 4 doubles per member, or NULL
 *                           (any host memory: the sums pass through a
 *                           page-locked array of the batch)
 * The caller owns every host array and must neither free nor change the
 * inputs, nor read the outputs, before lbm_batch_wait returns.  Invalid
 * fields (non-finite, rho <= 0) and non-finite populations are reported by
 * lbm_batch_wait.  FP16 members choose their storage scale on the device
 * from the staged fields, by lbm_init_field's rule, before the init; the
 * host copy (lbm_info's qscale) follows the last solve's at lbm_batch_wait. */
int lbm_batch_solve_packed(lbm_batch b, long n, const double *rho_in, const double *ux_in,
                           const double *uy_in, double *rho_out, double *ux_out,
                           double *uy_out, double *drift_out);
/* Wait for every solve queued by lbm_batch_solve_packed.  phase_ms (may be
 * NULL) receives 6 device times per solve, in ms, measured by events on the
 * streams that ran them: upload, init, steps, drift, moments, download --
 * each the median over the solves queued since the previous wait (the last
 * 32 of them at most; the last solve alone when none was queued since).  Returns LBM_EINVAL if any solve since the last wait had invalid
 * fields (message names the member), LBM_EUNSTABLE if a drift array passed
 * since then reports non-finite populations, else 0. */
int lbm_batch_wait(lbm_batch b, double *phase_ms);

/* As lbm_tune for the batch's launches (one variant for all its storage
 * types; the first lbm_batch_step of a batch of >= 2^20 nodes tunes unless
 * LBM_AUTOTUNE=0).  Batches have LBM_BATCH_TUNE_VARIANTS variants: the
 * three register caps with one block per record, then the same caps with a
 * persistent grid of a few blocks per SM striding over the records.
 * times_ms receives LBM_BATCH_TUNE_VARIANTS entries.  Members' states do
 * not change. */
#define LBM_BATCH_TUNE_VARIANTS 6
int lbm_batch_tune(lbm_batch b, double *times_ms, int *chosen);
/* As lbm_set_variant for a batch (0 .. LBM_BATCH_TUNE_VARIANTS-1); get
 * reports the variant in use (-1 before the first step of an untuned
 * batch). */
int lbm_batch_set_variant(lbm_batch b, int variant);
int lbm_batch_get_variant(lbm_batch b, int *variant);
/* (runtime; no counterpart in the paper) Which members the batch keeps in
 * shared memory for all the steps of a launch (flags: one int per member, 1
 * for such a member): lattices whose two step buffers of 9 compact planes,
 * 2 x 9 x nx x ny x element bytes, fit one block's shared memory (227 KB on
 * GB300: up to 56 x 56 nodes in FP32, 80 x 80 in FP16 / BF16), unless the
 * environment variable LBM_RESIDENT_BYTES, read when the batch is made,
 * caps that size (0: none).  One thread block per such member runs all the
 * steps of an lbm_batch_step call (or of a server generation) in one launch
 * beside the per-step launches of the other members, reading and writing
 * the member's populations in HBM once; results are bit-identical either
 * way. */
int lbm_batch_resident(lbm_batch b, int *flags);
/* (runtime; no counterpart in the paper) Which members' collision constants
 * the per-step launches read from a constant-memory table (flags: one int
 * per member, 1 for such a member).  Each storage type of a batch reserves
 * one slot per member of that type when the batch is made, out of a table
 * per storage type and device shared by all live batches (960 slots for
 * LBM_F16DEV and LBM_BF16DEV, 640 for LBM_F32DEV), and releases them when
 * it is destroyed; a type that finds no room, or a batch made with the
 * environment variable LBM_CONST_TABLE=0, reads the constants from its
 * members' entries in global memory instead.  The slots are refreshed from
 * the members' parameters at the start of every stepping call.  Results
 * are bit-identical either way. */
int lbm_batch_const_table(lbm_batch b, int *flags);
/* The sums of lbm_drift for every member at once (out: 4 doubles per member,
 * in member order): one reduction launch pair for the whole batch,
 * reproducible per member.  Synchronizes the batch stream; returns
 * LBM_EUNSTABLE when any member holds non-finite populations. */
int lbm_batch_drift(lbm_batch b, double *out);
int lbm_batch_destroy(lbm_batch b);

/* ------------------------------------------------------------- serving */
/* A request: one lattice solve.  init_kind is LBM_INIT_GAUSSIAN or
 * LBM_INIT_PLANE (params as for lbm_init_analytic) or LBM_INIT_FIELDS (the
 * host fields rho/ux/uy, ny x nx, copied at submit time). */
#define LBM_INIT_FIELDS 0
typedef struct {
  int nx, ny;
  double S[9];            /* Lallemand-Luo order, as for lbm_create        */
  double rho0, u0[2];
  int dtype;              /* LBM_F32DEV, LBM_F16DEV or LBM_BF16DEV          */
  long steps;
  int init_kind;
  double init_params[8];
  const double *rho, *ux, *uy; /* LBM_INIT_FIELDS only                     */
} lbm_request;

typedef struct lbm_server_ctx *lbm_server;

/* A continuous-batching server on the current device (runtime around the
 * step of section 2.1; no counterpart in the paper): a host scheduler
 * thread admits queued requests while their device bytes fit in
 * hbm_budget_bytes (see lbm_server_set_policy for order and caps), steps
 * all admitted lattices together in generations of at most chunk_steps
 * steps (one batched launch per step and storage type; each lattice stops
 * at its own step count), retires finished lattices (moments copied to
 * host, memory freed) and admits newcomers between generations.  Every
 * result equals the same solve run alone.  Thread-safe. */
int lbm_server_create(size_t hbm_budget_bytes, long chunk_steps,
                      lbm_server *out);

/* Admission order and resident-work cap of a server:
 *   LBM_SERVE_FIFO      requests are admitted in arrival order (default);
 *   LBM_SERVE_SHORTEST  the queued request with the least work
 *                       (nx * ny * steps) is admitted first;
 *   max_resident_nodes  > 0: admit only while the resident lattices hold at
 *                       most this many nodes (one request is always
 *                       admitted when the device is empty); 0: the byte
 *                       budget alone limits admission.
 * A cap keeps generations short -- every resident lattice advances in each
 * generation -- while enough work stays resident to saturate the GPU. */
#define LBM_SERVE_FIFO 0
#define LBM_SERVE_SHORTEST 1
int lbm_server_set_policy(lbm_server s, int policy, long long max_resident_nodes);

/* Queue a request; never waits for the GPU.  *id identifies it.
 * Errors: LBM_EINVAL (bad request), LBM_ENOMEM (the request alone exceeds
 * the budget), LBM_ECLOSED. */
int lbm_submit(lbm_server s, const lbm_request *req, long long *id);

/* LBM_PENDING while the request runs; LBM_OK once finished: copies its
 * rho, ux, uy (host, ny x nx; any may be NULL) and the latency from submit
 * to results-on-host in seconds, then forgets the request.  A request that
 * failed returns its error code (and is forgotten). */
int lbm_poll(lbm_server s, long long id, double *rho, double *ux, double *uy,
             double *latency_s);

typedef struct {
  long long submitted, admitted, completed, failed;
  long long generations;    /* batched step chunks run                    */
  int resident;             /* lattices on the device now                 */
  int peak_resident;
  size_t resident_bytes, peak_bytes;
  double lattice_updates;   /* node-steps done                            */
  double busy_s;            /* wall time with work on the device          */
  int variant;              /* batch launch variant in use (-1: not yet    *
                             * tuned; tuned once on the first generation   *
                             * of >= 2^24 nodes, whose populations exceed  *
                             * the L2, the default variant until then)     */
} lbm_server_stats_t;
int lbm_server_stats(lbm_server s, lbm_server_stats_t *out);

/* ------------------------------------------------------------------
 * One periodic lattice split into y-slabs (multi-device decomposition).
 * The periodic lattice of section 2.1 (Eq. blbs and its lattice-closure
 * condition) couples row y only to rows y - 1 and y + 1, so a lattice can be
 * cut into slabs of whole rows, each stepped by its own device: per step
 * and slab boundary only the three populations that cross it move (c_y = +1,
 * i = 2, 5, 6 upwards; c_y = -1, i = 4, 7, 8 downwards), one row each.  Each
 * slab stores one halo row below and above its rows.  Results equal those of
 * the unsplit lattice bit for bit.  FP64, FP32 and BF16 storage (FP16 slabs
 * would need one storage scale for the whole lattice: LBM_EINVAL).
 *
 * lbm_slabs_create -- nslabs >= 1 slabs of an nx x ny lattice (arguments of
 * lbm_create); slab k owns rows [floor(k ny / nslabs), floor((k+1) ny /
 * nslabs)), on device devices[k] (NULL: all on the current device).  The
 * halo exchange after each step is a set of device-to-device (peer) copies
 * on a copy stream per slab, overlapped with the slab's interior rows (its
 * two boundary rows run first).  The group owns all device memory.
 * init_field / moments take whole-lattice host arrays (ny x nx), get / set
 * populations 9 x ny x nx ones, as the single-lattice calls; drift sums the
 * slabs' drifts in slab order.  Not thread-safe. */
typedef struct lbm_slabs_ctx *lbm_slabs;
int lbm_slabs_create(int nx, int ny, const double S[9], double rho0, const double u0[2],
                     int storage_dtype, int nslabs, const int *devices, lbm_slabs *out);
int lbm_slabs_rows(lbm_slabs s, int k, int *y0, int *rows, int *device);
int lbm_slabs_init_field(lbm_slabs s, const double *rho, const double *ux, const double *uy);
int lbm_slabs_set_populations(lbm_slabs s, const double *f);
int lbm_slabs_step(lbm_slabs s, long n);
int lbm_slabs_moments(lbm_slabs s, double *rho, double *ux, double *uy);
int lbm_slabs_get_populations(lbm_slabs s, double *f);
int lbm_slabs_drift(lbm_slabs s, double out[4]);
int lbm_slabs_destroy(lbm_slabs s);

/* One slab per process (the caller moves the halo rows, e.g. by NCCL
 * send / recv between ranks).  lbm_slab_create makes a handle for rows
 * [y0, y0 + rows) of an nx x ny_total periodic lattice; lbm_init_field,
 * lbm_set_populations, lbm_moments, lbm_get_populations and lbm_drift take
 * that slab's rows (rows x nx host arrays), lbm_step takes at most one step
 * per call, and analytic fields, point sources and batches are refused.
 * Between steps, and once after every init / set_populations with
 * reverse = 1, each rank calls
 *   lbm_slab_pack(h, reverse, to_below, to_above)
 * which copies its outgoing rows into two device buffers of
 * lbm_slab_halo_bytes bytes each (one part for the lower neighbour, slab
 * rows below y0 cyclically, one for the upper), sends to_below to the lower
 * neighbour and to_above to the upper one, receives their parts and calls
 *   lbm_slab_unpack(h, reverse, from_below, from_above)
 * (from_below: what the lower neighbour sent upwards).  reverse = 0 after a
 * step: halo rows take the neighbours' boundary rows; reverse = 1 after an
 * initialisation: the boundary slots that the neighbours' nodes initialised
 * come back.  Both calls are enqueued on the handle's stream
 * (lbm_set_stream) and do not synchronize. */
int lbm_slab_create(int nx, int ny_total, int y0, int rows, const double S[9], double rho0,
                    const double u0[2], int storage_dtype, lbm_handle *out);
int lbm_slab_halo_bytes(lbm_handle h, size_t *bytes);
int lbm_slab_pack(lbm_handle h, int reverse, void *to_below, void *to_above);
int lbm_slab_unpack(lbm_handle h, int reverse, const void *from_below, const void *from_above);

/* (runtime; no counterpart in the paper) Ids of requests that finished
 * (completed or failed) since the previous call, in finishing order: up to
 * cap ids are written to ids and their number to *count; the rest are kept
 * for the next call.  Lets a client poll only finished requests instead of
 * every pending one.  Thread-safe. */
int lbm_server_done(lbm_server s, long long *ids, int cap, int *count);

/* Stop admitting, wait for admitted work, free everything. */
int lbm_server_destroy(lbm_server s);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */

// Batched von Neumann analysis of the linearized D2Q9 MRT scheme on the
// device (lbm_vn_eigs in include/lbm.h).
//
// For every case the kernel builds the amplification matrix of section 4.1,
//   G(k) = diag(exp(-i k.c_j)) M^-1 Psi M,
// with Psi the linearized relaxation of section 2.3 about rho = 1 and the
// mean flow (U, V) (Psi = I - S + S J, J the Jacobian of the equilibrium
// moments with respect to rho, jx, jy), and returns its 9 eigenvalues
// lambda = exp(-i omega): per-step damping -ln|lambda| and phase speed
// -arg(lambda) / |k|.  One thread per case, FP64 complex arithmetic:
// Householder reduction to upper Hessenberg form, then shifted QR sweeps
// (Givens rotations, Wilkinson shifts, deflation on negligible subdiagonal
// entries) with a bounded number of sweeps per eigenvalue.
#include <math.h>

#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>

#include "bounds.cuh"
#include "lbm_internal.h"

namespace {

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx mk(double r, double i) { return cplx{r, i}; }
__device__ __forceinline__ cplx add(cplx a, cplx b) { return mk(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cplx sub(cplx a, cplx b) { return mk(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cplx mul(cplx a, cplx b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ cplx conj(cplx a) { return mk(a.re, -a.im); }
__device__ __forceinline__ cplx scale(cplx a, double s) { return mk(a.re * s, a.im * s); }
__device__ __forceinline__ double cabs(cplx a) { return hypot(a.re, a.im); }
__device__ cplx csqrt(cplx a) {
  const double r = cabs(a);
  if (r == 0.0) return mk(0, 0);
  double x = sqrt(0.5 * (r + fabs(a.re)));
  double y = a.im / (2.0 * x);
  if (a.re >= 0) return mk(x, y);
  return mk(fabs(y), a.im >= 0 ? x : -x);
}

constexpr int N = 9;

// Lallemand-Luo D2Q9 moment matrix in the paper's row order and row norms
__device__ __forceinline__ int mrow(int k, int j) {
  constexpr int T[9][9] = {
      {1, 1, 1, 1, 1, 1, 1, 1, 1},     {0, 1, 0, -1, 0, 1, -1, -1, 1},
      {0, 0, 1, 0, -1, 1, 1, -1, -1},  {-4, -1, -1, -1, -1, 2, 2, 2, 2},
      {4, -2, -2, -2, -2, 1, 1, 1, 1}, {0, -2, 0, 2, 0, 1, -1, -1, 1},
      {0, 0, -2, 0, 2, 1, 1, -1, -1},  {0, 1, -1, 1, -1, 0, 0, 0, 0},
      {0, 0, 0, 0, 0, 1, -1, 1, -1}};
  return T[k][j];
}
__device__ __forceinline__ double rnorm(int k) {
  return k == 0 ? 9.0 : (k <= 2 ? 6.0 : (k <= 4 ? 36.0 : (k <= 6 ? 12.0 : 4.0)));
}

// Psi about rho = 1, j = (U, V): rows 0..2 identity; row k >= 3 has 1 - s_k
// on the diagonal and s_k dm^eq_k / d(rho, jx, jy) in columns 0..2.
__device__ void build_psi(const double s[9], double U, double V, double P[9][9]) {
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) P[i][j] = (i == j) ? 1.0 : 0.0;
  const double u2 = U * U + V * V;
  // Jacobian of {-2 rho + 3|j|^2/rho, rho - 3|j|^2/rho, -jx, -jy,
  // (jx^2 - jy^2)/rho, jx jy/rho} at (1, U, V)
  const double J[6][3] = {{-2.0 - 3.0 * u2, 6.0 * U, 6.0 * V},
                          {1.0 + 3.0 * u2, -6.0 * U, -6.0 * V},
                          {0.0, -1.0, 0.0},
                          {0.0, 0.0, -1.0},
                          {-(U * U - V * V), 2.0 * U, -2.0 * V},
                          {-U * V, V, U}};
  for (int r = 0; r < 6; ++r) {
    const int k = 3 + r;
    P[k][k] = 1.0 - s[k];
    for (int c = 0; c < 3; ++c) P[k][c] = s[k] * J[r][c];
  }
}

// Householder reduction of A to upper Hessenberg form, in place
__device__ void hessenberg(cplx A[9][9]) {
  for (int k = 0; k < N - 2; ++k) {
    double nrm = 0;
    for (int i = k + 1; i < N; ++i) nrm += A[i][k].re * A[i][k].re + A[i][k].im * A[i][k].im;
    nrm = sqrt(nrm);
    if (nrm == 0.0) continue;
    const int k1 = lbm::bounds::ck(k + 1, N, lbm::bounds::VN_HESS);
    const cplx x0 = A[k1][k];
    const double a0 = cabs(x0);
    const cplx ph = a0 > 0 ? scale(x0, 1.0 / a0) : mk(1, 0);
    cplx v[9];
    for (int i = 0; i < N; ++i) v[i] = mk(0, 0);
    // v = x + e^{i arg x0} ||x|| e1, normalized
    v[k1] = add(x0, scale(ph, nrm));
    for (int i = k + 2; i < N; ++i) v[i] = A[i][k];
    double vn = 0;
    for (int i = k + 1; i < N; ++i) vn += v[i].re * v[i].re + v[i].im * v[i].im;
    vn = sqrt(vn);
    if (vn == 0.0) continue;
    for (int i = k + 1; i < N; ++i) v[i] = scale(v[i], 1.0 / vn);
    // A <- (I - 2 v v^H) A
    for (int j = 0; j < N; ++j) {
      cplx d = mk(0, 0);
      for (int i = k + 1; i < N; ++i) d = add(d, mul(conj(v[i]), A[i][j]));
      for (int i = k + 1; i < N; ++i) A[i][j] = sub(A[i][j], scale(mul(v[i], d), 2.0));
    }
    // A <- A (I - 2 v v^H)
    for (int i = 0; i < N; ++i) {
      cplx d = mk(0, 0);
      for (int j = k + 1; j < N; ++j) d = add(d, mul(A[i][j], v[j]));
      for (int j = k + 1; j < N; ++j) A[i][j] = sub(A[i][j], scale(mul(d, conj(v[j])), 2.0));
    }
    for (int i = k + 2; i < N; ++i) A[i][k] = mk(0, 0);
  }
}

// Eigenvalues of the Hessenberg matrix H by shifted QR; returns the number
// of eigenvalues that did not converge within the sweep limit (reported as
// the current diagonal entries).
__device__ int hqr(cplx H[9][9], cplx ev[9]) {
  const double eps = 2.220446049250313e-16;
  int hi = N - 1, iter = 0, failed = 0;
  while (hi >= 0) {
    if (hi == 0) {
      ev[0] = H[0][0];
      break;
    }
    int l = hi;
    for (; l > 0; --l) {
      const int lm = lbm::bounds::ck(l - 1, N, lbm::bounds::VN_HQR);
      const double s = cabs(H[lm][lm]) + cabs(H[l][l]);
      if (cabs(H[l][lm]) <= eps * (s > 0 ? s : 1.0)) {
        H[l][lm] = mk(0, 0);
        break;
      }
    }
    if (l == hi) {  // one eigenvalue deflates
      ev[hi] = H[hi][hi];
      --hi;
      iter = 0;
      continue;
    }
    if (iter >= 60) {  // give up on this one, keep going
      ev[hi] = H[hi][hi];
      ++failed;
      --hi;
      iter = 0;
      continue;
    }
    // Wilkinson shift from the trailing 2x2 block; an exceptional shift
    // every 11 sweeps breaks cycles
    cplx mu;
    const int hm = lbm::bounds::ck(hi - 1, N, lbm::bounds::VN_HQR);
    if (iter > 0 && iter % 11 == 0) {
      mu = add(H[hi][hi], mk(fabs(H[hi][hm].re) + fabs(H[hm][hi > 1 ? hi - 2 : 0].re), 0));
    } else {
      const cplx a = H[hm][hm], b = H[hm][hi], c = H[hi][hm], d = H[hi][hi];
      const cplx half_tr = scale(add(a, d), 0.5);
      const cplx det = sub(mul(a, d), mul(b, c));
      const cplx disc = csqrt(sub(mul(half_tr, half_tr), det));
      const cplx m1 = add(half_tr, disc), m2 = sub(half_tr, disc);
      mu = cabs(sub(m1, d)) < cabs(sub(m2, d)) ? m1 : m2;
    }
    ++iter;
    // one QR sweep on rows/columns l..hi of H - mu I
    double gc[9];
    cplx gs[9];
    for (int i = l; i <= hi; ++i) H[i][i] = sub(H[i][i], mu);
    for (int k = l; k < hi; ++k) {
      const int k1 = lbm::bounds::ck(k + 1, N, lbm::bounds::VN_HQR);
      const cplx x = H[k][k], y = H[k1][k];
      const double ax = cabs(x), r = hypot(ax, cabs(y));
      double c;
      cplx s;
      if (r == 0.0) {
        c = 1.0;
        s = mk(0, 0);
      } else if (ax == 0.0) {
        c = 0.0;  // x = 0: swap the rows (s = 1)
        s = mk(1, 0);
      } else {
        c = ax / r;
        s = scale(mul(scale(x, 1.0 / ax), conj(y)), 1.0 / r);
      }
      gc[k] = c;
      gs[k] = s;
      for (int j = k; j <= hi; ++j) {
        const cplx hk = H[k][j], hk1 = H[k1][j];
        H[k][j] = add(scale(hk, c), mul(s, hk1));
        H[k1][j] = sub(scale(hk1, c), mul(conj(s), hk));
      }
    }
    for (int k = l; k < hi; ++k) {
      const double c = gc[k];
      const cplx s = gs[k];
      const int top = lbm::bounds::ck(k + 2 < hi ? k + 2 : hi, N, lbm::bounds::VN_HQR);
      const int k1 = lbm::bounds::ck(k + 1, N, lbm::bounds::VN_HQR);
      for (int i = l; i <= top; ++i) {
        const cplx hk = H[i][k], hk1 = H[i][k1];
        H[i][k] = add(scale(hk, c), mul(hk1, conj(s)));
        H[i][k1] = sub(scale(hk1, c), mul(hk, s));
      }
    }
    for (int i = l; i <= hi; ++i) H[i][i] = add(H[i][i], mu);
  }
  return failed;
}

struct VnCase {
  double kx, ky, U, V;
  double s[9];  // paper order
};

__global__ void k_vn_eigs(const VnCase *__restrict__ cases, int n, double *__restrict__ out,
                          int *__restrict__ failed) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const VnCase K = cases[c];
  double P[9][9];
  build_psi(K.s, K.U, K.V, P);
  // C = M^-1 Psi M = M^T D^-1 Psi M
  double PM[9][9];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double acc = 0;
      for (int k = 0; k < N; ++k) acc += P[i][k] * mrow(k, j);
      PM[i][j] = acc;
    }
  cplx G[9][9];
  for (int i = 0; i < N; ++i) {
    // phase of streaming direction i: exp(-i k.c_i)
    const double ph = -(K.kx * lbm::CXd(i) + K.ky * lbm::CYd(i));
    const cplx e = mk(cos(ph), sin(ph));
    for (int j = 0; j < N; ++j) {
      double acc = 0;
      for (int k = 0; k < N; ++k) acc += (mrow(k, i) / rnorm(k)) * PM[k][j];
      G[i][j] = scale(e, acc);
    }
  }
  hessenberg(G);
  cplx ev[9];
  const int f = hqr(G, ev);
  for (int i = 0; i < N; ++i) {
    out[(long long)c * 18 + 2 * i] = ev[i].re;
    out[(long long)c * 18 + 2 * i + 1] = ev[i].im;
  }
  if (f) atomicAdd(failed, f);
}

}  // namespace

namespace {

// Staging of lbm_vn_eigs, kept for the life of the process and grown to
// the largest call: page-locked host copies of the cases and results,
// their device copies, and one stream per chunk.  A call cuts its cases
// into up to kVnChunks chunks; the host fills chunk j while chunk j-1 is
// uploaded and solved, every chunk's kernel runs on its own stream (all of
// them together fill the GPU: one thread's QR iteration is a long
// dependent chain, so the kernel wants every case in flight at once), and
// the host drains each chunk's eigenvalues as soon as they are back.
constexpr int kVnChunks = 8;
constexpr int kVnMinChunk = 4096;

struct VnStage {
  int device = -1;
  long long cap = 0;
  VnCase *h_in = nullptr, *d_in = nullptr;
  double *h_out = nullptr, *d_out = nullptr;
  int *d_fail = nullptr;
  cudaStream_t st[kVnChunks] = {};
  cudaEvent_t ev[kVnChunks] = {};
};

std::mutex g_vn_mu;
VnStage g_vn;  // its CUDA objects are never released (none may be at process exit)

void vn_release(VnStage &v) {
  cudaFreeHost(v.h_in);
  cudaFreeHost(v.h_out);
  cudaFree(v.d_in);
  cudaFree(v.d_out);
  v.h_in = v.d_in = nullptr;
  v.h_out = v.d_out = nullptr;
  v.cap = 0;
  cudaGetLastError();
}

cudaError_t vn_ready(VnStage &v, long long n) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (v.device != dev) {
    if (v.device >= 0) {
      // staging of another device: let it go (on that device)
      cudaSetDevice(v.device);
      vn_release(v);
      cudaFree(v.d_fail);
      v.d_fail = nullptr;
      for (int k = 0; k < kVnChunks; ++k) {
        cudaStreamDestroy(v.st[k]);
        cudaEventDestroy(v.ev[k]);
        v.st[k] = nullptr;
        v.ev[k] = nullptr;
      }
      cudaSetDevice(dev);
      cudaGetLastError();
    }
    v.device = -1;
    for (int k = 0; k < kVnChunks; ++k) {
      if ((e = cudaStreamCreateWithFlags(&v.st[k], cudaStreamNonBlocking)) != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&v.ev[k], cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    if ((e = cudaMalloc(&v.d_fail, sizeof(int))) != cudaSuccess) return e;
    v.device = dev;
  }
  if (n > v.cap) {
    vn_release(v);
    if ((e = cudaHostAlloc(&v.h_in, sizeof(VnCase) * n, cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaHostAlloc(&v.h_out, sizeof(double) * 18 * n, cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaMalloc(&v.d_in, sizeof(VnCase) * n)) != cudaSuccess ||
        (e = cudaMalloc(&v.d_out, sizeof(double) * 18 * n)) != cudaSuccess) {
      vn_release(v);
      return e;
    }
    v.cap = n;
  }
  return cudaSuccess;
}

}  // namespace

extern "C" int lbm_vn_eigs(int n, const double *kx, const double *ky, const double *U,
                           const double *V, const double *S, double *eig, int *unconverged) {
  using namespace lbm;
  if (n < 0 || (n > 0 && (!kx || !ky || !U || !V || !S || !eig))) {
    set_error("lbm_vn_eigs: bad arguments");
    return LBM_EINVAL;
  }
  if (unconverged) *unconverged = 0;
  if (n == 0) return LBM_OK;
  const int ll_of_paper[9] = {0, 3, 5, 1, 2, 4, 6, 7, 8};
  std::lock_guard<std::mutex> lk(g_vn_mu);
  VnStage &v = g_vn;
  cudaError_t e = vn_ready(v, n);
  const int nch = std::max(1, std::min(kVnChunks, n / kVnMinChunk));
  auto lo = [&](int j) { return (int)((long long)n * j / nch); };
  // zero the failure count before any chunk stream runs (the legacy
  // stream of a plain memset does not order the non-blocking streams)
  if (e == cudaSuccess) e = cudaMemsetAsync(v.d_fail, 0, sizeof(int), v.st[0]);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.st[0]);
  int launched = 0;
  for (int j = 0; j < nch && e == cudaSuccess; ++j) {
    const int c0 = lo(j), c1 = lo(j + 1), cnt = c1 - c0;
    for (int c = c0; c < c1; ++c) {
      VnCase &k = v.h_in[c];
      k.kx = kx[c];
      k.ky = ky[c];
      k.U = U[c];
      k.V = V[c];
      for (int q = 0; q < 9; ++q) k.s[q] = S[9LL * c + ll_of_paper[q]];
    }
    e = cudaMemcpyAsync(v.d_in + c0, v.h_in + c0, sizeof(VnCase) * cnt, cudaMemcpyHostToDevice,
                        v.st[j]);
    if (e == cudaSuccess) {
      k_vn_eigs<<<(cnt + 127) / 128, 128, 0, v.st[j]>>>(v.d_in + c0, cnt, v.d_out + 18LL * c0,
                                                        v.d_fail);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(v.h_out + 18LL * c0, v.d_out + 18LL * c0, sizeof(double) * 18 * cnt,
                          cudaMemcpyDeviceToHost, v.st[j]);
    if (e == cudaSuccess) e = cudaEventRecord(v.ev[j], v.st[j]);
    if (e == cudaSuccess) ++launched;
  }
  // drain each chunk as it lands (after an error: wait for what was queued)
  for (int j = 0; j < launched; ++j) {
    const cudaError_t w = cudaEventSynchronize(v.ev[j]);
    if (e == cudaSuccess) e = w;
    if (e == cudaSuccess)
      memcpy(eig + 18LL * lo(j), v.h_out + 18LL * lo(j), sizeof(double) * 18 * (lo(j + 1) - lo(j)));
  }
  int fails = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&fails, v.d_fail, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_error(std::string("lbm_vn_eigs: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
  }
  if (unconverged) *unconverged = fails;
  return fails ? LBM_ETIMEOUT : LBM_OK;
}

namespace lbm {
unsigned bounds_word_vn(bool reset) { return bounds::read_word(reset); }
}  // namespace lbm

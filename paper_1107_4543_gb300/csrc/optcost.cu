// Cost functions of the free-parameter optimization (sections 2.2, 3 and
// 4.2) on the device, and the optimizer built on them (lbm_opt_cost,
// lbm_opt_minimize in include/lbm.h).
//
// For a wave direction theta and a mean flow (U, V) the recursive algorithm
// of section 2.2 gives the conserved-quantity equation dW/dt = B_n W with
// B_n = sum_{l<n} dt^l k^(l+1) b^l(theta).  With |k| = 1 and dt kept formal,
// every matrix of the two recursions (Eqs. R-A/R-B for the moment map
// m = Phi W, Eqs. R-D/R-E for B) is a polynomial in dt stored as its
// coefficients, and matrix powers of B are taken in that polynomial ring,
// truncated at dt^(n-1).  The scheme's operators A_l = (1/l!) M
// diag((-i v.k)^l) M^-1 Psi are applied as M (d_l o (G X)) with G = M^-1 Psi,
// never formed.
//
// One warp per quadrature point (theta, flow direction, flow speed), its
// polynomial matrices in shared memory and one lane per matrix entry.  The
// wave-number integral over dt k in [0, pi] of ||M_eps||_F^2, M_eps =
// sum_l (dt k)^(l+1) (b^l - b_exact^l), is taken in closed form per point;
// the point sums are reduced in a fixed order per candidate, so results are
// reproducible bit for bit.
#include <math.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

namespace {

constexpr int NMAX = 6;                       // largest truncation order
constexpr int SLOTS = NMAX * (NMAX + 1) / 2;  // coefficients of orders 1..NMAX
constexpr int WPB = 4;                        // warps (points) per block
constexpr int MAX_SPEED = 32;

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx cx(double r, double i) { return cplx{r, i}; }
__device__ __forceinline__ cplx operator+(cplx a, cplx b) { return cx(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cplx operator-(cplx a, cplx b) { return cx(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ cplx operator*(double s, cplx a) { return cx(s * a.re, s * a.im); }

// D2Q9 velocities (the order of the step kernels) and the Lallemand-Luo
// moment matrix in the paper's row order with its row norms
__device__ __forceinline__ int vx(int j) {
  return j == 1 || j == 5 || j == 8 ? 1 : (j == 3 || j == 6 || j == 7 ? -1 : 0);
}
__device__ __forceinline__ int vy(int j) {
  return j == 2 || j == 5 || j == 6 ? 1 : (j == 4 || j == 7 || j == 8 ? -1 : 0);
}
__device__ __forceinline__ int mm(int k, int j) {
  const int c2 = vx(j) * vx(j) + vy(j) * vy(j);
  switch (k) {
    case 0: return 1;
    case 1: return vx(j);
    case 2: return vy(j);
    case 3: return 3 * c2 - 4;
    case 4: return (9 * c2 * c2 - 21 * c2 + 8) / 2;
    case 5: return (3 * c2 - 5) * vx(j);
    case 6: return (3 * c2 - 5) * vy(j);
    case 7: return vx(j) * vx(j) - vy(j) * vy(j);
    default: return vx(j) * vy(j);
  }
}
__device__ __forceinline__ double dnorm(int k) {
  return k == 0 ? 9.0 : (k <= 2 ? 6.0 : (k <= 4 ? 36.0 : (k <= 6 ? 12.0 : 4.0)));
}

struct Rates {
  double s[9];  // paper order; s[0..2] unused
};

// the printed Psi of section 2.3 about rho = 1, j = (U, V)
__device__ double psi(int r, int c, double U, double V, const Rates &R) {
  const double se = R.s[3], seps = R.s[4], sq = R.s[5], snu = R.s[7];
  const double u2 = U * U + V * V;
  if (r == c) return r < 3 ? 1.0 : 1.0 - R.s[r];
  switch (r) {
    case 3: return c == 0 ? (-2 * se - 3 * u2 * se) : c == 1 ? 6 * U * se : c == 2 ? 6 * V * se : 0.0;
    case 4: return c == 0 ? (seps + 3 * u2 * seps) : c == 1 ? -6 * U * seps : c == 2 ? -6 * V * seps : 0.0;
    case 5: return c == 1 ? -sq : 0.0;
    case 6: return c == 2 ? -sq : 0.0;
    case 7: return c == 0 ? -(U * U - V * V) * snu : c == 1 ? 2 * U * snu : c == 2 ? -2 * V * snu : 0.0;
    case 8: return c == 0 ? -U * V * snu : c == 1 ? V * snu : c == 2 ? U * snu : 0.0;
    default: return 0.0;
  }
}

__device__ __forceinline__ int slot(int m, int d) { return m * (m - 1) / 2 + d; }

struct WarpMem {
  double G[81];          // M^-1 Psi
  cplx d[NMAX + 1][9];   // d_l,j = (-i v_j.k)^l / l!
  cplx phi[SLOTS][27];   // Phi_m, 9 x 3, coefficient d at slot(m, d)
  cplx B[SLOTS][9];      // B_m, 3 x 3
  cplx Y[27];            // G X
  cplx P[NMAX][9];       // powers of B
  cplx P2[NMAX][9];
  cplx T[27];            // rows 0..2 of A_l Phi (scratch)
  double part[9];
};

struct CostSpec {
  int kind;       // 0: zero mean flow (F), 1: mean flows (G)
  int order;      // truncation order n
  int part;       // 0 all, 1 odd powers of K, 2 even powers
  int reference;  // 0 convection + dissipation, 1 convection, 2 convection + shear
  int n_theta, n_dir, n_speed;
  double u0;
  double su[MAX_SPEED], wu[MAX_SPEED];  // speed nodes and weights
};

// out (rows lo..hi-1 of the 9 x 3 result, others untouched) += coef * A_l X
__device__ void apply_A(WarpMem &w, int l, const cplx *X, cplx *out, int lo, int hi, double coef,
                        int lane) {
  if (lane < 27) {
    const int r = lane / 3, c = lane % 3;
    cplx y = cx(0, 0);
#pragma unroll
    for (int j = 0; j < 9; ++j) y = y + w.G[r * 9 + j] * X[j * 3 + c];
    w.Y[lane] = w.d[l][r] * y;
  }
  __syncwarp();
  if (lane < 27) {
    const int r = lane / 3, c = lane % 3;
    if (r >= lo && r < hi) {
      cplx z = cx(0, 0);
#pragma unroll
      for (int j = 0; j < 9; ++j) z = z + (double)mm(r, j) * w.Y[j * 3 + c];
      out[lane] = out[lane] + coef * z;
    }
  }
  __syncwarp();
}

// P (3 x 3 polynomial, degrees 0..maxdeg) = B_m^p truncated
__device__ void bpow(WarpMem &w, int m, int p, int maxdeg, int lane) {
  for (int d = 0; d <= maxdeg; ++d)
    if (lane < 9) w.P[d][lane] = d < m ? w.B[slot(m, d)][lane] : cx(0, 0);
  __syncwarp();
  for (int q = 1; q < p; ++q) {
    if (lane < 9) {
      const int r = lane / 3, c = lane % 3;
      for (int d = 0; d <= maxdeg; ++d) {
        cplx acc = cx(0, 0);
        for (int a = 0; a <= d; ++a) {
          const int b = d - a;
          if (b >= m) continue;
#pragma unroll
          for (int k = 0; k < 3; ++k) acc = acc + w.P[a][r * 3 + k] * w.B[slot(m, b)][k * 3 + c];
        }
        w.P2[d][lane] = acc;
      }
    }
    __syncwarp();
    for (int d = 0; d <= maxdeg; ++d)
      if (lane < 9) w.P[d][lane] = w.P2[d][lane];
    __syncwarp();
  }
}

// exact coefficients (convection b_ex^0, dissipation b_ex^1) at |k| = 1
__device__ cplx exact_entry(int l, int e, double kx, double ky, double U, double V,
                            const CostSpec &cs, double sig_e, double sig_nu) {
  const int r = e / 3, c = e % 3;
  if (l == 0) {
    double v = 0.0;
    if (r == 0) v = c == 1 ? -kx : (c == 2 ? -ky : 0.0);
    if (r == 1) v = c == 0 ? (-kx / 3 + kx * U * U + ky * U * V) : (c == 1 ? (-2 * kx * U - ky * V) : -ky * U);
    if (r == 2) v = c == 0 ? (-ky / 3 + ky * V * V + kx * U * V) : (c == 1 ? -kx * V : (-2 * ky * V - kx * U));
    return cx(0.0, v);
  }
  if (l != 1 || cs.reference == 1) return cx(0, 0);
  const double se = cs.reference == 2 ? 0.0 : sig_e;
  double v = 0.0;
  if (r == 1 && c == 1) v = -(kx * kx * se + (kx * kx + ky * ky) * sig_nu) / 3;
  if ((r == 1 && c == 2) || (r == 2 && c == 1)) v = -kx * ky * se / 3;
  if (r == 2 && c == 2) v = -(ky * ky * se + (kx * kx + ky * ky) * sig_nu) / 3;
  return cx(v, 0.0);
}

__global__ void __launch_bounds__(WPB * 32)
k_opt_points(CostSpec cs, const double *__restrict__ sigmas, long long npoints,
             double *__restrict__ partial) {
  extern __shared__ unsigned char smem_raw[];
  WarpMem &w = reinterpret_cast<WarpMem *>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const long long p = (long long)blockIdx.x * WPB + (threadIdx.x >> 5);
  const int cand = blockIdx.y;
  if (p >= npoints) return;  // warp-uniform
  const int n = cs.order;

  // the point: theta (fastest), flow direction, flow speed
  const int it = (int)(p % cs.n_theta);
  const long long q = p / cs.n_theta;
  const int id = (int)(q % cs.n_dir);
  const int iu = (int)(q / cs.n_dir);
  const double th = 2.0 * M_PI * it / cs.n_theta;
  const double kx = cos(th), ky = sin(th);
  double U = 0.0, V = 0.0, weight = 2.0 * M_PI / cs.n_theta;
  if (cs.kind == 1) {
    const double ph = 2.0 * M_PI * id / cs.n_dir;
    U = cs.su[iu] * cos(ph);
    V = cs.su[iu] * sin(ph);
    weight *= 2.0 * M_PI / cs.n_dir * cs.wu[iu];
  }
  const double *sg = sigmas + 4 * (long long)cand;  // sigma_e, sigma_eps, sigma_q, sigma_nu
  Rates R;
  R.s[0] = R.s[1] = R.s[2] = 0.0;
  R.s[3] = 1.0 / (sg[0] + 0.5);
  R.s[4] = 1.0 / (sg[1] + 0.5);
  R.s[5] = R.s[6] = 1.0 / (sg[2] + 0.5);
  R.s[7] = R.s[8] = 1.0 / (sg[3] + 0.5);

  for (int e = lane; e < 81; e += 32) {
    const int r = e / 9, c = e % 9;
    double g = 0.0;
    for (int k = 0; k < 9; ++k) g += (double)mm(k, r) / dnorm(k) * psi(k, c, U, V, R);
    w.G[e] = g;
  }
  if (lane < 9) {
    const double vk = vx(lane) * kx + vy(lane) * ky;
    cplx pw = cx(1.0, 0.0);
    double fact = 1.0;
    w.d[0][lane] = pw;
    for (int l = 1; l <= n; ++l) {
      pw = pw * cx(0.0, -vk);
      fact *= l;
      w.d[l][lane] = (1.0 / fact) * pw;
    }
  }
  // Phi_1: identity on the conserved rows, Psi_ic / s_i below
  if (lane < 27) {
    const int r = lane / 3, c = lane % 3;
    w.phi[slot(1, 0)][lane] = r < 3 ? cx(r == c ? 1.0 : 0.0, 0.0) : cx(psi(r, c, U, V, R) / R.s[r], 0.0);
  }
  if (lane < 27) w.T[lane] = cx(0, 0);
  __syncwarp();
  // B_1 = rows 0..2 of A_1 Phi_1 (entries 0..8 of the 9 x 3 product)
  apply_A(w, 1, w.phi[slot(1, 0)], w.T, 0, 3, 1.0, lane);
  if (lane < 9) w.B[slot(1, 0)][lane] = w.T[lane];
  __syncwarp();

  for (int m = 2; m <= n; ++m) {
    const int deg = m - 1;
    // Phi_m accumulated in its slots: degree 0 = Psi (columns 0..2)
    for (int d = 0; d < m; ++d)
      if (lane < 27) {
        const int r = lane / 3, c = lane % 3;
        w.phi[slot(m, d)][lane] = d == 0 ? cx(psi(r, c, U, V, R), 0.0) : cx(0, 0);
      }
    __syncwarp();
    double fact = 1.0;
    for (int l = 1; l < m; ++l) {
      fact *= l;
      const int md = deg - l;  // degrees kept in the shifted terms
      bpow(w, m - l, l, md, lane);
      // T = Phi_{m-l} B_{m-l}^l, degrees 0..md
      if (lane < 27) {
        const int r = lane / 3, c = lane % 3;
        for (int d = 0; d <= md; ++d) {
          cplx acc = cx(0, 0);
          for (int a = 0; a <= d && a < m - l; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k)
              acc = acc + w.phi[slot(m - l, a)][r * 3 + k] * w.P[d - a][k * 3 + c];
          w.phi[slot(m, d + l)][lane] = w.phi[slot(m, d + l)][lane] - (1.0 / fact) * acc;
        }
      }
      __syncwarp();
      for (int a = 0; a < m - l && a + l <= deg; ++a)
        apply_A(w, l, w.phi[slot(m - l, a)], w.phi[slot(m, a + l)], 3, 9, 1.0, lane);
    }
    // rows 3..8 divided by s_i; rows 0..2 the identity
    for (int d = 0; d < m; ++d)
      if (lane < 27) {
        const int r = lane / 3, c = lane % 3;
        cplx v = w.phi[slot(m, d)][lane];
        if (r < 3) v = cx(d == 0 && r == c ? 1.0 : 0.0, 0.0);
        else v = (1.0 / R.s[r]) * v;
        w.phi[slot(m, d)][lane] = v;
      }
    __syncwarp();
    // B_m
    for (int d = 0; d < m; ++d)
      if (lane < 9) w.B[slot(m, d)][lane] = cx(0, 0);
    __syncwarp();
    fact = 1.0;
    for (int l = 1; l < m; ++l) {
      fact *= (l + 1);
      const int md = deg - l;
      bpow(w, m - l, l + 1, md, lane);
      if (lane < 9)
        for (int d = 0; d <= md; ++d)
          w.B[slot(m, d + l)][lane] = w.B[slot(m, d + l)][lane] - (1.0 / fact) * w.P[d][lane];
      __syncwarp();
    }
    for (int l = 1; l <= m; ++l) {
      const int src = m + 1 - l;
      for (int a = 0; a < src && a + l - 1 <= deg; ++a) {
        if (lane < 27) w.T[lane] = cx(0, 0);
        __syncwarp();
        apply_A(w, l, w.phi[slot(src, a)], w.T, 0, 3, 1.0, lane);
        if (lane < 9) w.B[slot(m, a + l - 1)][lane] = w.B[slot(m, a + l - 1)][lane] + w.T[lane];
        __syncwarp();
      }
    }
  }

  // closed-form K integral of ||sum_l K^(l+1) E^l||^2 over [0, pi]
  if (lane < 9) {
    double acc = 0.0;
    for (int l = 0; l < n; ++l) {
      const bool odd_l = ((l + 1) & 1) != 0;
      if ((cs.part == 1 && !odd_l) || (cs.part == 2 && odd_l)) continue;
      const cplx El = w.B[slot(n, l)][lane] - exact_entry(l, lane, kx, ky, U, V, cs, sg[0], sg[3]);
      for (int mq = 0; mq < n; ++mq) {
        const bool odd_m = ((mq + 1) & 1) != 0;
        if ((cs.part == 1 && !odd_m) || (cs.part == 2 && odd_m)) continue;
        const cplx Em =
            w.B[slot(n, mq)][lane] - exact_entry(mq, lane, kx, ky, U, V, cs, sg[0], sg[3]);
        const int pw = l + mq + 3;
        acc += (El.re * Em.re + El.im * Em.im) * pow(M_PI, pw) / pw;
      }
    }
    w.part[lane] = acc;
  }
  __syncwarp();
  if (lane == 0) {
    double v = 0.0;
    for (int e = 0; e < 9; ++e) v += w.part[e];
    partial[(long long)cand * npoints + p] = v * weight;
  }
}

// per candidate: the point values summed by a fixed tree
__global__ void __launch_bounds__(256)
k_opt_reduce(const double *__restrict__ partial, long long npoints, double *__restrict__ out) {
  __shared__ double sh[256];
  const int cand = blockIdx.x;
  double acc = 0.0;
  for (long long p = threadIdx.x; p < npoints; p += 256) acc += partial[(long long)cand * npoints + p];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int wdt = 128; wdt > 0; wdt >>= 1) {
    if (threadIdx.x < wdt) sh[threadIdx.x] += sh[threadIdx.x + wdt];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[cand] = sh[0];
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's iteration on the
// Legendre three-term recurrence (the classical method), nodes ascending
void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p0 = 1.0;
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n == 1 ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
    const double wt = 2.0 / ((1.0 - z * z) * dp * dp);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = wt;
  }
}

int make_spec(const lbm_cost_spec *in, CostSpec *cs) {
  if (!in) return LBM_EINVAL;
  cs->kind = in->kind;
  cs->order = in->order;
  cs->part = in->part;
  cs->reference = in->reference;
  cs->u0 = in->u0;
  if (cs->kind != LBM_COST_F && cs->kind != LBM_COST_G) return LBM_EINVAL;
  if (cs->order < 1 || cs->order > NMAX) return LBM_EINVAL;
  if (cs->part < 0 || cs->part > 2 || cs->reference < 0 || cs->reference > 2) return LBM_EINVAL;
  // exact for the integrands of orders <= NMAX (trigonometric / polynomial
  // degrees grow with the order)
  cs->n_theta = 4 * cs->order + 4;
  if (cs->kind == LBM_COST_F) {
    cs->n_dir = 1;
    cs->n_speed = 1;
    cs->su[0] = 0.0;
    cs->wu[0] = 1.0;
  } else {
    if (!(cs->u0 >= 0.0) || !std::isfinite(cs->u0)) return LBM_EINVAL;
    cs->n_dir = 6 * cs->order;
    cs->n_speed = 2 * cs->order + 2;
    if (in->fixed_speed) {
      cs->n_speed = 1;
      cs->su[0] = cs->u0;
      cs->wu[0] = 1.0;
    } else {
      double x[MAX_SPEED], w[MAX_SPEED];
      gauss_legendre(cs->n_speed, x, w);
      for (int i = 0; i < cs->n_speed; ++i) {
        cs->su[i] = 0.5 * cs->u0 * (x[i] + 1.0);
        cs->wu[i] = 0.5 * cs->u0 * w[i];
      }
    }
  }
  return LBM_OK;
}

// device buffers of the cost evaluations, grown on demand and reused by the
// many small evaluations of a minimization
struct Workspace {
  double *sig = nullptr, *part = nullptr, *out = nullptr;
  size_t cap_n = 0, cap_part = 0;
  ~Workspace() {
    lbm::dev_free(sig);
    lbm::dev_free(part);
    lbm::dev_free(out);
  }
  bool ensure(size_t n, size_t npart) {
    if (n > cap_n) {
      lbm::dev_free(sig);
      lbm::dev_free(out);
      sig = (double *)lbm::dev_alloc(sizeof(double) * 4 * n);
      out = (double *)lbm::dev_alloc(sizeof(double) * n);
      cap_n = (sig && out) ? n : 0;
      if (!cap_n) return false;
    }
    if (npart > cap_part) {
      lbm::dev_free(part);
      part = (double *)lbm::dev_alloc(sizeof(double) * npart);
      cap_part = part ? npart : 0;
      if (!cap_part) return false;
    }
    return true;
  }
};

int eval_costs(Workspace &ws, const CostSpec &cs, int n, const double *sig_host,
               double *out_host) {
  const long long npoints = (long long)cs.n_theta * cs.n_dir * cs.n_speed;
  if (!ws.ensure((size_t)n, (size_t)npoints * n)) {
    lbm::set_error("out of device memory for the cost evaluation");
    return LBM_ENOMEM;
  }
  cudaError_t e = cudaMemcpy(ws.sig, sig_host, sizeof(double) * 4 * n, cudaMemcpyHostToDevice);
  const size_t shm = sizeof(WarpMem) * WPB;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_opt_points, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e == cudaSuccess) {
    dim3 grid((unsigned)((npoints + WPB - 1) / WPB), (unsigned)n);
    k_opt_points<<<grid, WPB * 32, shm>>>(cs, ws.sig, npoints, ws.part);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_opt_reduce<<<n, 256>>>(ws.part, npoints, ws.out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out_host, ws.out, sizeof(double) * n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    lbm::set_error(std::string("cost evaluation: ") + cudaGetErrorString(e));
    cudaGetLastError();
    return LBM_ECUDA;
  }
  return LBM_OK;
}

bool valid_sigmas(const double *s) {
  for (int i = 0; i < 4; ++i)
    if (!(s[i] >= 0.0) || !std::isfinite(s[i])) return false;
  return true;
}

}  // namespace

extern "C" {

int lbm_opt_cost(const lbm_cost_spec *spec, int n, const double *sigmas, double *out) {
  lbm::NvtxRange nvtx("lbm_opt_cost");
  if (n < 0 || (n > 0 && (!sigmas || !out))) {
    lbm::set_error("bad cost arguments");
    return LBM_EINVAL;
  }
  CostSpec cs;
  if (make_spec(spec, &cs) != LBM_OK) {
    lbm::set_error("bad cost specification");
    return LBM_EINVAL;
  }
  for (int i = 0; i < n; ++i)
    if (!valid_sigmas(sigmas + 4 * i)) {
      lbm::set_error("sigmas must be finite and >= 0 (s in (0, 2])");
      return LBM_EINVAL;
    }
  if (n == 0) return LBM_OK;
  Workspace ws;
  return eval_costs(ws, cs, n, sigmas, out);
}

int lbm_opt_minimize(const lbm_cost_spec *spec, const double sigmas_in[4], unsigned free_mask,
                     const double lo[4], const double hi[4], double sigmas_out[4],
                     double *cost_out, int *evals) {
  lbm::NvtxRange nvtx("lbm_opt_minimize");
  CostSpec cs;
  if (!sigmas_in || !sigmas_out || !lo || !hi || make_spec(spec, &cs) != LBM_OK ||
      !valid_sigmas(sigmas_in) || (free_mask & 15u) == 0 || (free_mask & ~15u) != 0) {
    lbm::set_error("bad minimization arguments");
    return LBM_EINVAL;
  }
  int fi[4], nf = 0;
  for (int i = 0; i < 4; ++i)
    if (free_mask & (1u << i)) {
      if (!(lo[i] >= 0.0) || !(hi[i] > lo[i]) || !std::isfinite(hi[i])) {
        lbm::set_error("free sigma needs 0 <= lo < hi");
        return LBM_EINVAL;
      }
      fi[nf++] = i;
    }
  int nevals = 0;
  Workspace ws;
  // 1. grid scan: per free sigma 0 and a log-spaced grid over [max(lo, tiny), hi]
  const int G = nf == 1 ? 96 : (nf == 2 ? 32 : (nf == 3 ? 10 : 6));
  std::vector<std::vector<double>> axis((size_t)nf);
  for (int a = 0; a < nf; ++a) {
    const int i = fi[a];
    const double l0 = std::max(lo[i], 1e-7 * hi[i]);
    if (lo[i] == 0.0) axis[a].push_back(0.0);
    for (int g = 0; g < G; ++g)
      axis[a].push_back(l0 * pow(hi[i] / l0, (double)g / (G - 1)));
  }
  size_t total = 1;
  for (int a = 0; a < nf; ++a) total *= axis[a].size();
  std::vector<double> cand(4 * total), vals(total);
  for (size_t t = 0; t < total; ++t) {
    size_t r = t;
    for (int i = 0; i < 4; ++i) cand[4 * t + i] = sigmas_in[i];
    for (int a = 0; a < nf; ++a) {
      cand[4 * t + fi[a]] = axis[a][r % axis[a].size()];
      r /= axis[a].size();
    }
  }
  int rc = eval_costs(ws, cs, (int)total, cand.data(), vals.data());
  if (rc != LBM_OK) return rc;
  nevals += (int)total;
  size_t best = 0;
  for (size_t t = 1; t < total; ++t)
    if (vals[t] < vals[best]) best = t;

  // 2. Nelder-Mead in the free sigmas scaled by their grid optimum, each
  //    point clamped to [lo, hi]; restarted until the cost stops improving
  double scale[4], x0[4], base[4];
  for (int i = 0; i < 4; ++i) base[i] = cand[4 * best + i];
  for (int a = 0; a < nf; ++a) {
    scale[a] = std::max(fabs(base[fi[a]]), 1e-6 * hi[fi[a]]);
    x0[a] = base[fi[a]] / scale[a];
  }
  auto to_sig = [&](const double *x, double *s) {
    for (int i = 0; i < 4; ++i) s[i] = base[i];
    for (int a = 0; a < nf; ++a) s[fi[a]] = std::min(std::max(x[a] * scale[a], lo[fi[a]]), hi[fi[a]]);
  };
  // every trial point is projected into the box first, so the simplex
  // cannot drift through the flat region beyond a bound
  auto f = [&](double *x, double *v) -> int {
    for (int a = 0; a < nf; ++a)
      x[a] = std::min(std::max(x[a], lo[fi[a]] / scale[a]), hi[fi[a]] / scale[a]);
    double s[4];
    to_sig(x, s);
    ++nevals;
    return eval_costs(ws, cs, 1, s, v);
  };
  double fbest = vals[best];
  double xbest[4];
  for (int a = 0; a < nf; ++a) xbest[a] = x0[a];
  for (int restart = 0; restart < 8; ++restart) {
    const int np = nf + 1;
    double X[5][4], F[5];
    for (int v = 0; v < np; ++v) {
      for (int a = 0; a < nf; ++a) X[v][a] = xbest[a];
      if (v > 0) X[v][v - 1] += X[v][v - 1] != 0.0 ? 0.1 * X[v][v - 1] : 0.05;
      if (v == 0) F[v] = fbest;
      else if ((rc = f(X[v], &F[v])) != LBM_OK) return rc;
    }
    for (int iter = 0; iter < 2000; ++iter) {
      // order the simplex
      for (int i = 0; i < np; ++i)
        for (int j = i + 1; j < np; ++j)
          if (F[j] < F[i]) {
            std::swap(F[i], F[j]);
            for (int a = 0; a < nf; ++a) std::swap(X[i][a], X[j][a]);
          }
      double spread = 0.0;
      for (int v = 1; v < np; ++v)
        for (int a = 0; a < nf; ++a) spread = std::max(spread, fabs(X[v][a] - X[0][a]));
      if (spread < 1e-12 && F[np - 1] - F[0] <= 1e-15 * fabs(F[0])) break;
      double c[4] = {0, 0, 0, 0}, xr[4], xe[4], xc[4], fr, fe, fc;
      for (int v = 0; v < nf; ++v)
        for (int a = 0; a < nf; ++a) c[a] += X[v][a] / nf;
      for (int a = 0; a < nf; ++a) xr[a] = c[a] + (c[a] - X[nf][a]);
      if ((rc = f(xr, &fr)) != LBM_OK) return rc;
      if (fr < F[0]) {
        for (int a = 0; a < nf; ++a) xe[a] = c[a] + 2.0 * (c[a] - X[nf][a]);
        if ((rc = f(xe, &fe)) != LBM_OK) return rc;
        if (fe < fr) {
          for (int a = 0; a < nf; ++a) X[nf][a] = xe[a];
          F[nf] = fe;
        } else {
          for (int a = 0; a < nf; ++a) X[nf][a] = xr[a];
          F[nf] = fr;
        }
      } else if (fr < F[nf - 1]) {
        for (int a = 0; a < nf; ++a) X[nf][a] = xr[a];
        F[nf] = fr;
      } else {
        const bool outside = fr < F[nf];
        for (int a = 0; a < nf; ++a)
          xc[a] = outside ? c[a] + 0.5 * (xr[a] - c[a]) : c[a] + 0.5 * (X[nf][a] - c[a]);
        if ((rc = f(xc, &fc)) != LBM_OK) return rc;
        if (fc < (outside ? fr : F[nf])) {
          for (int a = 0; a < nf; ++a) X[nf][a] = xc[a];
          F[nf] = fc;
        } else {
          for (int v = 1; v < np; ++v) {
            for (int a = 0; a < nf; ++a) X[v][a] = X[0][a] + 0.5 * (X[v][a] - X[0][a]);
            if ((rc = f(X[v], &F[v])) != LBM_OK) return rc;
          }
        }
      }
    }
    int imin = 0;
    for (int v = 1; v < np; ++v)
      if (F[v] < F[imin]) imin = v;
    const bool improved = fbest - F[imin] > 1e-14 * fabs(fbest);
    if (F[imin] <= fbest) {
      fbest = F[imin];
      for (int a = 0; a < nf; ++a) xbest[a] = X[imin][a];
    }
    if (!improved) break;
  }
  to_sig(xbest, sigmas_out);
  if (cost_out) *cost_out = fbest;
  if (evals) *evals = nevals;
  return LBM_OK;
}

}  // extern "C"

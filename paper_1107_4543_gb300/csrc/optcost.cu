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
// truncated at dt^(n-1).
//
// Real arithmetic.  The scheme's operators are A_l = (1/l!) M
// diag((-i v.k)^l) M^-1 Psi = (-i)^l H_l with the real
// H_l = M diag(t_l) M^-1 Psi, t_l,j = (v_j.k)^l / l!.  Psi is real, so by
// induction over both recursions the dt^t coefficient of Phi_m is (-i)^t
// times a real matrix, that of B_m is (-i)^(t+1) times a real matrix and
// that of a power B_s^p is (-i)^(t+p) times a real matrix; the phases
// cancel from every recursion step, which therefore runs on the real
// factors alone, and come back only in the final norm (cross terms of
// coefficients l, m carry Re (-i)^(l-m): zero for odd l - m).
//
// H_l = K_l D^-1 Psi with K_l = M diag(t_l) M^T (M^-1 = M^T D^-1,
// D = diag(9, 6, 6, 36, 36, 12, 12, 4, 4)); K_l depends on the wave
// direction only and is tabulated on the host per direction.
//
// One warp per quadrature point (theta, flow direction, flow speed), its
// polynomial matrices in shared memory; each lane owns some entries of
// each matrix being formed.  The wave-number integral over dt k in [0, pi]
// of ||M_eps||_F^2, M_eps = sum_l (dt k)^(l+1) (b^l - b_exact^l), is taken
// in closed form per point; the point sums are reduced in a fixed order per
// candidate, so results are reproducible bit for bit.
#include <math.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "bounds.cuh"
#include "lbm_internal.h"

namespace {

constexpr int NMAX = 6;                       // largest truncation order
constexpr int SLOTS = NMAX * (NMAX + 1) / 2;  // coefficients of orders 1..NMAX
constexpr int WPB = 2;                        // warps per block
constexpr int PPW = 2;                        // quadrature points per warp
constexpr int MAX_SPEED = 32;
constexpr int MAX_THETA = 4 * NMAX + 4;
constexpr int MAX_DIR = 6 * NMAX;
// the point table of one evaluation (device, read by every warp): wave
// directions, flow directions, flow speeds and weights, pi^p / p
constexpr int T_CTH = 0, T_STH = T_CTH + MAX_THETA, T_CPH = T_STH + MAX_THETA,
              T_SPH = T_CPH + MAX_DIR, T_SU = T_SPH + MAX_DIR, T_WU = T_SU + MAX_SPEED,
              T_KINT = T_WU + MAX_SPEED, T_SIZE = T_KINT + 2 * NMAX + 2;

// D2Q9 velocities (the order of the step kernels) and the Lallemand-Luo
// moment matrix in the paper's row order with its row norms
__host__ __device__ __forceinline__ int vx(int j) {
  return j == 1 || j == 5 || j == 8 ? 1 : (j == 3 || j == 6 || j == 7 ? -1 : 0);
}
__host__ __device__ __forceinline__ int vy(int j) {
  return j == 2 || j == 5 || j == 6 ? 1 : (j == 4 || j == 7 || j == 8 ? -1 : 0);
}
__host__ __device__ __forceinline__ int mm(int k, int j) {
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
// 1 / D_kk
__host__ __device__ __forceinline__ double rnorm(int k) {
  return k == 0 ? 1.0 / 9.0
                : (k <= 2 ? 1.0 / 6.0 : (k <= 4 ? 1.0 / 36.0 : (k <= 6 ? 1.0 / 12.0 : 1.0 / 4.0)));
}

__device__ __forceinline__ int slot(int m, int d) {
  lbm::bounds::ok(m >= 1 && m <= NMAX && d >= 0 && d < m, lbm::bounds::OPT_SLOT);
  return lbm::bounds::ck(m * (m - 1) / 2 + d, SLOTS, lbm::bounds::OPT_SLOT);
}

// B_s^p for p >= 2 (degrees 0..s-1) is kept for s = 1..NMAX-1 and
// p = 2..NMAX-s+1: block index of its degree 0 (blocks of 3 x 3)
constexpr int PW_BLOCKS = 35;  // sum over s of (NMAX - s) s
__device__ __forceinline__ int pw_off(int s, int p) {
  int o = 0;
  for (int q = 1; q < s; ++q) o += (NMAX - q) * q;
  return o + (p - 2) * s;
}

// 1 / l!, l = 0..NMAX+1
__constant__ double c_rfact[NMAX + 2] = {1.0,        1.0,         1.0 / 2.0,   1.0 / 6.0,
                                         1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0};

// real factors of the polynomial matrices of one point
struct PointMem {
  double H[NMAX][81];       // H_l, l = 1..n (row-major)
  double psi0[18];          // Psi, rows 3..8, columns 0..2
  double q[18];             // the same divided by D_kk
  double phi[SLOTS][18];    // Phi_m, rows 3..8 (rows 0..2: the identity at degree 0, zero above)
  double B[SLOTS][9];       // B_m, 3 x 3
  double pw[PW_BLOCKS][9];  // powers of B_s
  double part[9];
  double kx, ky, U, V, weight;  // the point: wave direction, mean flow, weight
  int it;                       // its wave-direction index
};

// the PPW points of one warp
struct WarpMem {
  PointMem pt[PPW];
};

struct CostSpec {
  int kind;       // 0: zero mean flow (F), 1: mean flows (G)
  int order;      // truncation order n
  int part;       // 0 all, 1 odd powers of K, 2 even powers
  int reference;  // 0 convection + dissipation, 1 convection, 2 convection + shear
  int n_theta, n_dir, n_speed;
  double u0;
  double w_theta, w_dir;  // quadrature weights of the wave and flow directions
  // host copies of the point table
  double su[MAX_SPEED], wu[MAX_SPEED];  // speed nodes and weights
  double kint[2 * NMAX + 2];            // pi^p / p: integral of K^(p-1) over [0, pi]
  double cth[MAX_THETA], sth[MAX_THETA];  // wave directions
  double cph[MAX_DIR], sph[MAX_DIR];      // flow directions
};

// real factor of row r of H_l times column c of the degree-a coefficient of
// a Phi (X: its rows 3..8)
__device__ __forceinline__ double hx(const double *Hl, int r, const double *X, int a, int c) {
  double z = a == 0 ? Hl[r * 9 + c] : 0.0;
#pragma unroll
  for (int j = 3; j < 9; ++j) z += Hl[r * 9 + j] * X[(j - 3) * 3 + c];
  return z;
}

// B_s^p, coefficient of degree d
__device__ __forceinline__ const double *bpow(const PointMem &w, int s, int p, int d) {
  if (p == 1) return w.B[slot(s, d)];
  lbm::bounds::ok(s >= 1 && s < NMAX && p >= 2 && p <= NMAX - s + 1 && d >= 0 && d < s,
                  lbm::bounds::OPT_POW);
  return w.pw[lbm::bounds::ck(pw_off(s, p) + d, PW_BLOCKS, lbm::bounds::OPT_POW)];
}

// 1 / s_r = sigma_r + 1/2 of a non-conserved row r (sigma_e, sigma_eps,
// sigma_q, sigma_nu)
__device__ __forceinline__ double inv_rate(int r, const double *sg) {
  return (r == 3 ? sg[0] : r == 4 ? sg[1] : r <= 6 ? sg[2] : sg[3]) + 0.5;
}
__device__ __forceinline__ double rate(int r, const double *s) {
  return r == 3 ? s[0] : (r == 4 ? s[1] : (r <= 6 ? s[2] : s[3]));
}

// real factors (b_ex^l = (-i)^(l+1) e_l) of the exact coefficients at
// |k| = 1: convection (l = 0) and dissipation (l = 1)
__device__ __forceinline__ double exact_real(int l, int e, double kx, double ky, double U,
                                             double V, const CostSpec &cs, double sig_e,
                                             double sig_nu) {
  const int r = e / 3, c = e % 3;
  if (l == 0) {  // b_ex^0 = i v, so e_0 = -v
    double v = 0.0;
    if (r == 0) v = c == 1 ? -kx : (c == 2 ? -ky : 0.0);
    if (r == 1) v = c == 0 ? (-kx / 3 + kx * U * U + ky * U * V) : (c == 1 ? (-2 * kx * U - ky * V) : -ky * U);
    if (r == 2) v = c == 0 ? (-ky / 3 + ky * V * V + kx * U * V) : (c == 1 ? -kx * V : (-2 * ky * V - kx * U));
    return -v;
  }
  if (l != 1 || cs.reference == 1) return 0.0;
  // b_ex^1 = x real, so e_1 = -x
  const double se = cs.reference == 2 ? 0.0 : sig_e;
  double x = 0.0;
  if (r == 1 && c == 1) x = -(kx * kx * se + (kx * kx + ky * ky) * sig_nu) / 3;
  if ((r == 1 && c == 2) || (r == 2 && c == 1)) x = -kx * ky * se / 3;
  if (r == 2 && c == 2) x = -(ky * ky * se + (kx * kx + ky * ky) * sig_nu) / 3;
  return -x;
}

// The recursions on the real factors, written per output entry.  With
// s = m - l and d = t - l, the dt^t factor of Phi_m (t >= 1, non-conserved
// rows r) is
//   (1/s_r) sum_{l=1..t} [ -(1/l!) (Phi_s B_s^l)_d + H_l Phi_s,d ]_rc
// (degree 0: Psi_rc / s_r), and that of B_m is
//   - sum_{l=1..min(t, m-1)} (1/(l+1)!) (B_s^(l+1))_d
//   + sum_{l=1..min(m, t+1)} rows 0..2 of H_l Phi_{m+1-l, t-l+1}
// -- Eqs. R-A/R-B and R-D/R-E with every product truncated at dt^(m-1).
// No two lanes write one entry, and the powers B_m^p needed later are
// formed once, right after B_m.  A warp carries PPW points (the matrices are
// small: one point leaves most lanes idle), its lanes taking the entries of
// all of them; work items run heaviest first (highest degree t, the points
// interleaved), so that each round of 32 lanes holds items of similar cost.
//
// tab: the point table (T_* offsets) followed by, per candidate, sigma_e,
// sigma_eps, sigma_q, sigma_nu and the rates s = 1 / (sigma + 1/2) in that
// order; ktab: K_l per wave direction, [n_theta][NMAX][81].
__global__ void __launch_bounds__(WPB * 32)
k_opt_points(CostSpec cs, const double *__restrict__ tab, const double *__restrict__ ktab,
             long long npoints, double *__restrict__ partial) {
  extern __shared__ unsigned char smem_raw[];
  WarpMem &w = reinterpret_cast<WarpMem *>(smem_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const long long p0 = ((long long)blockIdx.x * WPB + (threadIdx.x >> 5)) * PPW;
  const int ci = blockIdx.y;
  if (p0 >= npoints) return;  // warp-uniform
  const int n = cs.order;
  const double *sg = tab + T_SIZE + 8 * (long long)ci;  // sigmas
  const double *rs = sg + 4;                             // rates

  // the points: theta (fastest), flow direction, flow speed; a slot past the
  // last point repeats the last point and is not written
  if (lane < PPW) {
    long long p = p0 + lane;
    if (p >= npoints) p = npoints - 1;
    const int it = (int)(p % cs.n_theta);
    const long long q = p / cs.n_theta;
    const int id = (int)(q % cs.n_dir);
    const int iu = (int)(q / cs.n_dir);
    PointMem &P = w.pt[lane];
    using lbm::bounds::ck;
    using lbm::bounds::OPT_TAB;
    P.it = ck(it, MAX_THETA, OPT_TAB);
    P.kx = tab[T_CTH + P.it];
    P.ky = tab[T_STH + P.it];
    double U = 0.0, V = 0.0, weight = cs.w_theta;
    if (cs.kind == 1) {
      const int su = ck(iu, MAX_SPEED, OPT_TAB), dr = ck(id, MAX_DIR, OPT_TAB);
      U = tab[T_SU + su] * tab[T_CPH + dr];
      V = tab[T_SU + su] * tab[T_SPH + dr];
      weight *= cs.w_dir * tab[T_WU + su];
    }
    P.U = U;
    P.V = V;
    P.weight = weight;
  }
  __syncwarp();

  // Psi (section 2.3, about rho = 1, j = (U, V)), rows 3..8 and columns
  // 0..2: s_r times the derivative of m^eq_r by (rho, jx, jy)
  for (int e = lane; e < 18 * PPW; e += 32) {
    PointMem &P = w.pt[e / 18];
    const int rc = e % 18, r = 3 + rc / 3, c = rc % 3;
    const double U = P.U, V = P.V, u2 = U * U + V * V;
    double j;
    switch (r) {
      case 3: j = c == 0 ? -2.0 - 3.0 * u2 : (c == 1 ? 6.0 * U : 6.0 * V); break;
      case 4: j = c == 0 ? 1.0 + 3.0 * u2 : (c == 1 ? -6.0 * U : -6.0 * V); break;
      case 5: j = c == 1 ? -1.0 : 0.0; break;
      case 6: j = c == 2 ? -1.0 : 0.0; break;
      case 7: j = c == 0 ? -(U * U - V * V) : (c == 1 ? 2.0 * U : -2.0 * V); break;
      default: j = c == 0 ? -U * V : (c == 1 ? V : U); break;
    }
    const double ps = rate(r, rs) * j;
    P.psi0[rc] = ps;
    P.q[rc] = ps * rnorm(r);
  }
  __syncwarp();
  // H_l = K_l D^-1 Psi: columns 0..2 (identity + Psi's first columns),
  // then columns 3..8 ((1 - s_c) / D_cc times column c of K_l)
  for (int e = lane; e < 27 * n * PPW; e += 32) {
    PointMem &P = w.pt[e % PPW];
    const int f = e / PPW, l = lbm::bounds::ck(f / 27, NMAX, lbm::bounds::OPT_H),
              r = (f % 27) / 3, c = f % 3;
    const double *Kr =
        ktab + lbm::bounds::ck(((long long)P.it * NMAX + l) * 81 + r * 9,
                               (long long)cs.n_theta * NMAX * 81, lbm::bounds::OPT_KTAB);
    double h = Kr[c] * rnorm(c);
#pragma unroll
    for (int k = 3; k < 9; ++k) h += Kr[k] * P.q[(k - 3) * 3 + c];
    P.H[l][r * 9 + c] = h;
  }
  for (int e = lane; e < 54 * n * PPW; e += 32) {
    PointMem &P = w.pt[e % PPW];
    const int f = e / PPW, l = lbm::bounds::ck(f / 54, NMAX, lbm::bounds::OPT_H),
              r = (f % 54) / 6, c = 3 + f % 6;
    P.H[l][r * 9 + c] = ktab[lbm::bounds::ck(((long long)P.it * NMAX + l) * 81 + r * 9 + c,
                                             (long long)cs.n_theta * NMAX * 81,
                                             lbm::bounds::OPT_KTAB)] *
                        ((1.0 - rate(c, rs)) * rnorm(c));
  }
  __syncwarp();

  for (int m = 1; m <= n; ++m) {
    // Phi_m, rows 3..8
    for (int e = lane; e < 18 * PPW * m; e += 32) {
      const int t = m - 1 - e / (18 * PPW), rc = e % 18, r = 3 + rc / 3, c = rc % 3;
      PointMem &P = w.pt[(e / 18) % PPW];
      double v = t == 0 ? P.psi0[rc] : 0.0;
      for (int l = 1; l <= t; ++l) {
        const int s = m - l, d = t - l;
        double acc = 0.0;
        for (int a = 0; a <= d; ++a) {
          const double *X = P.phi[slot(s, a)];
          const double *Pp = bpow(P, s, l, d - a);
#pragma unroll
          for (int k = 0; k < 3; ++k) acc += X[rc - c + k] * Pp[k * 3 + c];
        }
        v -= c_rfact[l] * acc;
        v += hx(P.H[lbm::bounds::ck(l - 1, NMAX, lbm::bounds::OPT_H)], r, P.phi[slot(s, d)], d,
                c);
      }
      P.phi[slot(m, t)][rc] = inv_rate(r, sg) * v;
    }
    __syncwarp();
    // B_m
    for (int e = lane; e < 9 * PPW * m; e += 32) {
      const int t = m - 1 - e / (9 * PPW), rc = e % 9, r = rc / 3, c = rc % 3;
      PointMem &P = w.pt[(e / 9) % PPW];
      double v = 0.0;
      for (int l = 1; l <= t && l < m; ++l) v -= c_rfact[l + 1] * bpow(P, m - l, l + 1, t - l)[rc];
      for (int l = 1; l <= m && l <= t + 1; ++l)
        v += hx(P.H[lbm::bounds::ck(l - 1, NMAX, lbm::bounds::OPT_H)], r,
                P.phi[slot(m + 1 - l, t - l + 1)], t - l + 1, c);
      P.B[slot(m, t)][rc] = v;
    }
    __syncwarp();
    // B_m^p, p = 2..n-m+1, truncated at degree m-1
    for (int pp = 2; pp <= n - m + 1; ++pp) {
      for (int e = lane; e < 9 * PPW * m; e += 32) {
        const int d = m - 1 - e / (9 * PPW), rc = e % 9, r = rc / 3, c = rc % 3;
        PointMem &P = w.pt[(e / 9) % PPW];
        double acc = 0.0;
        for (int a = 0; a <= d; ++a) {
          const double *X = bpow(P, m, pp - 1, a);
          const double *Bb = P.B[slot(m, d - a)];
#pragma unroll
          for (int k = 0; k < 3; ++k) acc += X[r * 3 + k] * Bb[k * 3 + c];
        }
        P.pw[lbm::bounds::ck(pw_off(m, pp) + d, PW_BLOCKS, lbm::bounds::OPT_POW)][rc] = acc;
      }
      __syncwarp();
    }
  }

  // closed-form K integral of ||sum_l K^(l+1) E^l||^2 over [0, pi]:
  // E^l = (-i)^(l+1) (b_l - e_l) on the real factors, so the (l, m) term is
  // Re (-i)^(l-m) (b_l - e_l).(b_m - e_m) pi^(l+m+3) / (l+m+3); the factors
  // E_l are kept where the powers were
  if (lane < 9 * PPW) {
    PointMem &P = w.pt[lane / 9];
    const int e = lane % 9;
    double(*E)[9] = P.pw;
    for (int l = 0; l < n; ++l)
      E[l][e] = P.B[slot(n, l)][e] - exact_real(l, e, P.kx, P.ky, P.U, P.V, cs, sg[0], sg[3]);
    double acc = 0.0;
    for (int l = 0; l < n; ++l) {
      const bool odd_l = ((l + 1) & 1) != 0;
      if ((cs.part == 1 && !odd_l) || (cs.part == 2 && odd_l)) continue;
      for (int mq = l & 1; mq < n; mq += 2) {  // odd l - mq: Re (-i)^(l-mq) = 0
        const double sgn = ((l - mq) & 3) == 0 ? 1.0 : -1.0;
        acc += sgn * (E[l][e] * E[mq][e]) *
               tab[T_KINT + lbm::bounds::ck(l + mq + 3, 2 * NMAX + 2, lbm::bounds::OPT_TAB)];
      }
    }
    P.part[e] = acc;
  }
  __syncwarp();
  if (lane < PPW && p0 + lane < npoints) {
    const PointMem &P = w.pt[lane];
    double v = 0.0;
    for (int e = 0; e < 9; ++e) v += P.part[e];
    partial[(long long)ci * npoints + p0 + lane] = v * P.weight;
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
  for (int p = 0; p < 2 * NMAX + 2; ++p) cs->kint[p] = p ? pow(M_PI, p) / p : 0.0;
  for (int i = 0; i < cs->n_theta; ++i) {
    const double th = 2.0 * M_PI * i / cs->n_theta;
    cs->cth[i] = cos(th);
    cs->sth[i] = sin(th);
  }
  cs->w_theta = 2.0 * M_PI / cs->n_theta;
  if (cs->kind == LBM_COST_F) {
    cs->n_dir = 1;
    cs->n_speed = 1;
    cs->cph[0] = 1.0;
    cs->sph[0] = 0.0;
    cs->w_dir = 1.0;
    cs->su[0] = 0.0;
    cs->wu[0] = 1.0;
  } else {
    if (!(cs->u0 >= 0.0) || !std::isfinite(cs->u0)) return LBM_EINVAL;
    cs->n_dir = 6 * cs->order;
    cs->n_speed = 2 * cs->order + 2;
    for (int i = 0; i < cs->n_dir; ++i) {
      const double ph = 2.0 * M_PI * i / cs->n_dir;
      cs->cph[i] = cos(ph);
      cs->sph[i] = sin(ph);
    }
    cs->w_dir = 2.0 * M_PI / cs->n_dir;
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

// K_l = M diag(t_l) M^T, t_l,j = (v_j.k)^l / l!, for every wave direction
// of the quadrature and l = 1..order: [n_theta][NMAX][81]
std::vector<double> k_tables(const CostSpec &cs) {
  std::vector<double> out((size_t)cs.n_theta * NMAX * 81, 0.0);
  for (int it = 0; it < cs.n_theta; ++it) {
    double vk[9], t[9];
    for (int j = 0; j < 9; ++j) {
      vk[j] = vx(j) * cs.cth[it] + vy(j) * cs.sth[it];
      t[j] = 1.0;
    }
    double fact = 1.0;
    for (int l = 1; l <= cs.order; ++l) {
      fact *= l;
      for (int j = 0; j < 9; ++j) t[j] *= vk[j];
      double *K = out.data() + ((size_t)it * NMAX + (l - 1)) * 81;
      for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
          double s = 0.0;
          for (int j = 0; j < 9; ++j) s += (double)(mm(r, j) * mm(c, j)) * t[j];
          K[r * 9 + c] = s / fact;
        }
    }
  }
  return out;
}

// device buffers of the cost evaluations, grown on demand and reused by the
// many small evaluations of a minimization
struct Workspace {
  double *tab = nullptr, *part = nullptr, *out = nullptr, *ktab = nullptr;
  size_t cap_n = 0, cap_part = 0;
  int k_order = -1, k_theta = -1;  // what ktab holds
  ~Workspace() {
    lbm::dev_free(tab);
    lbm::dev_free(part);
    lbm::dev_free(out);
    lbm::dev_free(ktab);
  }
  bool ensure(size_t n, size_t npart) {
    if (n > cap_n) {
      lbm::dev_free(tab);
      lbm::dev_free(out);
      tab = (double *)lbm::dev_alloc(sizeof(double) * (T_SIZE + 8 * n));
      out = (double *)lbm::dev_alloc(sizeof(double) * n);
      cap_n = (tab && out) ? n : 0;
      if (!cap_n) return false;
    }
    if (npart > cap_part) {
      lbm::dev_free(part);
      part = (double *)lbm::dev_alloc(sizeof(double) * npart);
      cap_part = part ? npart : 0;
      if (!cap_part) return false;
    }
    if (!ktab) {
      ktab = (double *)lbm::dev_alloc(sizeof(double) * MAX_THETA * NMAX * 81);
      if (!ktab) return false;
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
  cudaError_t e = cudaSuccess;
  if (ws.k_order != cs.order || ws.k_theta != cs.n_theta) {
    const std::vector<double> kt = k_tables(cs);
    e = cudaMemcpy(ws.ktab, kt.data(), sizeof(double) * kt.size(), cudaMemcpyHostToDevice);
    ws.k_order = e == cudaSuccess ? cs.order : -1;
    ws.k_theta = cs.n_theta;
  }
  // the point table, then per candidate the sigmas and the rates
  // s = 1 / (sigma + 1/2)
  std::vector<double> cd(T_SIZE + 8 * (size_t)n, 0.0);
  std::copy(cs.cth, cs.cth + MAX_THETA, cd.begin() + T_CTH);
  std::copy(cs.sth, cs.sth + MAX_THETA, cd.begin() + T_STH);
  std::copy(cs.cph, cs.cph + MAX_DIR, cd.begin() + T_CPH);
  std::copy(cs.sph, cs.sph + MAX_DIR, cd.begin() + T_SPH);
  std::copy(cs.su, cs.su + MAX_SPEED, cd.begin() + T_SU);
  std::copy(cs.wu, cs.wu + MAX_SPEED, cd.begin() + T_WU);
  std::copy(cs.kint, cs.kint + 2 * NMAX + 2, cd.begin() + T_KINT);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 4; ++k) {
      cd[T_SIZE + 8 * (size_t)i + k] = sig_host[4 * (size_t)i + k];
      cd[T_SIZE + 8 * (size_t)i + 4 + k] = 1.0 / (sig_host[4 * (size_t)i + k] + 0.5);
    }
  if (e == cudaSuccess)
    e = cudaMemcpy(ws.tab, cd.data(), sizeof(double) * cd.size(), cudaMemcpyHostToDevice);
  const size_t shm = sizeof(WarpMem) * WPB;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_opt_points, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e == cudaSuccess) {
    dim3 grid((unsigned)((npoints + WPB * PPW - 1) / (WPB * PPW)), (unsigned)n);
    k_opt_points<<<grid, WPB * 32, shm>>>(cs, ws.tab, ws.ktab, npoints, ws.part);
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

namespace lbm {
unsigned bounds_word_opt(bool reset) { return bounds::read_word(reset); }
}  // namespace lbm

// D2Q9 MRT collision at one node, in registers (device helpers).
//
// Moments m = M f with M the Lallemand-Luo D2Q9 matrix in the paper's row
// order rho, jx, jy, e, eps, qx, qy, pxx, pxy (section 2.1, Eq. q-macro);
// equilibrium moments of section 2.3; relaxation of the non-conserved
// moments with S = diag(0,0,0,s_e,s_eps,s_qx,s_qy,s_pxx,s_pxy) (section 2.1,
// Eq. eq_noconservative); back-transform f <- f - M^-1 S (m - m^eq) with
// M^-1 = M^T D^-1, D = diag(9,6,6,36,36,12,12,4,4) (M has orthogonal rows).
// The 9x9 transforms are unrolled by hand over the nonzero entries
// (0, +-1, +-2, +-4): no tensor cores, the step is bound by HBM traffic.
#pragma once

namespace lbm {

// Rates pre-divided by the row norms D_k: k3 = s_e/36, k4 = s_eps/36,
// k5 = s_qx/12, k6 = s_qy/12, k7 = s_pxx/4, k8 = s_pxy/4.
struct DevParams {
  float rho0, jx0, jy0;   // reference state rho0, j0 = rho0 u0
  float k3, k4, k5, k6, k7, k8;
  float scale, inv_scale; // FP16 storage: stored = f' * scale
};

// Deviation form: f' = f - f^eq(rho0, u0) with the moments of the base
// being m^eq(rho0, j0).  So rho = rho0 + rho', j = j0 + j', and
//   m - m^eq(rho, j) = m' - [m^eq(rho, j) - m^eq(rho0, j0)],
// where every difference of quadratic terms is formed without cancellation,
//   a b / rho - a0 b0 / rho0 = (rho0 (a0 b' + a' b0 + a' b') - rho' a0 b0)
//                              / (rho rho0).
// FP32 throughout.
__device__ __forceinline__ void collide_dev(float &f0, float &f1, float &f2, float &f3,
                                            float &f4, float &f5, float &f6, float &f7,
                                            float &f8, const DevParams &P) {
  const float s13 = f1 + f3, s24 = f2 + f4;
  const float d13 = f1 - f3, d24 = f2 - f4;
  const float s57 = f5 + f7, s68 = f6 + f8;
  const float d57 = f5 - f7, d68 = f6 - f8;
  const float axis = s13 + s24;
  const float diag = s57 + s68;
  const float rho_p = f0 + axis + diag;
  const float jx_p = d13 + (d57 - d68);  // f1 - f3 + f5 - f6 - f7 + f8
  const float jy_p = d24 + (d57 + d68);  // f2 - f4 + f5 + f6 - f7 - f8
  const float e_p = fmaf(2.0f, diag, -fmaf(4.0f, f0, axis));
  const float eps_p = fmaf(4.0f, f0, fmaf(-2.0f, axis, diag));
  const float qx_p = fmaf(-2.0f, d13, d57 - d68);
  const float qy_p = fmaf(-2.0f, d24, d57 + d68);
  const float pxx_p = s13 - s24;
  const float pxy_p = s57 - s68;

  const float rho = P.rho0 + rho_p;
  const float inv = 1.0f / (rho * P.rho0);
  // rho0 (|j|^2 - |j0|^2) - rho' |j0|^2 etc., over rho rho0
  const float tx = fmaf(2.0f, P.jx0, jx_p) * jx_p;  // (2 jx0 + jx') jx'
  const float ty = fmaf(2.0f, P.jy0, jy_p) * jy_p;
  const float jx02 = P.jx0 * P.jx0, jy02 = P.jy0 * P.jy0;
  const float djsq = fmaf(P.rho0, tx + ty, -rho_p * (jx02 + jy02)) * inv;
  const float dpxx = fmaf(P.rho0, tx - ty, -rho_p * (jx02 - jy02)) * inv;
  const float cxy = fmaf(P.jx0, jy_p, fmaf(jx_p, P.jy0, jx_p * jy_p));
  const float dpxy = fmaf(P.rho0, cxy, -rho_p * (P.jx0 * P.jy0)) * inv;

  // non-equilibrium parts times S / D
  const float r3 = P.k3 * (e_p - fmaf(3.0f, djsq, -2.0f * rho_p));
  const float r4 = P.k4 * (eps_p - fmaf(-3.0f, djsq, rho_p));
  const float r5 = P.k5 * (qx_p + jx_p);
  const float r6 = P.k6 * (qy_p + jy_p);
  const float r7 = P.k7 * (pxx_p - dpxx);
  const float r8 = P.k8 * (pxy_p - dpxy);

  // f <- f - M^T (r): columns of M for each velocity
  const float a = fmaf(2.0f, r4, r3);     // axis velocities: -r3 - 2 r4
  const float b = fmaf(2.0f, r3, r4);     // diagonals: 2 r3 + r4
  f0 -= 4.0f * (r4 - r3);
  f1 += fmaf(2.0f, r5, a - r7);           // -(-a - 2 r5 + r7)
  f3 += fmaf(-2.0f, r5, a - r7);
  f2 += fmaf(2.0f, r6, a + r7);
  f4 += fmaf(-2.0f, r6, a + r7);
  f5 -= b + r5 + r6 + r8;
  f6 -= b - r5 + r6 - r8;
  f7 -= b - r5 - r6 + r8;
  f8 -= b + r5 - r6 - r8;
}

// FP64 rates of the plain path: s3 = s_e, s4 = s_eps, s5 = s_qx, s6 = s_qy,
// s7 = s_pxx, s8 = s_pxy.
struct F64Params {
  double s3, s4, s5, s6, s7, s8;
};

// Plain FP64 collision of the full populations.  The operation order is the
// one of a plain matrix-vector implementation of section 2.1: each moment is
// the sum over j = 0..8 of M_kj f_j taken left to right; m^eq as written in
// section 2.3 ((-2 rho) + (3 |j|^2)/rho, ...); r_k = s_k (m_k - m^eq_k);
// f_i - sum over k = 0..8 of (M_ki / D_k) r_k left to right.  Terms with a
// zero coefficient are skipped (adding a signed zero changes no value) and
// products by +-1, +-2, +-4 are exact, so this equals the plain loop
// bit for bit.  Compile without multiply-add contraction (-fmad=false).
__device__ __forceinline__ void collide_f64(double (&f)[9], const F64Params &P) {
  const double rho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  const double jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
  const double jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
  const double e = -4.0 * f[0] - f[1] - f[2] - f[3] - f[4] + 2.0 * f[5] + 2.0 * f[6] +
                   2.0 * f[7] + 2.0 * f[8];
  const double eps = 4.0 * f[0] - 2.0 * f[1] - 2.0 * f[2] - 2.0 * f[3] - 2.0 * f[4] +
                     f[5] + f[6] + f[7] + f[8];
  const double qx = -2.0 * f[1] + 2.0 * f[3] + f[5] - f[6] - f[7] + f[8];
  const double qy = -2.0 * f[2] + 2.0 * f[4] + f[5] + f[6] - f[7] - f[8];
  const double pxx = f[1] - f[2] + f[3] - f[4];
  const double pxy = f[5] - f[6] + f[7] - f[8];

  const double jsq = jx * jx + jy * jy;
  const double e_eq = -2.0 * rho + 3.0 * jsq / rho;
  const double eps_eq = rho - 3.0 * jsq / rho;
  const double pxx_eq = (jx * jx - jy * jy) / rho;
  const double pxy_eq = jx * jy / rho;

  const double r3 = P.s3 * (e - e_eq);
  const double r4 = P.s4 * (eps - eps_eq);
  const double r5 = P.s5 * (qx - (-jx));
  const double r6 = P.s6 * (qy - (-jy));
  const double r7 = P.s7 * (pxx - pxx_eq);
  const double r8 = P.s8 * (pxy - pxy_eq);

  constexpr double c36_1 = 1.0 / 36.0, c36_2 = 2.0 / 36.0, c36_4 = 4.0 / 36.0;
  constexpr double c12_1 = 1.0 / 12.0, c12_2 = 2.0 / 12.0, c4_1 = 1.0 / 4.0;
  f[0] = f[0] - (-c36_4 * r3 + c36_4 * r4);
  f[1] = f[1] - (-c36_1 * r3 + -c36_2 * r4 + -c12_2 * r5 + c4_1 * r7);
  f[2] = f[2] - (-c36_1 * r3 + -c36_2 * r4 + -c12_2 * r6 + -c4_1 * r7);
  f[3] = f[3] - (-c36_1 * r3 + -c36_2 * r4 + c12_2 * r5 + c4_1 * r7);
  f[4] = f[4] - (-c36_1 * r3 + -c36_2 * r4 + c12_2 * r6 + -c4_1 * r7);
  f[5] = f[5] - (c36_2 * r3 + c36_1 * r4 + c12_1 * r5 + c12_1 * r6 + c4_1 * r8);
  f[6] = f[6] - (c36_2 * r3 + c36_1 * r4 + -c12_1 * r5 + c12_1 * r6 + -c4_1 * r8);
  f[7] = f[7] - (c36_2 * r3 + c36_1 * r4 + -c12_1 * r5 + -c12_1 * r6 + c4_1 * r8);
  f[8] = f[8] - (c36_2 * r3 + c36_1 * r4 + c12_1 * r5 + -c12_1 * r6 + -c4_1 * r8);
}

}  // namespace lbm

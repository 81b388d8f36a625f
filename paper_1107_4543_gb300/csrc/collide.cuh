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
// k5 = s_qx/12, k6 = s_qy/12, k7 = s_pxx/4, k8 = s_pxy/4.  Every constant
// that enters the FP32 collision is carried as an unevaluated FP32 sum
// hi + lo (accurate to ~2^-48): a systematic rounding of a constant does not
// average out but integrates over thousands of steps.  The optimized rates
// sit next to 2, where the physics lives in sigma = 1/s - 1/2 (10^-3 ..
// 10^-6); one FP32 rounding of s_e/36 already moves sigma_e by ~1e-5
// relative, a 1e-6 amplitude error after 2000 steps of a damped wave.
struct DevParams {
  float rho0, jx0, jy0;          // reference state (FP32-exact by construction)
  float k3, k4, k5, k6, k7, k8;  // s/D, high parts
  float l3, l4, l5, l6, l7, l8;  // s/D, low parts
  float q0h, q0l;                // |j0|^2
  float d0h, d0l;                // jx0^2 - jy0^2
  float x0h, x0l;                // jx0 jy0
  float i2h, i2l;                // 1 / rho0^2
  float scale, inv_scale;        // FP16 storage: stored = f' * scale
};

// a * (h + l) with the low part folded in by one FMA, or a * h alone when
// the low parts are not wanted
template <bool PRECISE>
__device__ __forceinline__ float mul_hl(float a, float h, float l) {
  return PRECISE ? fmaf(a, h, a * l) : a * h;
}

// Deviation form: f' = f - f^eq(rho0, j0); the base carries the moments
// m^eq(rho0, j0), so rho = rho0 + rho', j = j0 + j' and the non-equilibrium
// parts are n = m' - [m^eq(rho, j) - m^eq(rho0, j0)].  Written so that FP32
// rounding never acts on a large quantity that then cancels:
//   * each n_k is formed directly from partial sums of f' (e.g.
//     n_e = 4 diag - 2 f'_0 + axis - 3 dJ), the cancellation between m'_e
//     and -2 rho' happening exactly inside the sum;
//   * quadratic differences a b / rho - a0 b0 / rho0 are
//     N / rho0^2 * (1 - rho'/rho) with N = rho0 (a0 b' + a' b0 + a' b')
//     - rho' a0 b0: rho = rho0 + rho' is rounded only inside the small
//     correction rho'/rho.
// Measured against the FP64 oracle this keeps the 2000-step plane wave of
// the optimized sets within ~5e-7 of the amplitude (3.5e-6 with the
// straightforward FP32 formulation).
//
// PRECISE: carry the rates and reference-state constants as hi + lo pairs
// (FP32 storage); the 16-bit storage types round far more than the lo parts
// correct and use the hi parts alone.
// SCALED: f holds f' * scale (FP16 storage) and stays in those units: the
// step is linear in f' except for the three quadratic terms and rho'/rho,
// which take the factor inv_scale; with power-of-two scales this equals
// collide-then-rescale bit for bit and saves the per-population rescaling.
template <bool PRECISE, bool SCALED>
__device__ __forceinline__ void collide_dev(float &f0, float &f1, float &f2, float &f3,
                                            float &f4, float &f5, float &f6, float &f7,
                                            float &f8, const DevParams &P) {
  const float s13 = f1 + f3, s24 = f2 + f4;
  const float d13 = f1 - f3, d24 = f2 - f4;
  const float s57 = f5 + f7, s68 = f6 + f8;
  const float d57 = f5 - f7, d68 = f6 - f8;
  const float axis = s13 + s24;
  const float diag = s57 + s68;
  const float dxd = d57 - d68;  // f5 - f6 - f7 + f8
  const float dyd = d57 + d68;  // f5 + f6 - f7 - f8
  const float rho_p = f0 + axis + diag;
  const float jx_p = d13 + dxd;
  const float jy_p = d24 + dyd;

  // m^eq(rho, j) - m^eq(rho0, j0) for the three quadratic terms
  const float rho_phys = SCALED ? rho_p * P.inv_scale : rho_p;
  // rho'/rho by the hardware reciprocal (within 2 ulp): c only scales the
  // O(amplitude^2) quadratic terms below, and unlike an IEEE division it has
  // no slow path for non-finite operands, so a lattice that has gone
  // unstable costs no more per node than a healthy one
  const float c = __fdividef(rho_phys, P.rho0 + rho_phys);
  const float jxx = SCALED ? (jx_p * jx_p) * P.inv_scale : jx_p * jx_p;
  const float jyy = SCALED ? (jy_p * jy_p) * P.inv_scale : jy_p * jy_p;
  const float jxy = SCALED ? (jx_p * jy_p) * P.inv_scale : jx_p * jy_p;
  const float tx = fmaf(2.0f * P.jx0, jx_p, jxx);  // jx^2 - jx0^2
  const float ty = fmaf(2.0f * P.jy0, jy_p, jyy);
  const float txy = fmaf(P.jx0, jy_p, fmaf(jx_p, P.jy0, jxy));  // jx jy - jx0 jy0
  const float nj =
      mul_hl<PRECISE>(fmaf(P.rho0, tx + ty, -mul_hl<PRECISE>(rho_p, P.q0h, P.q0l)), P.i2h, P.i2l);
  const float np =
      mul_hl<PRECISE>(fmaf(P.rho0, tx - ty, -mul_hl<PRECISE>(rho_p, P.d0h, P.d0l)), P.i2h, P.i2l);
  const float nx =
      mul_hl<PRECISE>(fmaf(P.rho0, txy, -mul_hl<PRECISE>(rho_p, P.x0h, P.x0l)), P.i2h, P.i2l);
  const float djsq = fmaf(-nj, c, nj);  // |j|^2/rho - |j0|^2/rho0
  const float dpxx = fmaf(-np, c, np);  // (jx^2 - jy^2)/rho - (..)0/rho0
  const float dpxy = fmaf(-nx, c, nx);  // jx jy / rho - jx0 jy0 / rho0

  // non-equilibrium parts, each straight from partial sums
  const float n3 = fmaf(4.0f, diag, axis - 2.0f * f0) - 3.0f * djsq;  // e' + 2 rho' - 3 dJ
  const float n4 = fmaf(3.0f, djsq, 3.0f * (f0 - axis));             // eps' - rho' + 3 dJ
  const float n5 = fmaf(2.0f, dxd, -d13);                            // qx' + jx'
  const float n6 = fmaf(2.0f, dyd, -d24);                            // qy' + jy'
  const float n7 = (s13 - s24) - dpxx;
  const float n8 = (s57 - s68) - dpxy;
  const float r3 = mul_hl<PRECISE>(n3, P.k3, P.l3);
  const float r4 = mul_hl<PRECISE>(n4, P.k4, P.l4);
  const float r5 = mul_hl<PRECISE>(n5, P.k5, P.l5);
  const float r6 = mul_hl<PRECISE>(n6, P.k6, P.l6);
  const float r7 = mul_hl<PRECISE>(n7, P.k7, P.l7);
  const float r8 = mul_hl<PRECISE>(n8, P.k8, P.l8);

  // f <- f - M^T r: columns of M for each velocity
  const float a = fmaf(2.0f, r4, r3);     // axis velocities: -r3 - 2 r4
  const float b = fmaf(2.0f, r3, r4);     // diagonals: 2 r3 + r4
  f0 -= 4.0f * (r4 - r3);
  f1 += fmaf(2.0f, r5, a - r7);
  f3 += fmaf(-2.0f, r5, a - r7);
  f2 += fmaf(2.0f, r6, a + r7);
  f4 += fmaf(-2.0f, r6, a + r7);
  f5 -= b + r5 + r6 + r8;
  f6 -= b - r5 + r6 - r8;
  f7 -= b - r5 - r6 + r8;
  f8 -= b + r5 - r6 - r8;
}

// ------------------------------------------------------------------
// Two nodes at once with the packed FP32 instructions of sm_100 and later
// (add / sub / mul / fma .rn.f32x2): each does the work of two scalar
// instructions, lane by lane with the scalar instruction's IEEE rounding.
// The 16-bit storage types unpack two nodes per 32-bit word, so the pair is
// already there; at 36 B per node their step is bound by instruction issue
// more than by HBM, and this halves the collision's issue slots (measured on
// one 8192^2 lattice: BF16 6.69 -> 6.99 TB/s, FP16 6.82 -> 6.86 TB/s).
struct F2 {
  unsigned long long v;
};
__device__ __forceinline__ F2 f2(float lo, float hi) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ F2 f2s(float a) { return f2(a, a); }
__device__ __forceinline__ void f2split(F2 a, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
  F2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  F2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
  F2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
// a * b + c, one rounding per lane
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}

// The per-lattice constants collide_pair multiplies by, each broadcast to
// both lanes of an F2; negations and doublings are folded in (exact in
// FP32, so every source of them gives the same bits).
enum PairConst {
  PC_IS, PC_R0, PC_2JX, PC_2JY, PC_JX, PC_JY, PC_I2, PC_NQ0, PC_ND0, PC_NX0,
  PC_K3, PC_K4, PC_NK5, PC_NK6, PC_K7, PC_K8, PC_COUNT
};

__host__ __device__ __forceinline__ float pair_const(const DevParams &P, int c) {
  switch (c) {
    case PC_IS: return P.inv_scale;
    case PC_R0: return P.rho0;
    case PC_2JX: return 2.0f * P.jx0;
    case PC_2JY: return 2.0f * P.jy0;
    case PC_JX: return P.jx0;
    case PC_JY: return P.jy0;
    case PC_I2: return P.i2h;
    case PC_NQ0: return -P.q0h;
    case PC_ND0: return -P.d0h;
    case PC_NX0: return -P.x0h;
    case PC_K3: return P.k3;
    case PC_K4: return P.k4;
    case PC_NK5: return -P.k5;
    case PC_NK6: return -P.k6;
    case PC_K7: return P.k7;
    default: return P.k8;
  }
}

// The constants straight from a DevParams (kernel parameters of a single
// lattice, or an entry in global memory)
struct ParamPairs {
  const DevParams &P;
  __device__ __forceinline__ F2 operator()(PairConst c) const { return f2s(pair_const(P, c)); }
};

// collide_dev<false, SCALED> for two nodes, one per lane of the F2 values:
// the same formulation (partial sums, quadratic differences through
// rho'/rho, hi parts of the constants), written with explicit multiply-adds.
// Negations are folded into constants or operands where that is exact
// (a sign flip never rounds), so no extra instruction carries them.
template <bool SCALED, typename K>
__device__ __forceinline__ void collide_pair(F2 &f0, F2 &f1, F2 &f2_, F2 &f3, F2 &f4, F2 &f5,
                                             F2 &f6, F2 &f7, F2 &f8, const K &P) {
  const F2 s13 = f1 + f3, s24 = f2_ + f4;
  const F2 d13 = f1 - f3, d24 = f2_ - f4;
  const F2 s57 = f5 + f7, s68 = f6 + f8;
  const F2 d57 = f5 - f7, d68 = f6 - f8;
  const F2 axis = s13 + s24;
  const F2 diag = s57 + s68;
  const F2 dxd = d57 - d68;
  const F2 dyd = d57 + d68;
  const F2 rho_p = (f0 + axis) + diag;
  const F2 jx_p = d13 + dxd;
  const F2 jy_p = d24 + dyd;

  const F2 IS = P(PC_IS);
  const F2 rho_phys = SCALED ? rho_p * IS : rho_p;
  // -rho'/rho per lane by the hardware reciprocal (the sign folded into
  // the numerator, which is exact)
  const F2 den = P(PC_R0) + rho_phys;
  float rl, rh, dl, dh;
  f2split(rho_phys, rl, rh);
  f2split(den, dl, dh);
  const F2 nc = f2(__fdividef(-rl, dl), __fdividef(-rh, dh));
  F2 jxx = jx_p * jx_p, jyy = jy_p * jy_p, jxy = jx_p * jy_p;
  if (SCALED) {
    jxx = jxx * IS;
    jyy = jyy * IS;
    jxy = jxy * IS;
  }
  const F2 tx = fma2(P(PC_2JX), jx_p, jxx);  // jx^2 - jx0^2
  const F2 ty = fma2(P(PC_2JY), jy_p, jyy);
  const F2 txy = fma2(P(PC_JX), jy_p, fma2(jx_p, P(PC_JY), jxy));
  const F2 R0 = P(PC_R0), I2 = P(PC_I2);
  const F2 nj = fma2(R0, tx + ty, rho_p * P(PC_NQ0)) * I2;
  const F2 np = fma2(R0, tx - ty, rho_p * P(PC_ND0)) * I2;
  const F2 nx = fma2(R0, txy, rho_p * P(PC_NX0)) * I2;
  const F2 djsq = fma2(nj, nc, nj);  // |j|^2/rho - |j0|^2/rho0
  const F2 dpxx = fma2(np, nc, np);
  const F2 dpxy = fma2(nx, nc, nx);

  const F2 n3 = fma2(f2s(-3.0f), djsq, fma2(f2s(4.0f), diag, fma2(f2s(-2.0f), f0, axis)));
  const F2 n4 = fma2(f2s(3.0f), djsq, f2s(3.0f) * (f0 - axis));
  // m5 = -(qx' + jx'), m6 = -(qy' + jy'): their rates enter negated
  const F2 m5 = fma2(f2s(-2.0f), dxd, d13);
  const F2 m6 = fma2(f2s(-2.0f), dyd, d24);
  const F2 n7 = (s13 - s24) - dpxx;
  const F2 n8 = (s57 - s68) - dpxy;
  const F2 r3 = n3 * P(PC_K3);
  const F2 r4 = n4 * P(PC_K4);
  const F2 r5 = m5 * P(PC_NK5);
  const F2 r6 = m6 * P(PC_NK6);
  const F2 r7 = n7 * P(PC_K7);
  const F2 r8 = n8 * P(PC_K8);

  const F2 TWO = f2s(2.0f), NTWO = f2s(-2.0f);
  const F2 a = fma2(TWO, r4, r3);  // axis velocities: -r3 - 2 r4
  const F2 b = fma2(TWO, r3, r4);  // diagonals: 2 r3 + r4
  f0 = fma2(f2s(-4.0f), r4 - r3, f0);
  const F2 ax = a - r7, ay = a + r7;
  f1 = f1 + fma2(TWO, r5, ax);
  f3 = f3 + fma2(NTWO, r5, ax);
  f2_ = f2_ + fma2(TWO, r6, ay);
  f4 = f4 + fma2(NTWO, r6, ay);
  const F2 bp = b + r5, bm = b - r5;
  f5 = f5 - ((bp + r6) + r8);
  f6 = f6 - ((bm + r6) - r8);
  f7 = f7 - ((bm - r6) + r8);
  f8 = f8 - ((bp - r6) - r8);
}

// ------------------------------------------------------------------
// FP64 deviation storage (LBM_F64DEV): the deviation form of collide_dev in
// FP64 with fused multiply-adds -- fewer and cheaper FP64 operations than the
// plain path's canonical operation order (GB300's FP64 units bound both),
// and rounding at the size of the perturbation, not of f.
struct DevParams64 {
  double rho0, jx0, jy0;          // reference state
  double k3, k4, k5, k6, k7, k8;  // s/D: s_e/36, s_eps/36, s_qx/12, s_qy/12, s_pxx/4, s_pxy/4
  double q0, d0, x0;              // |j0|^2, jx0^2 - jy0^2, jx0 jy0
  double i2;                      // 1 / rho0^2
};

__device__ __forceinline__ void collide_dev64(double &f0, double &f1, double &f2, double &f3,
                                              double &f4, double &f5, double &f6, double &f7,
                                              double &f8, const DevParams64 &P) {
  const double s13 = f1 + f3, s24 = f2 + f4;
  const double d13 = f1 - f3, d24 = f2 - f4;
  const double s57 = f5 + f7, s68 = f6 + f8;
  const double d57 = f5 - f7, d68 = f6 - f8;
  const double axis = s13 + s24;
  const double diag = s57 + s68;
  const double dxd = d57 - d68;
  const double dyd = d57 + d68;
  const double rho_p = f0 + axis + diag;
  const double jx_p = d13 + dxd;
  const double jy_p = d24 + dyd;
  // rho'/rho: only scales the quadratic terms.  1/rho by the hardware's
  // approximate FP64 reciprocal refined by two Newton-Raphson steps
  // (r <- r + r (1 - d r), each squaring the relative error: well below
  // 2^-50 after two), cheaper on GB300's FP64 pipe than the IEEE quotient
  const double den = P.rho0 + rho_p;
  double rinv;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(rinv) : "d"(den));
  rinv = fma(rinv, fma(-den, rinv, 1.0), rinv);
  rinv = fma(rinv, fma(-den, rinv, 1.0), rinv);
  const double c = rho_p * rinv;
  const double tx = fma(2.0 * P.jx0, jx_p, jx_p * jx_p);  // jx^2 - jx0^2
  const double ty = fma(2.0 * P.jy0, jy_p, jy_p * jy_p);
  const double txy = fma(P.jx0, jy_p, fma(jx_p, P.jy0, jx_p * jy_p));
  const double nj = fma(P.rho0, tx + ty, -rho_p * P.q0) * P.i2;
  const double np = fma(P.rho0, tx - ty, -rho_p * P.d0) * P.i2;
  const double nx = fma(P.rho0, txy, -rho_p * P.x0) * P.i2;
  const double djsq = fma(-nj, c, nj);
  const double dpxx = fma(-np, c, np);
  const double dpxy = fma(-nx, c, nx);
  const double n3 = fma(4.0, diag, axis - 2.0 * f0) - 3.0 * djsq;
  const double n4 = fma(3.0, djsq, 3.0 * (f0 - axis));
  const double n5 = fma(2.0, dxd, -d13);
  const double n6 = fma(2.0, dyd, -d24);
  const double n7 = (s13 - s24) - dpxx;
  const double n8 = (s57 - s68) - dpxy;
  const double r3 = n3 * P.k3, r4 = n4 * P.k4, r5 = n5 * P.k5;
  const double r6 = n6 * P.k6, r7 = n7 * P.k7, r8 = n8 * P.k8;
  const double a = fma(2.0, r4, r3);
  const double b = fma(2.0, r3, r4);
  f0 = fma(-4.0, r4 - r3, f0);
  f1 += fma(2.0, r5, a - r7);
  f3 += fma(-2.0, r5, a - r7);
  f2 += fma(2.0, r6, a + r7);
  f4 += fma(-2.0, r6, a + r7);
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

/*
 * Plain FP64 CPU oracle of the D2Q9 multi-relaxation-time lattice Boltzmann
 * scheme of Xu & Sagaut, "Optimal low-dispersion low-dissipation LBM schemes
 * for computational aeroacoustics" (arXiv 1107.4543).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it.  It shares no code, header, table or constant with the
 * CUDA library; the two are written independently from the paper.
 *
 * What it computes, and where the paper defines it:
 *   - the evolution  f_i(x + v_i dt, t + dt) = f_i + Lambda_ij (f_j^eq - f_j)
 *     (section 2.1, Eq. blbs), with Lambda = M^-1 S M (section 2.1);
 *   - the conserved moments m_0..m_2 = rho, j_x, j_y left unchanged and the
 *     others relaxed as m_i <- m_i + s_i (m_i^eq - m_i)
 *     (section 2.1, Eqs. eq_conservative and eq_noconservative);
 *   - m = M f, m^eq = M f^eq (section 2.1, Eq. q-macro);
 *   - the D2Q9 equilibrium moments of section 2.3
 *     {rho, jx, jy, -2 rho + 3|j|^2/rho, rho - 3|j|^2/rho, -jx, -jy,
 *      (jx^2 - jy^2)/rho, jx jy/rho}, which fix the moment order;
 *   - S = diag(0,0,0,s_e,s_eps,s_q,s_q,s_nu,s_nu) (section 2.3).
 *
 * Readings where the paper is silent (it prints neither the velocity order
 * nor M): velocities c_0..c_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),
 * (-1,1),(-1,-1),(1,-1); M is the Lallemand-Luo D2Q9 matrix with its rows put
 * in the paper's moment order.  Its rows are mutually orthogonal, so
 * M^-1 = M^T D^-1 with D = diag(M M^T); the oracle forms D from M itself.
 *
 * Layout: populations f[i][y][x], i = 0..8, contiguous, row length nx.
 * Periodic in x and y.  All arithmetic is IEEE FP64; build with
 * -ffp-contract=off so that no multiply-add is fused.
 *
 * The arithmetic type of the collision and streaming is `real`, FP64 unless
 * the file is compiled with -DORC_REAL="long double": that second build
 * (oracle/_build/liboracle_ext.so, the same algorithm in extended precision:
 * 64-bit significand on x86-64, IEEE quadruple on AArch64) is the reference
 * for GPU paths whose FP64 rounding differs from this file's, since the FP64
 * oracle's own rounding of populations of size ~0.4 is larger than the
 * 1e-12 relative gate of a density fluctuation of 1e-3 over hundreds of
 * steps.  The entry points keep FP64 arguments in both builds.
 *
 * Parity pins (tests/test_oracle_*.py): M M^T diagonal; M^-1 m^eq equal to the
 * textbook second-order polynomial equilibrium; the Jacobian of m^eq equal to
 * the printed Psi of section 2.3; exact conservation; equilibria as fixed
 * points; the BGK special case; streaming by brute force; small-amplitude
 * waves evolving by the von Neumann eigenvalues of section 4.1 built from the
 * printed Psi; the Gaussian pulse of section 5.2.
 */
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL real;

/* discrete velocities (reading, see header) */
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* moment matrix, rows rho, jx, jy, e, eps, qx, qy, pxx, pxy (section 2.3) */
static const double MM[Q][Q] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
};

static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int orc_get_threads(void) { return g_threads; }

void orc_velocities(int cx[Q], int cy[Q]) {
    for (int i = 0; i < Q; ++i) { cx[i] = CX[i]; cy[i] = CY[i]; }
}

/* M (row-major 9x9) and M^-1 = M^T D^-1 with D_k = sum_j M_kj^2 */
void orc_matrices(double M[Q * Q], double Minv[Q * Q]) {
    double D[Q];
    for (int k = 0; k < Q; ++k) {
        D[k] = 0.0;
        for (int j = 0; j < Q; ++j) D[k] += MM[k][j] * MM[k][j];
    }
    for (int k = 0; k < Q; ++k)
        for (int j = 0; j < Q; ++j) M[k * Q + j] = MM[k][j];
    for (int i = 0; i < Q; ++i)
        for (int k = 0; k < Q; ++k) Minv[i * Q + k] = MM[k][i] / D[k];
}

/* equilibrium moments of section 2.3, in the paper's order */
static void meq_r(real rho, real jx, real jy, real meq[Q]) {
    real jsq = jx * jx + jy * jy;
    meq[0] = rho;
    meq[1] = jx;
    meq[2] = jy;
    meq[3] = -2.0 * rho + 3.0 * jsq / rho;
    meq[4] = rho - 3.0 * jsq / rho;
    meq[5] = -jx;
    meq[6] = -jy;
    meq[7] = (jx * jx - jy * jy) / rho;
    meq[8] = jx * jy / rho;
}

void orc_meq(double rho, double jx, double jy, double meq[Q]) {
    real m[Q];
    meq_r(rho, jx, jy, m);
    for (int k = 0; k < Q; ++k) meq[k] = (double)m[k];
}

/* M^-1 = M^T D^-1, built once from M in the arithmetic type */
static real g_Minv[Q * Q];
static int g_ready = 0;

static void ensure_tables(void) {
    if (g_ready) return;
    real D[Q];
    for (int k = 0; k < Q; ++k) {
        D[k] = 0.0;
        for (int j = 0; j < Q; ++j) D[k] += (real)MM[k][j] * (real)MM[k][j];
    }
    for (int i = 0; i < Q; ++i)
        for (int k = 0; k < Q; ++k) g_Minv[i * Q + k] = (real)MM[k][i] / D[k];
    g_ready = 1;
}

/* one MRT collision at a node, in place: m = M f; m* = m - S (m - m^eq);
   f* = M^-1 m*, written as f - M^-1 S (m - m^eq).  s[] in paper order. */
static void collide_r(const real s[Q], real f[Q]) {
    const real *Minv = g_Minv;
    real m[Q], meq[Q], r[Q];
    for (int k = 0; k < Q; ++k) {
        real acc = 0.0;
        for (int j = 0; j < Q; ++j) acc += (real)MM[k][j] * f[j];
        m[k] = acc;
    }
    meq_r(m[0], m[1], m[2], meq);
    for (int k = 0; k < Q; ++k) r[k] = s[k] * (m[k] - meq[k]);
    for (int i = 0; i < Q; ++i) {
        real acc = 0.0;
        for (int k = 0; k < Q; ++k) acc += Minv[i * Q + k] * r[k];
        f[i] = f[i] - acc;
    }
}

void orc_collide(const double s[Q], double f[Q]) {
    real sr[Q], fr[Q];
    ensure_tables();
    for (int k = 0; k < Q; ++k) { sr[k] = s[k]; fr[k] = f[k]; }
    collide_r(sr, fr);
    for (int k = 0; k < Q; ++k) f[k] = (double)fr[k];
}

static inline int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

/* nsteps of collide-then-stream (Eq. blbs) on a periodic nx x ny lattice.
   f: 9*ny*nx populations at time t (pre-collision), overwritten with those
   at time t + nsteps.  Returns 0, or -1 on bad arguments / no memory. */
int orc_run(int nx, int ny, const double s[Q], double *f, long nsteps) {
    if (nx < 1 || ny < 1 || nsteps < 0) return -1;
    ensure_tables(); /* built once, before any thread starts */
    size_t plane = (size_t)nx * (size_t)ny;
    real *a = (real *)malloc(sizeof(real) * Q * plane);
    real *g = (real *)malloc(sizeof(real) * Q * plane);
    if (!a || !g) { free(a); free(g); return -1; }
    real sr[Q];
    for (int k = 0; k < Q; ++k) sr[k] = s[k];
    for (size_t n = 0; n < Q * plane; ++n) a[n] = f[n];
    real *src = a, *dst = g;
    for (long t = 0; t < nsteps; ++t) {
#pragma omp parallel for num_threads(g_threads) schedule(static)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                real fn[Q];
                size_t n = (size_t)y * nx + x;
                for (int i = 0; i < Q; ++i) fn[i] = src[i * plane + n];
                collide_r(sr, fn);
                for (int i = 0; i < Q; ++i) {
                    int xd = wrap(x + CX[i], nx), yd = wrap(y + CY[i], ny);
                    dst[i * plane + (size_t)yd * nx + xd] = fn[i];
                }
            }
        }
        real *tmp = src; src = dst; dst = tmp;
    }
    for (size_t n = 0; n < Q * plane; ++n) f[n] = (double)src[n];
    free(a);
    free(g);
    return 0;
}

/* f^eq(rho, u) = M^-1 m^eq(rho, rho u) at one node */
static void feq_node(const double *Minv, double rho, double ux, double uy, double f[Q]) {
    double meq[Q];
    orc_meq(rho, rho * ux, rho * uy, meq);
    for (int i = 0; i < Q; ++i) {
        double acc = 0.0;
        for (int k = 0; k < Q; ++k) acc += Minv[i * Q + k] * meq[k];
        f[i] = acc;
    }
}

/* As orc_run, with the acoustic point source of section 5.1: before the
   collision of every step (lattice time t = t0, t0 + 1, ...) the node
   (sx, sy) is set to the equilibrium at rest with density
   rho0 + amp sin(2 pi t / period). */
int orc_run_source(int nx, int ny, const double s[Q], double *f, long nsteps, long t0,
                   int sx, int sy, double rho0, double amp, double period) {
    if (sx < 0 || sx >= nx || sy < 0 || sy >= ny || !(period > 0)) return -1;
    const double PI = 3.14159265358979323846;
    double M[Q * Q], Minv[Q * Q];
    orc_matrices(M, Minv);
    size_t plane = (size_t)nx * (size_t)ny;
    for (long k = 0; k < nsteps; ++k) {
        double fs[Q];
        double rho_t = rho0 + amp * sin(2.0 * PI * (double)(t0 + k) / period);
        feq_node(Minv, rho_t, 0.0, 0.0, fs);
        for (int i = 0; i < Q; ++i) f[i * plane + (size_t)sy * nx + sx] = fs[i];
        int rc = orc_run(nx, ny, s, f, 1);
        if (rc != 0) return rc;
    }
    return 0;
}

/* f = f^eq(rho, u) = M^-1 m^eq(rho, rho u) at every node */
void orc_init_eq(int nx, int ny, const double *rho, const double *ux,
                 const double *uy, double *f) {
    double M[Q * Q], Minv[Q * Q];
    orc_matrices(M, Minv);
    size_t plane = (size_t)nx * (size_t)ny;
    for (size_t n = 0; n < plane; ++n) {
        double meq[Q];
        orc_meq(rho[n], rho[n] * ux[n], rho[n] * uy[n], meq);
        for (int i = 0; i < Q; ++i) {
            double acc = 0.0;
            for (int k = 0; k < Q; ++k) acc += Minv[i * Q + k] * meq[k];
            f[i * plane + n] = acc;
        }
    }
}

/* rho = m_0, u = (m_1, m_2) / rho at every node */
void orc_moments(int nx, int ny, const double *f, double *rho, double *ux,
                 double *uy) {
    size_t plane = (size_t)nx * (size_t)ny;
    for (size_t n = 0; n < plane; ++n) {
        double m[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < Q; ++j) m[k] += MM[k][j] * f[j * plane + n];
        rho[n] = m[0];
        ux[n] = m[1] / m[0];
        uy[n] = m[2] / m[0];
    }
}

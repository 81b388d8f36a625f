/* Drives the C oracle (oracle/lbm_oracle.c) through every entry point on
 * small ragged lattices, built with AddressSanitizer and
 * UndefinedBehaviorSanitizer by tests/test_oracle_sanitizers.py: any
 * out-of-bounds access, use of uninitialized memory through a bad index, or
 * undefined arithmetic aborts the run.  Prints "OK" at the end. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#define Q 9
void orc_set_threads(int n);
void orc_velocities(int cx[Q], int cy[Q]);
void orc_matrices(double M[Q * Q], double Minv[Q * Q]);
void orc_meq(double rho, double jx, double jy, double meq[Q]);
void orc_collide(const double s[Q], double f[Q]);
int orc_run(int nx, int ny, const double s[Q], double *f, long nsteps);
int orc_run_source(int nx, int ny, const double s[Q], double *f, long nsteps, long t0,
                   int sx, int sy, double rho0, double amp, double period);
void orc_init_eq(int nx, int ny, const double *rho, const double *ux, const double *uy,
                 double *f);
void orc_moments(int nx, int ny, const double *f, double *rho, double *ux, double *uy);

int main(void) {
  const double s[Q] = {0, 0, 0, 1.64, 1.54, 1.9, 1.9, 1.99, 1.99};
  int cx[Q], cy[Q];
  double M[Q * Q], Minv[Q * Q], meq[Q], f1[Q];
  orc_velocities(cx, cy);
  orc_matrices(M, Minv);
  orc_meq(1.01, 0.02, -0.01, meq);
  for (int i = 0; i < Q; ++i) f1[i] = 1.0 / 9.0 + 1e-3 * i;
  orc_collide(s, f1);
  const int sizes[][2] = {{2, 2}, {3, 5}, {7, 2}, {33, 17}, {2, 9}};
  for (int threads = 1; threads <= 4; threads += 3) {
    orc_set_threads(threads);
    for (int k = 0; k < 5; ++k) {
      const int nx = sizes[k][0], ny = sizes[k][1], n = nx * ny;
      double *rho = malloc(sizeof(double) * n), *ux = malloc(sizeof(double) * n);
      double *uy = malloc(sizeof(double) * n), *f = malloc(sizeof(double) * Q * n);
      for (int j = 0; j < n; ++j) {
        rho[j] = 1.0 + 1e-3 * sin(0.3 * j);
        ux[j] = 1e-3 * cos(0.2 * j);
        uy[j] = -1e-3 * sin(0.1 * j);
      }
      orc_init_eq(nx, ny, rho, ux, uy, f);
      orc_run(nx, ny, s, f, 7);
      orc_run_source(nx, ny, s, f, 5, 3, nx - 1, ny - 1, 1.0, 1e-3, 20.0);
      orc_moments(nx, ny, f, rho, ux, uy);
      for (int j = 0; j < n; ++j)
        if (!isfinite(rho[j]) || !isfinite(ux[j]) || !isfinite(uy[j])) {
          printf("non-finite moment\n");
          return 1;
        }
      free(rho);
      free(ux);
      free(uy);
      free(f);
    }
  }
  printf("OK\n");
  return 0;
}

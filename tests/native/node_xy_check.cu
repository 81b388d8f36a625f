// Host-compiled check of the auxiliary kernels' node coordinates
// (node_xy.cuh): node_xy against 64-bit division on sampled indices around
// the 32-bit boundary, and NodeWalk against division at every node of
// grid-stride walks of the strides the drift kernels use.  Built and run by
// tests/test_node_xy_cpu.py; prints "OK" and exits 0 when every check holds.
#include <stdio.h>

#include "../../paper_1107_4543_gb300/csrc/node_xy.cuh"

using namespace lbm;

static int failures = 0;
#define CHECK(cond, ...)                                  \
  do {                                                    \
    if (!(cond)) {                                        \
      if (failures < 20) {                                \
        printf("FAIL %s:%d: ", __FILE__, __LINE__);       \
        printf(__VA_ARGS__);                              \
        printf("\n");                                     \
      }                                                   \
      ++failures;                                         \
    }                                                     \
  } while (0)

static void check_xy(long long n, int nx) {
  int x = -1, y = -1;
  node_xy(n, nx, x, y);
  CHECK(y == (int)(n / nx) && x == (int)(n % nx), "node_xy(%lld, %d) = (%d, %d)", n, nx, x, y);
}

static void check_walk(int nx, long long N, long long stride) {
  for (long long n0 = 0; n0 < stride && n0 < N; n0 += (stride > 97 ? stride / 97 : 1)) {
    NodeWalk w(n0, stride, nx);
    for (long long n = n0; n < N; n += stride, w.next())
      CHECK(w.y == (int)(n / nx) && w.x == (int)(n % nx),
            "walk nx=%d stride=%lld n=%lld: (%d, %d)", nx, stride, n, w.x, w.y);
  }
}

int main() {
  const int widths[] = {1, 2, 3, 7, 31, 32, 33, 255, 256, 1000, 4095, 4096, 4097, 65536,
                        100003, 1 << 20, (1 << 30) + 7, 0x7fffffff};
  const long long edges[] = {0, 1, 2, 0x7ffffffdLL, 0x7ffffffeLL, 0x7fffffffLL, 0x80000000LL,
                             0x80000001LL, 0xffffffffLL, 0x100000000LL, 0x100000001LL,
                             (1LL << 40) + 12345};
  for (int nx : widths) {
    for (long long n : edges) check_xy(n, nx);
    for (long long n = 0; n < 5000; ++n) check_xy(n, nx);
    for (long long k = -3; k <= 3; ++k)
      for (long long m : {1LL, 2LL, 1000LL, 0x7fffffffLL / nx, 0x80000000LL / nx + 1}) {
        const long long n = m * nx + k;
        if (n >= 0) check_xy(n, nx);
      }
  }
  // grid-stride walks: the drift kernels' strides (16 or more blocks of 256
  // threads), strides below, equal to and above the width, and a lattice
  // whose node count passes 2^31
  const long long strides[] = {1, 7, 256, 4096, 4097, 65536, 16LL * 256, 1024LL * 256,
                               152LL * 16 * 256};
  const int wnx[] = {1, 3, 32, 37, 255, 256, 4096, 4097, 1000, 8192, 100003};
  for (int nx : wnx)
    for (long long s : strides) {
      const long long ny = nx < 64 ? 997 : (nx < 5000 ? 211 : 23);
      check_walk(nx, (long long)nx * ny, s);
    }
  {
    // 65536 x 32769 nodes (> 2^31): the walk crosses the 32-bit boundary
    const int nx = 65536;
    const long long N = (long long)nx * 32769, s = 152LL * 16 * 256 * 97;
    NodeWalk w(12345, s, nx);
    for (long long n = 12345; n < N; n += s, w.next())
      CHECK(w.y == (int)(n / nx) && w.x == (int)(n % nx), "big walk n=%lld", n);
  }
  if (failures) {
    printf("%d failures\n", failures);
    return 1;
  }
  printf("OK\n");
  return 0;
}

// Host-compiled check of the step kernels' work mapping (d2q9_pull.cuh):
// make_geom and lane_pos, exhaustively on tiny lattices, and the
// multiply-shift row division on sampled chunk indices.  Built and run by
// tests/test_lane_map_cpu.py; prints "OK" and exits 0 when every check holds.
#include <stdio.h>
#include <stdlib.h>

#include <vector>

#include "../../paper_1107_4543_gb300/csrc/d2q9_pull.cuh"

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

template <int V>
static void check_lattice(int nx, int ny, int esize) {
  const Geom g = make_geom(nx, ny, V, esize);
  // rows start on 128-byte lines (4-byte elements) or 64-byte halves of
  // lines (2-byte elements)
  const int line = esize == 2 ? 64 : 128;
  CHECK(g.pitch >= nx && (g.pitch * esize) % line == 0 && g.pitch - nx < line / esize + V,
        "pitch %d nx %d", g.pitch, nx);
  CHECK(g.nchunks * V >= nx && (g.nchunks - 1) * V < nx, "chunks nx %d V %d", nx, V);
  // whole lines of chunk slots per row, or the real chunks alone where the
  // padding slots exceed an eighth of the row
  const int slots = g.pitch / V;
  const bool whole = (slots - g.nchunks) * 8 <= slots;
  CHECK(g.cpr == (whole ? slots : g.nchunks), "mapping nx %d V %d cpr %d", nx, V, g.cpr);
  CHECK(g.plane == g.pitch && g.rstride == 9LL * g.pitch, "layout");
  std::vector<int> seen((size_t)ny * g.nchunks, 0);
  for (long long task = 0; task < g.tasks; ++task)
    for (int lane = 0; lane < 32; ++lane) {
      const LanePos p = lane_pos<V>(g, task, lane);
      const long long c = task * 32 + lane;
      const long long y = c / g.cpr, xc = c % g.cpr;
      const bool real = y < ny && xc < g.nchunks;
      CHECK(p.active == real, "active nx %d ny %d V %d c %lld", nx, ny, V, c);
      if (!real) continue;
      CHECK(p.y == y && p.x0 == xc * V, "position nx %d ny %d V %d c %lld", nx, ny, V, c);
      CHECK(p.first == (lane == 0 || xc == 0), "first nx %d V %d c %lld", nx, V, c);
      CHECK(p.last == (lane == 31 || xc + 1 == g.nchunks), "last nx %d V %d c %lld", nx, V, c);
      // with whole lines per row every task starts on such a line
      if (lane == 0 && whole)
        CHECK((xc * V * esize) % line == 0, "task alignment nx %d V %d", nx, V);
      seen[(size_t)y * g.nchunks + xc]++;
    }
  for (size_t k = 0; k < seen.size(); ++k) CHECK(seen[k] == 1, "chunk %zu seen %d times", k, seen[k]);
}

static void check_division() {
  unsigned long long state = 12345;
  auto next = [&]() {
    state = state * 6364136223846793005ULL + 1442695040888963407ULL;
    return (unsigned)(state >> 33);  // < 2^31
  };
  for (int cpr = 1; cpr <= 70000; cpr = cpr < 512 ? cpr + 1 : cpr * 2 + 7) {
    Geom g = make_geom(cpr * 4, 1, 4, 4);  // FP32: cpr = pitch / 4 when nx is a multiple of 32
    if (g.cpr != cpr) continue;
    for (int s = 0; s < 2000; ++s) {
      unsigned c = next();
      if (s < 6) c = s < 3 ? (unsigned)(cpr * (long long)(s + 1) - 1) : 0x7fffffffu - s;
      const unsigned y = (unsigned)(((unsigned long long)c * g.dmul) >> g.dshift);
      CHECK(y == c / (unsigned)cpr, "division cpr %d c %u", cpr, c);
    }
  }
}

int main() {
  for (int ny = 1; ny <= 7; ++ny)
    for (int nx = 1; nx <= 300; ++nx) {
      check_lattice<2>(nx, ny, 8);
      check_lattice<4>(nx, ny, 4);
      check_lattice<8>(nx, ny, 2);
    }
  check_division();
  if (failures) {
    printf("%d failures\n", failures);
    return 1;
  }
  printf("OK\n");
  return 0;
}

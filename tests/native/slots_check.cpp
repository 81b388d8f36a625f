// Host check of SlotRanges (slots.h), the slot ranges of the batched step's
// constant tables: first fit, release and reuse, exhaustion, bad sizes and
// ranges, against a brute-force model on a random sequence of operations.
// Built and run by tests/test_slots_cpu.py; prints "OK" and exits 0 when
// every check holds.
#include <stdio.h>

#include <random>
#include <utility>
#include <vector>

#include "../../paper_1107_4543_gb300/csrc/slots.h"

using lbm::SlotRanges;

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

// the lowest start of n free slots in a plain occupancy array, or -1
static int model_first_fit(const std::vector<int> &used, int n) {
  const int cap = (int)used.size();
  if (n < 1 || n > cap) return -1;
  for (int b = 0; b + n <= cap; ++b) {
    bool ok = true;
    for (int k = b; k < b + n && ok; ++k) ok = used[k] == 0;
    if (ok) return b;
  }
  return -1;
}

int main() {
  // fixed cases on a table of 960 slots
  {
    SlotRanges t(960);
    CHECK(t.capacity() == 960 && t.free_slots() == 960, "fresh table");
    CHECK(t.reserve(0) == -1 && t.reserve(-3) == -1 && t.reserve(961) == -1, "bad sizes");
    const int a = t.reserve(958);
    CHECK(a == 0, "first range at 0, got %d", a);
    CHECK(t.reserve(3) == -1, "no room for 3 after 958");
    const int b = t.reserve(2);
    CHECK(b == 958, "the last 2 slots, got %d", b);
    CHECK(t.free_slots() == 0, "full");
    t.release(0, 958);
    const int c = t.reserve(4);
    CHECK(c == 0, "released slots taken again from 0, got %d", c);
    t.release(-1, 5);
    t.release(958, 3);  // past the end: ignored
    t.release(3, 0);
    CHECK(t.free_slots() == 954, "ignored bad releases, %d free", t.free_slots());
    t.release(958, 2);
    CHECK(t.free_slots() == 956, "valid release, %d free", t.free_slots());
  }
  {
    SlotRanges z(0);
    CHECK(z.capacity() == 0 && z.reserve(1) == -1, "empty table");
  }
  // random reserve / release sequences against the model
  std::mt19937 rng(1107);
  for (int trial = 0; trial < 200; ++trial) {
    const int cap = 1 + (int)(rng() % 700);
    SlotRanges t(cap);
    std::vector<int> used(cap, 0);
    std::vector<std::pair<int, int>> held;
    for (int op = 0; op < 400; ++op) {
      if (!held.empty() && rng() % 3 == 0) {
        const size_t k = rng() % held.size();
        t.release(held[k].first, held[k].second);
        for (int s = held[k].first; s < held[k].first + held[k].second; ++s) used[s] = 0;
        held.erase(held.begin() + (long)k);
      } else {
        const int n = (int)(rng() % 4 == 0 ? rng() % (cap + 2) : 1 + rng() % 40);
        const int want = model_first_fit(used, n);
        const int got = t.reserve(n);
        CHECK(got == want, "cap %d reserve %d: got %d, model %d", cap, n, got, want);
        if (got >= 0) {
          for (int s = got; s < got + n; ++s) used[s] = 1;
          held.push_back({got, n});
        }
      }
      int fr = 0;
      for (int u : used) fr += u == 0;
      CHECK(t.free_slots() == fr, "free count %d, model %d", t.free_slots(), fr);
    }
  }
  if (failures) {
    printf("%d failures\n", failures);
    return 1;
  }
  printf("OK\n");
  return 0;
}

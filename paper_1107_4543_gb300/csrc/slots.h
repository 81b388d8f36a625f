// Contiguous slot ranges of a fixed-capacity table (host only): the
// batched step's constant-memory tables hand each batch group one range of
// lattice slots for the group's lifetime.  First fit from slot 0; not
// thread-safe by itself (batch.cu holds a mutex around it).
#pragma once
#include <algorithm>
#include <vector>

namespace lbm {

class SlotRanges {
 public:
  explicit SlotRanges(int capacity) : used_(capacity > 0 ? capacity : 0, 0) {}

  int capacity() const { return (int)used_.size(); }

  // First slot of the lowest run of n free slots, now taken; -1 when n is
  // not in [1, capacity] or no run of n free slots exists.
  int reserve(int n) {
    const int cap = capacity();
    if (n < 1 || n > cap) return -1;
    for (int s = 0, run = 0; s < cap; ++s) {
      run = used_[s] ? 0 : run + 1;
      if (run == n) {
        std::fill(used_.begin() + (s - n + 1), used_.begin() + (s + 1), 1);
        return s - n + 1;
      }
    }
    return -1;
  }

  // Free slots base .. base + n - 1 (a range reserve returned); a range
  // outside the table is ignored.
  void release(int base, int n) {
    if (base < 0 || n < 1 || base + n > capacity()) return;
    std::fill(used_.begin() + base, used_.begin() + base + n, 0);
  }

  int free_slots() const { return (int)std::count(used_.begin(), used_.end(), 0); }

 private:
  std::vector<char> used_;
};

}  // namespace lbm

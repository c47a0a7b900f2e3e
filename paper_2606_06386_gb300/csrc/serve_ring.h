// Ring allocator of the serving loop's pinned operand and result rings (host
// code only, so that its logic is tested on the CPU): allocations in digits,
// released first-in first-out.
#pragma once
#include <cstdint>
#include <deque>

namespace mp_serve {

// Ring allocator in digits with first-in first-out release; an allocation
// that would cross the end starts again at 0 and the skipped tail counts as
// used until it is released with its allocation.
struct Ring {
  int64_t cap = 0, tail = 0, used = 0;
  struct Entry {
    int64_t len;  // includes any skipped gap before the allocation
    bool done;
  };
  std::deque<Entry> live;
  int64_t front_seq = 0;  // sequence number of live.front()
  // returns the offset (or -1) and the allocation's sequence number in *seq
  int64_t alloc(int64_t n, int64_t* seq) {
    n = (n + 3) & ~int64_t(3);
    if (n > cap) return -1;
    int64_t off = tail, gap = 0;
    if (off + n > cap) {
      gap = cap - off;
      off = 0;
    }
    if (used + gap + n > cap) return -1;
    tail = off + n;
    if (tail == cap) tail = 0;
    used += gap + n;
    *seq = front_seq + (int64_t)live.size();
    live.push_back({gap + n, false});
    return off;
  }
  // mark allocation `seq` finished, then free finished ones from the front
  void release(int64_t seq) {
    live[(size_t)(seq - front_seq)].done = true;
    while (!live.empty() && live.front().done) {
      used -= live.front().len;
      live.pop_front();
      front_seq++;
    }
    if (live.empty()) {
      tail = 0;
      used = 0;
    }
  }
};

}  // namespace mp_serve

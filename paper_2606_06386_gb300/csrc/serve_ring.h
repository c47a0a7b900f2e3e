// Ring allocator of the serving loop's pinned operand and result rings (host
// code only, so that its logic is tested on the CPU): allocations in digits,
// released first-in first-out.
#pragma once
#include <algorithm>
#include <cstdint>
#include <deque>
#include <vector>

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

// Allocation by class in chunks of a Ring: the requests of one class take
// consecutive space in the class's current chunk, so that a batch of one
// class's requests covers one contiguous run of the ring, or a few (one per
// chunk it reaches into), with nothing of other classes inside. A chunk that
// is no longer current goes back to the ring with its last request; a
// current chunk goes back as soon as none of its requests is live, so an
// idle class holds no space.
struct ChunkedRing {
  struct Chunk {
    int64_t off = 0, len = 0, used = 0, seq = -1;
    int live = 0;  // requests allocated and not yet released
    int cls = -1;  // the class whose current chunk it is (-1: closed)
  };
  Ring ring;
  int64_t chunk_digits = 1 << 20;  // default chunk size (a request larger than that gets its own)
  std::vector<Chunk*> cur;         // current chunk per class (null: none)

  explicit ChunkedRing(int classes = 1) : cur((size_t)classes, nullptr) {}
  ChunkedRing(const ChunkedRing&) = delete;
  ChunkedRing& operator=(const ChunkedRing&) = delete;
  ~ChunkedRing() {
    for (Chunk* c : cur) delete c;
  }
  // n digits (rounded up to 4) for a request of class cls: the offset, and
  // its chunk in *out; -1 when the ring has no room for a new chunk
  int64_t alloc(int cls, int64_t n, Chunk** out) {
    n = (n + 3) & ~int64_t(3);
    Chunk* c = cur[(size_t)cls];
    if (c != nullptr && c->used + n <= c->len) {
      const int64_t off = c->off + c->used;
      c->used += n;
      c->live++;
      *out = c;
      return off;
    }
    int64_t seq = -1;
    const int64_t len = std::max(n, std::min(chunk_digits, ring.cap / 8));
    const int64_t off = ring.alloc(len, &seq);
    if (off < 0) return -1;
    if (c != nullptr) c->cls = -1;  // closed; it has live requests (an empty current chunk is already gone)
    Chunk* d = new Chunk;
    d->off = off;
    d->len = len;
    d->used = n;
    d->seq = seq;
    d->live = 1;
    d->cls = cls;
    cur[(size_t)cls] = d;
    *out = d;
    return off;
  }
  // one request of chunk c is done
  void release(Chunk* c) {
    if (--c->live > 0) return;
    if (c->cls >= 0) cur[(size_t)c->cls] = nullptr;
    ring.release(c->seq);
    delete c;
  }
};

}  // namespace mp_serve

// Randomised check of the serving loop's ring allocator against a model of
// the live byte ranges: allocations stay inside the ring, never overlap a live
// allocation, are refused only when no room is left, and the ring is whole
// again once everything is released. Prints "ok" or the first violation.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>
#include <vector>

#include "serve_ring.h"

struct Live {
  int64_t off, len, seq;
};

int main() {
  std::mt19937_64 rng(12345);
  for (int trial = 0; trial < 200; trial++) {
    mp_serve::Ring r;
    r.cap = 64 + (int64_t)(rng() % 4000) * 4;
    std::vector<Live> live;  // in allocation order
    for (int step = 0; step < 4000; step++) {
      const bool do_alloc = live.empty() || (rng() % 100) < 55;
      if (do_alloc) {
        const int64_t n = 1 + (int64_t)(rng() % (r.cap / 3 + 1));
        int64_t seq = -1;
        const int64_t off = r.alloc(n, &seq);
        const int64_t len = (n + 3) & ~int64_t(3);
        if (off < 0) {
          // a refusal must mean there is no free run of len digits at the
          // ring's next position or after wrapping to 0
          if (live.empty() && len <= r.cap) {
            std::printf("refused %lld digits in an empty ring of %lld\n", (long long)len, (long long)r.cap);
            return 1;
          }
          continue;
        }
        if (off < 0 || off + len > r.cap || (off & 3)) {
          std::printf("allocation [%lld, %lld) outside ring %lld\n", (long long)off, (long long)(off + len),
                      (long long)r.cap);
          return 1;
        }
        for (const Live& l : live)
          if (off < l.off + l.len && l.off < off + len) {
            std::printf("allocation [%lld, %lld) overlaps live [%lld, %lld)\n", (long long)off, (long long)(off + len),
                        (long long)l.off, (long long)(l.off + l.len));
            return 1;
          }
        if (!live.empty() && seq != live.back().seq + 1 && seq <= live.back().seq) {
          std::printf("sequence numbers not increasing\n");
          return 1;
        }
        live.push_back({off, len, seq});
      } else {
        // release a random live allocation (out of order); the ring frees
        // space only from its oldest allocation on
        const size_t k = rng() % live.size();
        r.release(live[k].seq);
        live.erase(live.begin() + (long)k);
      }
      if (r.used < 0 || r.used > r.cap) {
        std::printf("used %lld outside [0, %lld]\n", (long long)r.used, (long long)r.cap);
        return 1;
      }
    }
    for (const Live& l : live) r.release(l.seq);
    if (r.used != 0 || !r.live.empty() || r.tail != 0) {
      std::printf("ring not whole after releasing everything\n");
      return 1;
    }
    int64_t seq = -1;
    if (r.alloc(r.cap, &seq) != 0) {
      std::printf("a whole-ring allocation failed after release\n");
      return 1;
    }
  }
  // the chunked allocation by class on top of the ring: live requests never
  // overlap, a class's requests in one chunk are consecutive, an empty ring
  // never refuses, and everything returns to the ring once released
  for (int trial = 0; trial < 200; trial++) {
    const int classes = 1 + (int)(rng() % 5);
    mp_serve::ChunkedRing cr(classes);
    cr.ring.cap = 256 + (int64_t)(rng() % 8000) * 4;
    cr.chunk_digits = 16 + (int64_t)(rng() % 600);
    struct Req {
      int64_t off, len;
      mp_serve::ChunkedRing::Chunk* chunk;
    };
    std::vector<Req> live;
    std::vector<Req> last(classes, Req{-1, 0, nullptr});  // each class's latest allocation
    for (int step = 0; step < 4000; step++) {
      const bool do_alloc = live.empty() || (rng() % 100) < 55;
      if (do_alloc) {
        const int cls = (int)(rng() % classes);
        const int64_t n = 1 + (int64_t)(rng() % (cr.ring.cap / 16 + 1));
        mp_serve::ChunkedRing::Chunk* c = nullptr;
        const int64_t off = cr.alloc(cls, n, &c);
        const int64_t len = (n + 3) & ~int64_t(3);
        if (off < 0) {
          if (live.empty()) {
            std::printf("chunked: refused %lld digits with nothing live\n", (long long)len);
            return 1;
          }
          continue;
        }
        if (off + len > cr.ring.cap || (off & 3) || c == nullptr || off < c->off || off + len > c->off + c->len) {
          std::printf("chunked: allocation [%lld, %lld) outside its chunk or the ring\n", (long long)off,
                      (long long)(off + len));
          return 1;
        }
        for (const Req& l : live)
          if (off < l.off + l.len && l.off < off + len) {
            std::printf("chunked: allocation [%lld, %lld) overlaps live [%lld, %lld)\n", (long long)off,
                        (long long)(off + len), (long long)l.off, (long long)(l.off + l.len));
            return 1;
          }
        const Req& p = last[cls];
        if (p.chunk == c && p.off + p.len != off) {
          std::printf("chunked: a class's requests in one chunk are not consecutive\n");
          return 1;
        }
        live.push_back({off, len, c});
        last[cls] = {off, len, c};
      } else {
        const size_t k = rng() % live.size();
        mp_serve::ChunkedRing::Chunk* c = live[k].chunk;
        live.erase(live.begin() + (long)k);
        bool still = false;  // the chunk stays allocated while one of its requests is live
        for (const Req& l : live) still = still || l.chunk == c;
        for (Req& l : last)
          if (l.chunk == c && !still) l = Req{-1, 0, nullptr};
        cr.release(c);
      }
    }
    for (const Req& l : live) cr.release(l.chunk);
    if (cr.ring.used != 0 || !cr.ring.live.empty()) {
      std::printf("chunked: ring not whole after releasing everything\n");
      return 1;
    }
    for (auto* c : cr.cur)
      if (c != nullptr) {
        std::printf("chunked: a current chunk outlived its requests\n");
        return 1;
      }
  }
  std::printf("ok\n");
  return 0;
}

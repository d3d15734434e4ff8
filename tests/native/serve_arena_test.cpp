// Unit test of the serving loop's host logic (no GPU): the output arena and
// the admission rule of paper_2408_11971_gb300/csrc/serve_arena.h.
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <random>
#include <vector>

#include "serve_arena.h"

using hz::serve::Arena;

#define CHECK(c)                                                     \
  do {                                                               \
    if (!(c)) {                                                      \
      std::fprintf(stderr, "%s:%d: CHECK failed: %s\n", __FILE__, __LINE__, #c); \
      std::exit(1);                                                  \
    }                                                                \
  } while (0)

struct Req {
  int id;
  uint64_t bytes;
  uint64_t arrival_us;
};

static void arena_basics() {
  Arena a(10 * 256 + 100);  // rounded down to 10 granules
  CHECK(a.size() == 2560);
  uint64_t o1, o2, o3, o4;
  CHECK(a.alloc(1, &o1) && o1 == 0);          // one granule
  CHECK(a.alloc(300, &o2) && o2 == 256);      // two granules
  CHECK(a.alloc(0, &o3) && o3 == 768);        // zero bytes still takes a granule
  CHECK(a.in_use() == 4 * 256 && a.peak() == 4 * 256);
  CHECK(!a.alloc(7 * 256, &o4));              // 6 granules left
  CHECK(a.alloc(6 * 256, &o4) && o4 == 1024);
  CHECK(a.largest_free() == 0);
  CHECK(a.release(o2));                       // hole of 2 granules at 256
  CHECK(!a.release(o2));                      // not a block any more
  CHECK(!a.release(12345));
  CHECK(a.largest_free() == 512);
  CHECK(a.release(o1));                       // merges with the hole: 3 granules at 0
  CHECK(a.largest_free() == 768);
  CHECK(a.shrink(o4, 256));                   // keep 1 granule, 5 return
  CHECK(a.largest_free() == 5 * 256);
  CHECK(a.release(o3));                       // [0, 1024) free again
  CHECK(a.largest_free() == 5 * 256);         // 1024..1280 used by o4
  CHECK(a.release(o4));
  CHECK(a.largest_free() == 2560 && a.in_use() == 0 && a.blocks() == 0);
  CHECK(a.peak() == 10 * 256);
}

// Random alloc/free/shrink against a shadow map of the granules.
static void arena_random() {
  std::mt19937_64 rng(7);
  const uint64_t G = 512;
  Arena a(G * 256);
  std::vector<int> owner(G, -1);
  std::vector<std::pair<uint64_t, uint64_t>> live;  // offset, granules
  for (int it = 0; it < 20000; it++) {
    const int act = (int)(rng() % 3);
    if (act == 0 || live.empty()) {
      const uint64_t bytes = rng() % (8 * 256) + 1;
      uint64_t off;
      const uint64_t g = (bytes + 255) / 256;
      // first fit must find a run if the shadow has one
      uint64_t run = 0, first = ~0ull;
      for (uint64_t i = 0; i < G; i++) {
        run = owner[i] < 0 ? run + 1 : 0;
        if (run == g) { first = i + 1 - g; break; }
      }
      const bool ok = a.alloc(bytes, &off);
      CHECK(ok == (first != ~0ull));
      if (ok) {
        CHECK(off == first * 256);
        for (uint64_t i = 0; i < g; i++) owner[first + i] = it;
        live.push_back({off, g});
      }
    } else if (act == 1) {
      const size_t k = rng() % live.size();
      CHECK(a.release(live[k].first));
      for (uint64_t i = 0; i < live[k].second; i++) owner[live[k].first / 256 + i] = -1;
      live.erase(live.begin() + k);
    } else {
      const size_t k = rng() % live.size();
      const uint64_t keep = rng() % (live[k].second * 256) + 1;
      const uint64_t kg = (keep + 255) / 256;
      CHECK(a.shrink(live[k].first, keep));
      for (uint64_t i = kg; i < live[k].second; i++) owner[live[k].first / 256 + i] = -1;
      live[k].second = kg;
    }
    uint64_t used = 0;
    for (uint64_t i = 0; i < G; i++) used += owner[i] >= 0;
    CHECK(a.in_use() == used * 256);
  }
}

static void admission() {
  Arena a(4 * 256);
  auto need = [](const Req& r) { return r.bytes; };
  std::deque<Req> q;
  uint64_t off;
  // FIFO: the head goes first
  q = {{0, 256, 0}, {1, 0, 0}};
  CHECK(hz::serve::pick_next(q, 10, a, need, &off) == 0 && off == 0);
  // a head that waits for memory is passed only by requests needing none
  q = {{2, 4 * 256, 0}, {3, 256, 0}, {4, 0, 0}, {5, 0, 0}};
  CHECK(hz::serve::pick_next(q, 10, a, need, &off) == 2 && off == ~0ull);
  q.erase(q.begin() + 2);
  CHECK(hz::serve::pick_next(q, 10, a, need, &off) == 2 && off == ~0ull);
  q.erase(q.begin() + 2);
  CHECK(hz::serve::pick_next(q, 10, a, need, &off) == -1);  // request 3 fits but may not pass
  CHECK(a.release(0));
  CHECK(hz::serve::pick_next(q, 10, a, need, &off) == 0 && off == 0);  // the head fits now
  q.pop_front();
  CHECK(hz::serve::pick_next(q, 10, a, need, &off) == -1);  // arena full again
  // requests that have not arrived yet are not admitted
  Arena b(8 * 256);
  q = {{6, 256, 100}, {7, 0, 100}};
  CHECK(hz::serve::pick_next(q, 99, b, need, &off) == -1);
  CHECK(hz::serve::pick_next(q, 100, b, need, &off) == 0);
}

int main() {
  arena_basics();
  arena_random();
  admission();
  std::printf("serve_arena_test ok\n");
  return 0;
}

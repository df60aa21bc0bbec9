// Randomised check of the server's HBM arena (csrc/arena.h) against a model
// that tracks every 256-byte granule: blocks never overlap, every allocation
// is the lowest-offset free run that fits (first fit), an allocation fails
// only when no free run fits, and the free list stays fully merged.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "arena.h"

static int fail(const char* what, long long i) {
  std::printf("FAIL %s at op %lld\n", what, i);
  return 1;
}

int main(int argc, char** argv) {
  const unsigned seed = argc > 1 ? (unsigned)std::atoi(argv[1]) : 1u;
  std::mt19937_64 rng(seed);
  const size_t size = (size_t)(1 << 20) + 700;  // not a multiple of 256
  const size_t G = 256, ng = size / G;           // whole granules
  pc::Arena a;
  a.init(nullptr, size);
  std::vector<char> used(ng, 0);
  struct Block { size_t off, n; };
  std::vector<Block> live;
  for (long long i = 0; i < 200000; ++i) {
    const bool do_alloc = live.empty() || (rng() % 100) < 55;
    if (do_alloc) {
      const size_t n = 1 + rng() % (rng() % 8 ? 16384 : 262144);
      const size_t g = (n + G - 1) / G;
      // model: lowest granule run of length g
      size_t want = (size_t)-1, run = 0;
      for (size_t k = 0; k < ng; ++k) {
        run = used[k] ? 0 : run + 1;
        if (run == g) { want = k + 1 - g; break; }
      }
      size_t off = 0;
      const bool ok = a.alloc(n, &off);
      if (ok != (want != (size_t)-1)) return fail("alloc success differs from the model", i);
      if (!ok) continue;
      if (off != want * G) return fail("not the first fit", i);
      for (size_t k = want; k < want + g; ++k) {
        if (used[k]) return fail("overlap", i);
        used[k] = 1;
      }
      live.push_back({off, n});
    } else {
      const size_t j = rng() % live.size();
      const Block b = live[j];
      live[j] = live.back();
      live.pop_back();
      a.release(b.off, b.n);
      for (size_t k = b.off / G; k < (b.off + b.n + G - 1) / G; ++k) used[k] = 0;
    }
    if (i % 97 == 0) {  // the free list: sorted, merged, and the model's free runs
      size_t prev_end = (size_t)-1, free_bytes = 0;
      for (const auto& kv : a.free_) {
        if (kv.first == prev_end) return fail("adjacent free blocks not merged", i);
        prev_end = kv.first + kv.second;
        free_bytes += kv.second;
        for (size_t k = kv.first / G; k < ng && k < (kv.first + kv.second) / G; ++k)
          if (used[k]) return fail("free block covers a live granule", i);
      }
      size_t live_bytes = 0;
      for (const auto& b : live) live_bytes += (b.n + G - 1) / G * G;
      if (free_bytes + live_bytes != size) return fail("bytes lost", i);
    }
  }
  for (const auto& b : live) a.release(b.off, b.n);
  if (a.free_.size() != 1 || a.free_.begin()->first != 0 || a.largest() != size)
    return fail("arena not whole after releasing everything", -1);
  std::printf("ok\n");
  return 0;
}

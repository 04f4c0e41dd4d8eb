// Randomised check of the alignment server's arena bookkeeping
// (paper_2205_07610_gb300/csrc/ga_arena.h), run by tests/test_server_arena.py.
//
// Requests of the serving configuration's length mix (LogNormal, median
// 1000) are admitted and completed in random order, as the scheduler does:
// a request's strip edges from the first-fit arena, then its codes from the
// code slabs, the edges given back when the codes find no room.  Checked:
//   - no two live code ranges and no two live arena ranges overlap;
//   - codes admitted one after another without a new slab are contiguous
//     (what lets one scheduler tick copy them in one transfer);
//   - with nothing in flight every request that fits the arena is admitted;
//   - when everything has completed the whole arena is free again.
// Exit status 0 on success; the first failure is printed.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <random>
#include <vector>

#include "../paper_2205_07610_gb300/csrc/ga_arena.h"

namespace {

struct Live {
  int64_t edge_off, edge_bytes, code_off, code_bytes;
  int slab;
};

bool overlaps(const std::map<int64_t, int64_t> &ranges, int64_t off, int64_t len) {
  auto it = ranges.upper_bound(off);
  if (it != ranges.end() && off + len > it->first) return true;
  if (it != ranges.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second > off) return true;
  }
  return false;
}

int run(int64_t arena_bytes, int steps, uint64_t seed) {
  ga::ArenaAlloc arena(arena_bytes);
  ga::CodeSlabs slabs(arena_bytes);
  std::mt19937_64 rng(seed);
  std::lognormal_distribution<double> len(std::log(1000.0), 1.2);
  std::vector<Live> live;
  std::map<int64_t, int64_t> used;  // every live arena range: edges and codes
  bool have = false, follows = false;  // follows: the last event was an admission
  int64_t seq = 0, edges = 0, last_code_end = -1;
  int last_slab = -1;
  int admitted = 0;
  for (int step = 0; step < steps; ++step) {
    if (!have) {
      const int64_t L = std::min<int64_t>(std::max<int64_t>(100, (int64_t)len(rng)), 20000);
      seq = ((((L + 15) & ~15ll) * 2) + 255) & ~255ll;
      edges = 8 * ((L + 511) / 512 - 1) * (L + 1);
      if (seq + ((edges + 255) & ~255ll) > arena_bytes) continue;  // rejected at submission
      have = true;
    }
    const uint64_t r = rng() % 4;
    bool done = false;
    if (r != 3) {  // try to admit the next request
      int64_t eo = -1;
      bool fail = false, trimmed = false;
      if (edges > 0) {
        eo = arena.alloc(edges);
        if (eo < 0 && (trimmed = slabs.trim(arena))) eo = arena.alloc(edges);
        if (eo < 0) fail = true;
      }
      int slab = -1;
      int64_t so = -1;
      if (!fail) {
        so = slabs.alloc(arena, seq, &slab);
        if (so < 0) {
          if (eo >= 0) arena.release(eo, edges);
          fail = true;
        }
      }
      if (!fail) {
        // codes admitted right after other codes, into the same slab, follow
        // them directly (edges come from the arena, not from the slab)
        if (follows && !trimmed && slab == last_slab && so != last_code_end) {
          std::printf("codes of one slab not contiguous: %lld after %lld\n", (long long)so,
                      (long long)last_code_end);
          return 1;
        }
        if ((eo >= 0 && overlaps(used, eo, (edges + 255) & ~255ll)) || overlaps(used, so, seq)) {
          std::printf("overlapping ranges at step %d\n", step);
          return 1;
        }
        if (eo >= 0) used[eo] = (edges + 255) & ~255ll;
        used[so] = seq;
        live.push_back({eo, edges, so, seq, slab});
        last_code_end = so + seq;
        last_slab = slab;
        follows = true;
        have = false;
        done = true;
        ++admitted;
      } else if (live.empty()) {
        std::printf("a request of %lld + %lld bytes is refused with nothing in flight (arena %lld)\n",
                    (long long)seq, (long long)edges, (long long)arena_bytes);
        return 1;
      }
    }
    if (!done && !live.empty()) {  // complete a random request
      const size_t k = rng() % live.size();
      const Live l = live[k];
      live[k] = live.back();
      live.pop_back();
      used.erase(l.code_off);
      slabs.release(arena, l.slab);
      if (l.edge_off >= 0) {
        used.erase(l.edge_off);
        arena.release(l.edge_off, l.edge_bytes);
      }
      follows = false;  // a completion may leave the slab idle, which restarts it
    }
  }
  for (const Live &l : live) {
    slabs.release(arena, l.slab);
    if (l.edge_off >= 0) arena.release(l.edge_off, l.edge_bytes);
  }
  slabs.trim(arena);
  if (arena.alloc(arena_bytes) != 0) {
    std::printf("arena of %lld bytes not entirely free at the end\n", (long long)arena_bytes);
    return 1;
  }
  if (admitted < steps / 8) {
    std::printf("only %d requests admitted in %d steps\n", admitted, steps);
    return 1;
  }
  std::printf("arena %lld: %d requests admitted, high water %lld\n", (long long)arena_bytes, admitted,
              (long long)arena.high_water());
  return 0;
}

}  // namespace

int main() {
  const int64_t sizes[] = {8ll << 20, 64ll << 20, 256ll << 20, 4ll << 30};
  for (int64_t a : sizes)
    if (run(a, 100000, 20220607u + (uint64_t)(a >> 20))) return 1;
  return 0;
}

// tune_file.h -- the autotuner's choices on disk: {"W,L,pbin": threads, ...}.
// Host code only, no CUDA.  Reading skips anything it cannot parse and every
// CTA size the resident solver could not launch (a damaged or foreign file
// never turns into a failing launch).
#pragma once

#include <cstdio>
#include <map>
#include <tuple>

namespace pc {

using TuneKey = std::tuple<int, int, int>;  // (W, L, p bin)

inline void tune_read(std::FILE* f, int max_threads, std::map<TuneKey, int>& out) {
  int W, L, B, T, ch;
  while ((ch = std::fgetc(f)) != EOF) {
    if (ch != '"') continue;
    if (std::fscanf(f, "%d,%d,%d\": %d", &W, &L, &B, &T) == 4 && T >= 32 && T <= max_threads && T % 32 == 0)
      out[{W, L, B}] = T;
  }
}

inline void tune_write(std::FILE* f, const std::map<TuneKey, int>& m) {
  std::fputs("{", f);
  bool first = true;
  for (const auto& kv : m) {
    std::fprintf(f, "%s\"%d,%d,%d\": %d", first ? "" : ", ", std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), kv.second);
    first = false;
  }
  std::fputs("}\n", f);
}

}  // namespace pc

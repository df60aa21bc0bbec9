// The autotuner's file format (csrc/tune_file.h): what tune_write writes,
// tune_read reads back unchanged; damaged or foreign entries are skipped.
#include <cstdio>
#include <map>

#include "tune_file.h"

int main(int argc, char** argv) {
  if (argc < 2) return 2;
  std::map<pc::TuneKey, int> m{{{4, 16, 6}, 128}, {{8, 64, 7}, 256}, {{32, 2048, 6}, 640}, {{0, 1, 40}, 32}};
  std::FILE* f = std::fopen(argv[1], "w");
  pc::tune_write(f, m);
  std::fclose(f);
  std::map<pc::TuneKey, int> back;
  f = std::fopen(argv[1], "r");
  pc::tune_read(f, 640, back);
  std::fclose(f);
  if (back != m) { std::puts("FAIL round trip"); return 1; }
  // damaged entries: not a multiple of a warp, beyond the solver's limit,
  // zero, negative, truncated, garbage; then one good entry
  f = std::fopen(argv[1], "w");
  std::fputs("{\"1,2,3\": 100, \"1,2,4\": 1024, \"1,2,5\": 0, \"1,2,6\": -64, \"1,2,7\": , "
             "\"x\": 5, \"1,2\": 64, \"9,9,9\": 384}\n", f);
  std::fclose(f);
  std::map<pc::TuneKey, int> d;
  f = std::fopen(argv[1], "r");
  pc::tune_read(f, 640, d);
  std::fclose(f);
  if (d.size() != 1 || d.at({9, 9, 9}) != 384) { std::puts("FAIL damaged entries"); return 1; }
  std::puts("ok");
  return 0;
}

// Tick-by-tick simulation of one streamed-solver slot (csrc/plan.h) for many
// fibre lengths L.  A tick's units run concurrently, so every plan may rely
// only on what earlier ticks finished.  Checked at every step m (sweep of
// layers t <= tmax = min(m, L-1)):
//   * the FP units read layer tmax+1's plane and the degrees of layers <= tmax:
//     F >= min(tmax + 2, L) layers are prepared;
//   * the BITS units update word rows <= tmax/32 from their occupancy:
//     G >= min(32 (tmax/32 + 1), L) layers are drawn;
//   * the preparation of layers [F, F2) needs the occupancy of layer F2
//     (degrees of layer F2 - 1): G >= min(F2 + 1, L); it covers whole word
//     rows: F and F2 multiples of 32, or L;
//   * one draw unit per tick, on the next word row, G a multiple of 32 or L;
//   * F and G never shrink and reach L.
#include <cstdio>

#include "plan.h"

using namespace pc;

static int fail(int L, int m, const char* what) {
  std::printf("FAIL L=%d m=%d: %s\n", L, m, what);
  return 1;
}

static int check(int L) {
  const int TW = (L + 31) / 32;
  Plan p = make_plan(PH_DRAW0, 0, 0, 0, L, TW);
  if (p.lo[U_DRAW] != 0 || p.hi[U_DRAW] < 1 || p.hi[U_DRAW] > TW) return fail(L, 0, "first draw rows");
  if (p.hi[U_CLEAN] != 1) return fail(L, 0, "clean unit");
  int G = p.G2, F = 0;
  if (G != (64 < L ? 64 : L)) return fail(L, 0, "first draw size");
  p = make_plan(PH_PREP0, 0, G, F, L, TW);
  if (p.lo[U_PREP] != 0 || p.hi[U_PREP] != (L < 32 ? L : 32)) return fail(L, 0, "first preparation");
  if (G < (p.hi[U_PREP] + 1 < L ? p.hi[U_PREP] + 1 : L)) return fail(L, 0, "first preparation before draw");
  F = p.F2;
  if (L == 1) return 0;
  for (int m = 1; m <= L + 80; ++m) {
    p = make_plan(PH_STEP, m, G, F, L, TW);
    const int tmax = m < L - 1 ? m : L - 1;
    if (p.lo[U_FP] != 0 || p.hi[U_FP] != tmax + 1) return fail(L, m, "FP window");
    if (p.lo[U_BITS] != 0 || p.hi[U_BITS] != (tmax >> 5) + 1) return fail(L, m, "BITS window");
    if (F < (tmax + 2 < L ? tmax + 2 : L)) return fail(L, m, "sweep reads an unprepared layer");
    const int need_g = 32 * ((tmax >> 5) + 1);
    if (G < (need_g < L ? need_g : L)) return fail(L, m, "bit update reads undrawn occupancy");
    if (p.lo[U_PREP] != F || p.hi[U_PREP] < F || p.hi[U_PREP] > L || p.F2 != p.hi[U_PREP])
      return fail(L, m, "preparation range");
    if (p.hi[U_PREP] > F && G < (p.hi[U_PREP] + 1 < L ? p.hi[U_PREP] + 1 : L))
      return fail(L, m, "degrees before the occupancy they count");
    if (p.hi[U_PREP] != L && p.hi[U_PREP] % 32 != 0) return fail(L, m, "preparation not on a word row");
    if (p.hi[U_DRAW] > p.lo[U_DRAW]) {
      if (p.hi[U_DRAW] != p.lo[U_DRAW] + 1 || p.lo[U_DRAW] != (G >> 5) || p.lo[U_DRAW] >= TW)
        return fail(L, m, "draw row");
      if (G % 32 != 0) return fail(L, m, "draw from a partial row");
    }
    if (p.G2 < G || p.F2 < F || p.G2 > L) return fail(L, m, "G or F shrank or overran");
    if (p.G2 != L && p.G2 % 32 != 0) return fail(L, m, "G not on a word row");
    G = p.G2;
    F = p.F2;
  }
  if (F != L || G != L) return fail(L, L + 80, "preparation did not reach the end of the fibre");
  return 0;
}

int main() {
  int bad = 0;
  for (int L = 1; L <= 400; ++L) bad += check(L);
  const int big[] = {1000, 4095, 4096, 4097, 65535, 100003, 1 << 20, (1 << 24) - 1};
  for (int L : big) bad += check(L);
  if (bad) return 1;
  std::puts("ok");
  return 0;
}

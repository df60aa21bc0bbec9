// plan.h -- the streamed solver's tick planner: which work units one tick of
// a slot runs, from the slot's phase, step m and preparation state.  Shared
// by the device (sweep and control kernels) and host-side checks; no CUDA
// types.
//
// Per slot, G = tube layers whose occupancy is drawn (a multiple of 32, or
// L) and F = layers prepared (degrees, zeroed nu planes, cleaned reached-set
// rows; a multiple of 32, or L).  A tick's units run concurrently, so a plan
// only uses what earlier ticks completed: step m sweeps layers
// t <= min(m, L-1) (Eqs. (3)-(4) move mass one layer per step); the next word
// row (32 layers) is prepared once the window comes within 10 layers of the
// prepared ones, and the occupancy is drawn two word rows ahead of the
// preparation (the degrees of a row count the occupancy of the row after
// it).
#pragma once

#ifdef __CUDACC__
#define PC_PLAN_FN __host__ __device__ inline
#else
#define PC_PLAN_FN inline
#endif

namespace pc {

enum : int { PH_EMPTY = 0, PH_DRAW0 = 1, PH_PREP0 = 2, PH_STEP = 3 };
enum : int { U_FP = 0, U_BITS = 1, U_PREP = 2, U_DRAW = 3, U_CLEAN = 4, U_KINDS = 5 };

// [lo, hi) per unit kind: layers for FP and PREP, word rows for BITS and
// DRAW, one unit row for CLEAN; G2, F2 = G and F once the tick is done
struct Plan {
  int lo[U_KINDS], hi[U_KINDS];
  int G2, F2;
};

PC_PLAN_FN Plan make_plan(int phase, int m, int G, int F, int L, int TW) {
  Plan p;
  for (int k = 0; k < U_KINDS; ++k) { p.lo[k] = 0; p.hi[k] = 0; }
  p.G2 = G; p.F2 = F;
  if (phase == PH_DRAW0) {
    const int rows = TW < 2 ? TW : 2;  // first 64 layers
    p.hi[U_DRAW] = rows;
    p.G2 = rows * 32 < L ? rows * 32 : L;
    // a slot may have held another lattice: zero the padding rows and the
    // sentinel column of this one (one unit per column chunk)
    p.hi[U_CLEAN] = 1;
  } else if (phase == PH_PREP0) {
    p.hi[U_PREP] = L < 32 ? L : 32;  // word row 0
    p.F2 = p.hi[U_PREP];
  } else if (phase == PH_STEP) {
    const int tmax = m < L - 1 ? m : L - 1;
    p.hi[U_FP] = tmax + 1;
    p.hi[U_BITS] = (tmax >> 5) + 1;
    // the next word row of degrees when the window nears the prepared
    // layers; the degrees of layer F2 - 1 need the occupancy of layer F2
    int F2 = F;
    if (F < L && F < tmax + 10 && G >= (F + 33 < L ? F + 33 : L)) F2 = F + 32 < L ? F + 32 : L;
    p.lo[U_PREP] = F; p.hi[U_PREP] = F2;
    p.F2 = F2;
    if (G < L && G < F2 + 64) {  // keep occupancy two word rows ahead
      p.lo[U_DRAW] = G >> 5; p.hi[U_DRAW] = (G >> 5) + 1;
      p.G2 = G + 32 < L ? G + 32 : L;
    }
  }
  return p;
}

}  // namespace pc

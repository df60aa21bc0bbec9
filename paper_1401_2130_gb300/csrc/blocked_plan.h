// blocked_plan.h -- pass planning of the verdict-only blocked solver
// (blocked.cu): the slabs and occupancy rows one pass of 32 steps needs, the
// rows a slab holds, and what the pass's per-step growth / hit masks say
// about the configuration (Sec. II.B: the first step that reaches layer L-1
// gives first_hit, the first step without growth m_stop).  Shared by the
// device and a host-side check; no CUDA types.
#pragma once

#ifdef __CUDACC__
#define PC_BPLAN_FN __host__ __device__ inline
#else
#define PC_BPLAN_FN inline
#endif

namespace pc {

constexpr int kPassSteps = 32;  // steps per pass: one 32-tube word row of halo on each side

enum : int { BP_EMPTY = 0, BP_DRAW0 = 1, BP_STEP = 2 };

// Highest word row that the 32 steps after step m0 can reach (the reached
// set moves at most one tube along the fibre per step, from t = 0).
PC_BPLAN_FN int pass_top_row(int m0, int TW) {
  const int r = (m0 + kPassSteps) >> 5;
  return r < TW - 1 ? r : TW - 1;
}

struct PassItems {
  int tiles;  // slabs of nw valid word rows over rows 0 .. pass_top_row
  int draws;  // occupancy word rows to draw, from row G on
};

// Items of a slot's next pass.  Before the first pass: rows 0 and 1 (what
// the first pass reads).  Then each pass draws the row that the following
// pass reads first, so the occupancy is always drawn up to the top row.
PC_BPLAN_FN PassItems pass_items(int phase, int m0, int G, int TW, int nw) {
  PassItems p{0, 0};
  if (phase == BP_DRAW0) {
    p.draws = TW < 2 ? TW : 2;
  } else if (phase == BP_STEP) {
    p.tiles = (pass_top_row(m0, TW) + 1 + nw - 1) / nw;
    if (G < TW && G <= ((m0 + 2 * kPassSteps) >> 5)) p.draws = 1;
  }
  return p;
}

struct Slab {
  int w0;     // first valid word row; local row i holds word row w0 - 1 + i
  int n_eff;  // local rows computed (the rows above the top row stay empty)
  int ivmax;  // valid local rows 1 .. ivmax
};

PC_BPLAN_FN Slab slab_of(int k, int m0, int TW, int nw, int nrow) {
  Slab s;
  s.w0 = k * nw;
  const int rtop = pass_top_row(m0, TW);
  s.n_eff = nrow < rtop - s.w0 + 2 ? nrow : rtop - s.w0 + 2;
  s.ivmax = nw < s.n_eff - 1 ? nw : s.n_eff - 1;
  return s;
}

struct PassOutcome {
  int finish;     // the configuration is done
  int verdict;    // 1: it percolates
  int first_hit;  // step + 1 of the step that reached layer L - 1, else -1
  int m_stop;     // first_hit, or the first step without growth
};

// The pass of steps m0 + 1 .. m0 + 32: bit j of g = step m0 + 1 + j grew the
// reached set, bit j of h = it reached layer L - 1.  The first step that hit
// or did not grow ends the configuration; a reached set that stopped growing
// stays fixed, so the steps after it cannot change the outcome.
PC_BPLAN_FN PassOutcome pass_outcome(unsigned g, unsigned h, int m0) {
  PassOutcome o{0, 0, -1, 0};
  const unsigned stop = h | ~g;
  if (!stop) return o;
  int j = 0;
  while (!((stop >> j) & 1u)) ++j;
  const int step = m0 + 1 + j;
  o.finish = 1;
  if ((h >> j) & 1u) { o.verdict = 1; o.first_hit = step + 1; o.m_stop = step + 1; }
  else o.m_stop = step;
  return o;
}

}  // namespace pc

// Pass-by-pass simulation of one slot of the verdict-only blocked solver
// (csrc/blocked_plan.h) for many fibre lengths L, slab heights and
// configuration histories.  A history is either "percolates, first reaching
// layer L-1 at step F-1" (F >= L: the reached set advances one layer per
// step at most) or "stops growing at step M".  Checked at every pass of the
// 32 steps after step m0:
//   * every word row a slab reads with live data (rows <= the top row the
//     pass can reach) has its occupancy drawn: G >= top + 1;
//   * one occupancy row drawn per pass at most, never past the fibre;
//   * the slabs' valid rows cover rows 0 .. top exactly once; every slab
//     holds at least one valid row and fits its shared-memory rows;
//   * halo: within 32 steps nothing outside a slab's rows reaches its valid
//     rows -- one full word row (32 tubes) below it unless it starts at row
//     0, and above it one word row or nothing live (its rows end at the top
//     row);
//   * the growth / hit masks of the pass decode to exactly the history's
//     verdict, first_hit and m_stop, in the pass that holds the terminating
//     step and in no earlier one; a hit's row lies at or below the top row;
//   * the pass count is (terminating step - 1) / 32 + 1.
#include <cstdio>
#include <random>

#include "blocked_plan.h"

using namespace pc;

static int fail(int L, int nw, int S, const char* what) {
  std::printf("FAIL L=%d nw=%d S=%d: %s\n", L, nw, S, what);
  return 1;
}

// perc: the configuration percolates with first_hit = S + 1 (its end layer
// is reached at step S), else it stops growing at step S (m_stop = S).
static int run(int L, int nw, bool perc, int S) {
  const int TW = (L + 31) / 32, nrow = nw + 2, endw = (L - 1) >> 5;
  PassItems it = pass_items(BP_DRAW0, 0, 0, TW, nw);
  if (it.tiles != 0 || it.draws != (TW < 2 ? TW : 2)) return fail(L, nw, S, "first draw");
  int G = it.draws, m0 = 0, passes = 0;
  for (;;) {
    it = pass_items(BP_STEP, m0, G, TW, nw);
    const int top = pass_top_row(m0, TW);
    // after step m0 the reached set lies in layers <= m0, after 32 more steps
    // in layers <= m0 + 32: rows above (m0 + 32) / 32 stay empty
    const int reach = (m0 + 32) >> 5 < TW - 1 ? (m0 + 32) >> 5 : TW - 1;
    if (top < reach || top > TW - 1) return fail(L, nw, S, "top row below the reach");
    if (G < top + 1) return fail(L, nw, S, "a slab reads undrawn occupancy");
    if (it.draws < 0 || it.draws > 1 || G + it.draws > TW) return fail(L, nw, S, "draw count");
    // coverage and halo of the slabs
    static int cover[1 << 12];
    for (int r = 0; r <= top; ++r) cover[r] = 0;
    for (int k = 0; k < it.tiles; ++k) {
      const Slab sb = slab_of(k, m0, TW, nw, nrow);
      if (sb.n_eff < 2 || sb.n_eff > nrow || sb.ivmax < 1 || sb.ivmax > nw) return fail(L, nw, S, "slab rows");
      const int lo = sb.w0, hi = sb.w0 + sb.ivmax - 1, last = sb.w0 - 1 + sb.n_eff - 1;
      if (hi > top || last > top) return fail(L, nw, S, "slab past the top row");
      for (int r = lo; r <= hi; ++r) ++cover[r];
      // below: local row 0 (word row w0 - 1) is a full word of halo, or w0 = 0
      // above: a halo row above the valid ones, or the rows end at the top row
      if (!(last >= hi + 1 || last == top)) return fail(L, nw, S, "no halo above the valid rows");
    }
    for (int r = 0; r <= top; ++r)
      if (cover[r] != 1) return fail(L, nw, S, "valid rows do not cover the reachable rows once");
    G += it.draws;
    // the pass's masks from the history
    unsigned g = 0u, h = 0u;
    for (int j = 0; j < 32; ++j) {
      const int step = m0 + 1 + j;
      if (step <= S - (perc ? 0 : 1)) g |= 1u << j;
      if (perc && step == S) h |= 1u << j;
    }
    const PassOutcome o = pass_outcome(g, h, m0);
    ++passes;
    const bool here = S >= m0 + 1 && S <= m0 + 32;
    if (o.finish != (here ? 1 : 0)) return fail(L, nw, S, "finished in the wrong pass");
    if (o.finish) {
      if (perc && (o.verdict != 1 || o.first_hit != S + 1 || o.m_stop != S + 1)) return fail(L, nw, S, "hit outcome");
      if (!perc && (o.verdict != 0 || o.first_hit != -1 || o.m_stop != S)) return fail(L, nw, S, "stop outcome");
      if (perc && endw > top) return fail(L, nw, S, "hit beyond the top row");
      break;
    }
    m0 += 32;
    if (passes > (1 << 20)) return fail(L, nw, S, "no end");
  }
  if (passes != (S - 1) / 32 + 1) return fail(L, nw, S, "pass count");
  return 0;
}

int main() {
  std::mt19937 rng(7);
  const int nws[] = {1, 2, 4, 10, 14, 21, 22, 34};
  int bad = 0;
  for (int L = 2; L <= 4200 && !bad; L += (L < 200 ? 1 : L < 1100 ? 29 : 523)) {
    for (int nw : nws) {
      // percolating: the end layer L-1 is reached at step S >= L - 1
      for (int S : {L - 1, L, L + 31, L + 32, L + 33}) bad |= run(L, nw, true, S);
      // stopping: m_stop = S >= 1
      for (int S : {1, 2, 31, 32, 33, 64, 65, L, L + 1}) bad |= run(L, nw, false, S);
      for (int r = 0; r < 6; ++r) {
        bad |= run(L, nw, true, L - 1 + (int)(rng() % (unsigned)(3 * L + 100)));
        bad |= run(L, nw, false, 1 + (int)(rng() % (unsigned)(3 * L + 100)));
      }
      if (bad) break;
    }
  }
  if (!bad) std::printf("ok\n");
  return bad;
}

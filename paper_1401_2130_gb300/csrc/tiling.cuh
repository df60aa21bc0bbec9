// tiling.cuh -- register-tiled FP32 site update on the padded-row planes
// (layout in lattice.cu), shared by the resident and streamed solvers.
//
// One step of Eq. (3) in forward form at a site j of sublattice s = (q - r)
// mod 3: mu(j) = sum of nu over its 14 neighbours (Sec. II.A):
//   same FCC layer   : (q+1, r+1), (q-2, r+1), (q-1, r-1), (q+2, r-1),
//                      (q-1, r+2), (q+1, r-2)                   at tube t
//   layer above      : (q-1, r+1), (q, r-1), (q+1, r)           at t + [s == 2]
//   layer below      : (q, r+1), (q+1, r-1), (q-1, r)           at t - [s == 0]
//   end contacts     : (q, r)                                   at t - 1, t + 1
// A strip is the 3 plane positions 3s', 3s'+1, 3s'+2, whose sublattices are
// 0, 1, 2.  With q0 the column of its first position, the strip reads, per
// layer, the runs
//   U = row r+1, q0-2 .. q0+3     D = row r-1, q0-1 .. q0+4
//   C = row r,   q0-1 .. q0+3     E = row r+2, q0-1 .. q0+1
//   F = row r-2, q0+1 .. q0+3
// and keeps U, D, C of layers t-1, t, t+1 in registers while it walks up the
// fibre: 23 loads per layer for 3 site updates.
#pragma once

#include "common.cuh"

namespace pc {

struct Runs {
  float U[6], D[6], C[5];
};

__device__ __forceinline__ void load_runs(Runs& R, const float* __restrict__ pl, int u0, int d0, int c0) {
#pragma unroll
  for (int i = 0; i < 6; ++i) R.U[i] = pl[u0 + i];
#pragma unroll
  for (int i = 0; i < 6; ++i) R.D[i] = pl[d0 + i];
#pragma unroll
  for (int i = 0; i < 5; ++i) R.C[i] = pl[c0 + i];
}

// Site updates of layer t for one strip: c = runs of layer t, n = layer t+1;
// (up2, dp2, cp) = the layer t-1 values the sublattice-0 site needs; g0..g2
// the degrees of the three sites.  The 14-term sums are short trees; the
// pairs (U1 + U3, D1 + D3) and (U2 + U4, D2 + D4) are shared by neighbouring
// sites of the strip.
__device__ __forceinline__ void strip_emit_deg(const Runs& c, const Runs& n, float up2, float dp2,
                                               const float (&cp)[4], const float* __restrict__ plc,
                                               int e0, int f0, float* __restrict__ out_pl, int b,
                                               int g0, int g1, int g2,
                                               const float* __restrict__ inv) {
  const float e_0 = plc[e0], e_1 = plc[e0 + 1], e_2 = plc[e0 + 2];
  const float f_0 = plc[f0], f_1 = plc[f0 + 1], f_2 = plc[f0 + 2];
  const float q13 = (c.U[1] + c.U[3]) + (c.D[1] + c.D[3]);  // sites 0 and 1
  const float q24 = (c.U[2] + c.U[4]) + (c.D[2] + c.D[4]);  // sites 1 and 2
  // sublattice 0: layer-below neighbours at t-1, layer-above ones at t
  const float s0 = ((q13 + (c.U[0] + up2)) + ((c.D[0] + dp2) + (c.C[2] + cp[0]))) +
                   ((cp[1] + n.C[1]) + (e_0 + f_0));
  // sublattice 1: all in tube t (end contacts at t +- 1)
  const float s1 = (q13 + q24) + (((c.C[3] + c.C[1]) + (cp[2] + n.C[2])) + (e_1 + f_1));
  // sublattice 2: layer-above neighbours at t+1, layer-below ones at t
  const float s2 = ((q24 + (c.U[5] + n.U[3])) + ((c.D[5] + n.D[3]) + (n.C[4] + c.C[2]))) +
                   ((cp[3] + n.C[3]) + (e_2 + f_2));
  out_pl[b] = inv[g0] * s0;
  out_pl[b + 1] = inv[g1] * s1;
  out_pl[b + 2] = inv[g2] * s2;
}

// As strip_emit_deg, for an output in global memory: out points at the
// strip's first position; the stores bypass L1 (the next step reads the
// plane back through a bulk copy).
__device__ __forceinline__ void strip_emit_deg_global(const Runs& c, const Runs& n, float up2, float dp2,
                                                      const float (&cp)[4], const float* __restrict__ plc,
                                                      int e0, int f0, float* __restrict__ out,
                                                      int g0, int g1, int g2,
                                                      const float* __restrict__ inv) {
  const float e_0 = plc[e0], e_1 = plc[e0 + 1], e_2 = plc[e0 + 2];
  const float f_0 = plc[f0], f_1 = plc[f0 + 1], f_2 = plc[f0 + 2];
  const float q13 = (c.U[1] + c.U[3]) + (c.D[1] + c.D[3]);
  const float q24 = (c.U[2] + c.U[4]) + (c.D[2] + c.D[4]);
  const float s0 = ((q13 + (c.U[0] + up2)) + ((c.D[0] + dp2) + (c.C[2] + cp[0]))) +
                   ((cp[1] + n.C[1]) + (e_0 + f_0));
  const float s1 = (q13 + q24) + (((c.C[3] + c.C[1]) + (cp[2] + n.C[2])) + (e_1 + f_1));
  const float s2 = ((q24 + (c.U[5] + n.U[3])) + ((c.D[5] + n.D[3]) + (n.C[4] + c.C[2]))) +
                   ((cp[3] + n.C[3]) + (e_2 + f_2));
  __stcg(out, inv[g0] * s0);
  __stcg(out + 1, inv[g1] * s1);
  __stcg(out + 2, inv[g2] * s2);
}

// As strip_emit_deg, with the degrees read from the layer's degree plane dgl.
__device__ __forceinline__ void strip_emit(const Runs& c, const Runs& n, float up2, float dp2,
                                           const float (&cp)[4], const float* __restrict__ plc,
                                           int e0, int f0, float* __restrict__ out_pl, int b,
                                           const uint8_t* __restrict__ dgl,
                                           const float* __restrict__ inv) {
  strip_emit_deg(c, n, up2, dp2, cp, plc, e0, f0, out_pl, b, dgl[b], dgl[b + 1], dgl[b + 2], inv);
}

// Layers [t0, t1) of the strip at plane position b.  Layer t of nu is the
// plane at src + (t + 2) * P; degrees of layer t at dg + t * P.  Row offsets:
// oF (r-2), oD (r-1), oU (r+1), oE (r+2).  Positions with degree 0 (zeros of
// the layout, insulating sites) are written 0.
__device__ __forceinline__ void strip_sweep(const float* __restrict__ src, float* __restrict__ dst,
                                            const uint8_t* __restrict__ dg,
                                            const float* __restrict__ inv, int P, int b, int oF,
                                            int oD, int oU, int oE, int t0, int t1) {
  const int u0 = b - 2 + oU, d0 = b - 1 + oD, c0 = b - 1, e0 = b - 1 + oE, f0 = b + 1 + oF;
  const float* pl = src + (size_t)(t0 + 1) * P;  // layer t0 - 1
  float up2 = pl[u0 + 2], dp2 = pl[d0 + 2];
  float cp[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) cp[i] = pl[c0 + i];
  Runs A, B;
  load_runs(A, pl + P, u0, d0, c0);  // layer t0
  int t = t0;
  for (;;) {
    const float* plc = src + (size_t)(t + 2) * P;
    load_runs(B, plc + P, u0, d0, c0);  // layer t + 1
    strip_emit(A, B, up2, dp2, cp, plc, e0, f0, dst + (size_t)(t + 2) * P, b, dg + (size_t)t * P, inv);
    up2 = A.U[2]; dp2 = A.D[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) cp[i] = A.C[i];
    if (++t >= t1) break;
    const float* pld = src + (size_t)(t + 2) * P;
    load_runs(A, pld + P, u0, d0, c0);  // layer t + 1, with the roles swapped
    strip_emit(B, A, up2, dp2, cp, pld, e0, f0, dst + (size_t)(t + 2) * P, b, dg + (size_t)t * P, inv);
    up2 = B.U[2]; dp2 = B.D[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) cp[i] = B.C[i];
    if (++t >= t1) break;
  }
}

}  // namespace pc

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

// Shared-memory loads at a 32-bit shared address plus a compile-time byte
// offset, so that each run costs one address computation and its loads
// take the offset as an immediate.
template <int OFF>
__device__ __forceinline__ float lds_f(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ int lds_u8(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u8 %0, [%1+%2];" : "=r"(v) : "r"(a), "n"(OFF));
  return (int)v;
}

// load_runs at shared addresses u, d, c (bytes) of the runs' first entries
__device__ __forceinline__ void load_runs_s(Runs& R, uint32_t u, uint32_t d, uint32_t c) {
  R.U[0] = lds_f<0>(u); R.U[1] = lds_f<4>(u); R.U[2] = lds_f<8>(u);
  R.U[3] = lds_f<12>(u); R.U[4] = lds_f<16>(u); R.U[5] = lds_f<20>(u);
  R.D[0] = lds_f<0>(d); R.D[1] = lds_f<4>(d); R.D[2] = lds_f<8>(d);
  R.D[3] = lds_f<12>(d); R.D[4] = lds_f<16>(d); R.D[5] = lds_f<20>(d);
  R.C[0] = lds_f<0>(c); R.C[1] = lds_f<4>(c); R.C[2] = lds_f<8>(c);
  R.C[3] = lds_f<12>(c); R.C[4] = lds_f<16>(c);
}

// strip_emit_deg_global with the E and F runs at shared addresses e, f and
// the three degrees at shared address g; inv at shared address iv.
__device__ __forceinline__ void strip_emit_s(const Runs& c, const Runs& n, float up2, float dp2,
                                             const float (&cp)[4], uint32_t e, uint32_t f, uint32_t g,
                                             uint32_t iv, float* __restrict__ out) {
  const float e_0 = lds_f<0>(e), e_1 = lds_f<4>(e), e_2 = lds_f<8>(e);
  const float f_0 = lds_f<0>(f), f_1 = lds_f<4>(f), f_2 = lds_f<8>(f);
  const int g0 = lds_u8<0>(g), g1 = lds_u8<1>(g), g2 = lds_u8<2>(g);
  const float q13 = (c.U[1] + c.U[3]) + (c.D[1] + c.D[3]);
  const float q24 = (c.U[2] + c.U[4]) + (c.D[2] + c.D[4]);
  const float s0 = ((q13 + (c.U[0] + up2)) + ((c.D[0] + dp2) + (c.C[2] + cp[0]))) +
                   ((cp[1] + n.C[1]) + (e_0 + f_0));
  const float s1 = (q13 + q24) + (((c.C[3] + c.C[1]) + (cp[2] + n.C[2])) + (e_1 + f_1));
  const float s2 = ((q24 + (c.U[5] + n.U[3])) + ((c.D[5] + n.D[3]) + (n.C[4] + c.C[2]))) +
                   ((cp[3] + n.C[3]) + (e_2 + f_2));
  __stcg(out, lds_f<0>(iv + 4u * (uint32_t)g0) * s0);
  __stcg(out + 1, lds_f<0>(iv + 4u * (uint32_t)g1) * s1);
  __stcg(out + 2, lds_f<0>(iv + 4u * (uint32_t)g2) * s2);
}

template <int OFF>
__device__ __forceinline__ void lds_v2(uint32_t a, float& x, float& y) {
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(x), "=f"(y) : "r"(a), "n"(OFF));
}
template <int OFF>
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
  uint16_t v;
  asm volatile("ld.shared.u16 %0, [%1+%2];" : "=h"(v) : "r"(a), "n"(OFF));
  return v;
}

// The three 14-term sums of one strip (sublattices 0, 1, 2) from its runs:
// U, D, C of layer t (U[0..5], D[0..5], C[0..4]), the layer t-1 values
// (up2, dp2, cp[0..3]), the layer t+1 values (nU3, nD3, nC[1..4]) and the
// E, F runs of layer t.  The addition trees are those of strip_emit_deg.
__device__ __forceinline__ void strip_sums(const float* U, const float* D, const float* C, float up2,
                                           float dp2, const float* cp, float nU3, float nD3,
                                           const float* nC, const float* E, const float* F, float& s0,
                                           float& s1, float& s2) {
  const float q13 = (U[1] + U[3]) + (D[1] + D[3]);  // sites 0 and 1
  const float q24 = (U[2] + U[4]) + (D[2] + D[4]);  // sites 1 and 2
  s0 = ((q13 + (U[0] + up2)) + ((D[0] + dp2) + (C[2] + cp[0]))) + ((cp[1] + nC[1]) + (E[0] + F[0]));
  s1 = (q13 + q24) + (((C[3] + C[1]) + (cp[2] + nC[2])) + (E[1] + F[1]));
  s2 = ((q24 + (U[5] + nU3)) + ((D[5] + nD3) + (nC[4] + C[2]))) + ((cp[3] + nC[3]) + (E[2] + F[2]));
}

// Runs of a strip pair (positions b .. b+5, b = 6h) in one layer of the
// paired layout: u[i] = row r+1 at b-2+i, d[i] = row r-1 at b-1+i (i < 9),
// c[i] = row r at b-1+i (i < 8).  Strip j of the pair (j = 0, 1) has its
// U, D, C runs at u + 3j, d + 3j, c + 3j.
struct PairRuns {
  float u[9], d[9], c[8];
};

// Loads at shared byte addresses u, d, c of the row r+1, r-1 and r entries
// at position b - 2 (8-byte aligned: every row offset of the paired layout
// is even): five 64-bit loads per run, one entry of each discarded.
__device__ __forceinline__ void load_pair_runs(PairRuns& R, uint32_t u, uint32_t d, uint32_t c) {
  float x;
  lds_v2<0>(u, R.u[0], R.u[1]); lds_v2<8>(u, R.u[2], R.u[3]); lds_v2<16>(u, R.u[4], R.u[5]);
  lds_v2<24>(u, R.u[6], R.u[7]); lds_v2<32>(u, R.u[8], x);
  lds_v2<0>(d, x, R.d[0]); lds_v2<8>(d, R.d[1], R.d[2]); lds_v2<16>(d, R.d[3], R.d[4]);
  lds_v2<24>(d, R.d[5], R.d[6]); lds_v2<32>(d, R.d[7], R.d[8]);
  lds_v2<0>(c, x, R.c[0]); lds_v2<8>(c, R.c[1], R.c[2]); lds_v2<16>(c, R.c[3], R.c[4]);
  lds_v2<24>(c, R.c[5], R.c[6]); lds_v2<32>(c, R.c[7], x);
}

// Layer t of a strip pair: c = runs of layer t, n = of layer t+1; pu, pd,
// pc = the layer t-1 values (pu[j] = U[2], pd[j] = D[2] of strip j,
// pc[0..6] = c[0..6]); e, f = shared byte addresses of the row r+2 entry at
// b - 2 and the row r-2 entry at b; g = shared byte address of the six
// degree bytes at b (2-byte aligned); iv = the 1/deg table.  Writes the six
// values to out[0..5] (global, 8-byte aligned; bypasses L1).
__device__ __forceinline__ void pair_emit(const PairRuns& c, const PairRuns& n, const float (&pu)[2],
                                          const float (&pd)[2], const float (&pc)[7], uint32_t e,
                                          uint32_t f, uint32_t g, uint32_t iv, float* __restrict__ out) {
  float E[8], F[8];
  lds_v2<0>(e, E[0], E[1]); lds_v2<8>(e, E[2], E[3]); lds_v2<16>(e, E[4], E[5]); lds_v2<24>(e, E[6], E[7]);
  lds_v2<0>(f, F[0], F[1]); lds_v2<8>(f, F[2], F[3]); lds_v2<16>(f, F[4], F[5]); lds_v2<24>(f, F[6], F[7]);
  const uint32_t g01 = lds_u16<0>(g), g23 = lds_u16<2>(g), g45 = lds_u16<4>(g);
  float a0, a1, a2, b0, b1, b2;
  strip_sums(c.u, c.d, c.c, pu[0], pd[0], pc, n.u[3], n.d[3], n.c, E + 1, F + 1, a0, a1, a2);
  strip_sums(c.u + 3, c.d + 3, c.c + 3, pu[1], pd[1], pc + 3, n.u[6], n.d[6], n.c + 3, E + 4, F + 4,
             b0, b1, b2);
  const float i0 = lds_f<0>(iv + 4u * (g01 & 0xffu)), i1 = lds_f<0>(iv + 4u * (g01 >> 8));
  const float i2 = lds_f<0>(iv + 4u * (g23 & 0xffu)), i3 = lds_f<0>(iv + 4u * (g23 >> 8));
  const float i4 = lds_f<0>(iv + 4u * (g45 & 0xffu)), i5 = lds_f<0>(iv + 4u * (g45 >> 8));
  __stcg(reinterpret_cast<float2*>(out), make_float2(i0 * a0, i1 * a1));
  __stcg(reinterpret_cast<float2*>(out) + 1, make_float2(i2 * a2, i3 * b0));
  __stcg(reinterpret_cast<float2*>(out) + 2, make_float2(i4 * b1, i5 * b2));
}

// strip_emit_s with the output in shared memory (the resident solver)
__device__ __forceinline__ void strip_emit_s_shared(const Runs& c, const Runs& n, float up2, float dp2,
                                                    const float (&cp)[4], uint32_t e, uint32_t f, uint32_t g,
                                                    uint32_t iv, float* __restrict__ out) {
  const float e_0 = lds_f<0>(e), e_1 = lds_f<4>(e), e_2 = lds_f<8>(e);
  const float f_0 = lds_f<0>(f), f_1 = lds_f<4>(f), f_2 = lds_f<8>(f);
  const int g0 = lds_u8<0>(g), g1 = lds_u8<1>(g), g2 = lds_u8<2>(g);
  const float q13 = (c.U[1] + c.U[3]) + (c.D[1] + c.D[3]);
  const float q24 = (c.U[2] + c.U[4]) + (c.D[2] + c.D[4]);
  const float s0 = ((q13 + (c.U[0] + up2)) + ((c.D[0] + dp2) + (c.C[2] + cp[0]))) +
                   ((cp[1] + n.C[1]) + (e_0 + f_0));
  const float s1 = (q13 + q24) + (((c.C[3] + c.C[1]) + (cp[2] + n.C[2])) + (e_1 + f_1));
  const float s2 = ((q24 + (c.U[5] + n.U[3])) + ((c.D[5] + n.D[3]) + (n.C[4] + c.C[2]))) +
                   ((cp[3] + n.C[3]) + (e_2 + f_2));
  out[0] = lds_f<0>(iv + 4u * (uint32_t)g0) * s0;
  out[1] = lds_f<0>(iv + 4u * (uint32_t)g1) * s1;
  out[2] = lds_f<0>(iv + 4u * (uint32_t)g2) * s2;
}

// strip_sweep (below) on planes in shared memory at explicit shared
// addresses: src_s, dg_s and inv_s are the shared byte addresses of the nu
// planes, the degree planes and the 1/deg table; dst is the output planes.
__device__ __forceinline__ void strip_sweep_s(uint32_t src_s, float* __restrict__ dst, uint32_t dg_s,
                                              uint32_t inv_s, int P, int b, int oF, int oD, int oU,
                                              int oE, int t0, int t1) {
  const uint32_t P4 = 4u * (uint32_t)P;
  const uint32_t u0 = (uint32_t)(4 * (b - 2 + oU)), d0 = (uint32_t)(4 * (b - 1 + oD));
  const uint32_t c0 = (uint32_t)(4 * (b - 1)), e0 = (uint32_t)(4 * (b - 1 + oE));
  const uint32_t f0 = (uint32_t)(4 * (b + 1 + oF));
  uint32_t pl = src_s + (uint32_t)(t0 + 1) * P4;  // layer t0 - 1
  float up2 = lds_f<8>(pl + u0), dp2 = lds_f<8>(pl + d0);
  float cp[4];
  cp[0] = lds_f<0>(pl + c0); cp[1] = lds_f<4>(pl + c0); cp[2] = lds_f<8>(pl + c0); cp[3] = lds_f<12>(pl + c0);
  Runs A, B;
  pl += P4;  // layer t0
  load_runs_s(A, pl + u0, pl + d0, pl + c0);
  uint32_t g = dg_s + (uint32_t)(t0 * P + b);
  float* out = dst + (size_t)(t0 + 2) * P + b;
  int t = t0;
  for (;;) {
    uint32_t pn = pl + P4;  // layer t + 1
    load_runs_s(B, pn + u0, pn + d0, pn + c0);
    strip_emit_s_shared(A, B, up2, dp2, cp, pl + e0, pl + f0, g, inv_s, out);
    up2 = A.U[2]; dp2 = A.D[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) cp[i] = A.C[i];
    pl = pn; g += (uint32_t)P; out += P;
    if (++t >= t1) break;
    pn = pl + P4;
    load_runs_s(A, pn + u0, pn + d0, pn + c0);  // roles swapped
    strip_emit_s_shared(B, A, up2, dp2, cp, pl + e0, pl + f0, g, inv_s, out);
    up2 = B.U[2]; dp2 = B.D[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) cp[i] = B.C[i];
    pl = pn; g += (uint32_t)P; out += P;
    if (++t >= t1) break;
  }
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

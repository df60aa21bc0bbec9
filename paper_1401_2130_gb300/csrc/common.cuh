// common.cuh -- device and host pieces shared by the libpercol kernels.
//
// Lattice of Sec. II.A (Fig. 1): columns (q, r) of a hexagon of radius W in
// axial coordinates, sublattice sigma = (q - r) mod 3 (the A, B, C layers of
// Fig. 1(b)), FCC layer height h = 3t + sigma.  Every site has 12 side
// contacts -- the FCC nearest neighbours: 6 in its own (111) layer, 3 in the
// layer above and 3 below -- and 2 end contacts (same column, t +- 1).
// The 12 side contacts as column offsets, with the tube-index shift they
// imply (a step of one layer up from sigma = 2 enters the next tube period):
//   d = 0..5   same layer : (1,1) (2,-1) (1,-2) (-1,-1) (-2,1) (-1,2), dt = 0
//   d = 6..8   layer up   : (1,0) (-1,1) (0,-1),            dt = [sigma == 2]
//   d = 9..11  layer down : (-1,0) (1,-1) (0,1),            dt = -[sigma == 0]
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/percol.h"

namespace pc {

constexpr int kLateral = 12;

__host__ __device__ constexpr int dir_dq(int d) {
  return d == 0 ? 1 : d == 1 ? 2 : d == 2 ? 1 : d == 3 ? -1 : d == 4 ? -2 : d == 5 ? -1
       : d == 6 ? 1 : d == 7 ? -1 : d == 8 ? 0 : d == 9 ? -1 : d == 10 ? 1 : 0;
}
__host__ __device__ constexpr int dir_dr(int d) {
  return d == 0 ? 1 : d == 1 ? -1 : d == 2 ? -2 : d == 3 ? -1 : d == 4 ? 1 : d == 5 ? 2
       : d == 6 ? 0 : d == 7 ? 1 : d == 8 ? -1 : d == 9 ? 0 : d == 10 ? -1 : 1;
}
// tube-index shift of direction d for a column of sublattice sigma
__host__ __device__ inline int dir_dt(int d, int sigma) {
  return d < 6 ? 0 : d < 9 ? (sigma == 2 ? 1 : 0) : (sigma == 0 ? -1 : 0);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (J. K. Salmon et al., "Parallel Random Numbers: As Easy as
// 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplications whose high
// halves are xored with the other two words and the round key; the key is
// bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct u32x4 { uint32_t x, y, z, w; };

__host__ __device__ inline u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
  for (int i = 0; i < 10; ++i) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    u32x4 n;
    n.x = (uint32_t)(p1 >> 32) ^ c.y ^ k0;
    n.y = (uint32_t)p1;
    n.z = (uint32_t)(p0 >> 32) ^ c.w ^ k1;
    n.w = (uint32_t)p0;
    c = n;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Occupancy stream of one configuration: word j (j = 0..3) of the block for
// counter (block, config, W | L << 8, 0) decides site 4*block + j.
struct OccStream {
  uint32_t k0, k1, cfg, wl;
  uint64_t T;  // threshold floor(p * 2^32); 2^32 = every site metallic
  __device__ inline uint32_t block_bits(uint32_t block) const {
    const u32x4 r = philox4x32_10(u32x4{block, cfg, wl, 0u}, k0, k1);
    return (uint32_t)((uint64_t)r.x < T) | ((uint32_t)((uint64_t)r.y < T) << 1) |
           ((uint32_t)((uint64_t)r.z < T) << 2) | ((uint32_t)((uint64_t)r.w < T) << 3);
  }
};

inline uint64_t threshold_of(double p) {
  // p * 2^32 is exact in double; floor gives the integer threshold
  double v = p * 4294967296.0;
  return (uint64_t)v;  // p >= 0, truncation == floor
}

// ---------------------------------------------------------------------------
// Lattice description handed to kernels (all device pointers).
// ---------------------------------------------------------------------------
struct Lattice {
  int W, L;
  int A;         // columns
  int64_t N;     // sites
  int S;         // row stride of per-layer float arrays: A + 1 (column A is an always-zero sentinel)
  int TW;        // 32-bit words per column for bit arrays along t: ceil(L / 32)
  int TWP;       // TW + 2: one zero padding word before and after
  const int32_t* nbr;   // [A][12] neighbour column or A (sentinel) if outside the hexagon
  const int8_t* sigma;  // [A]
  // Padded-row plane layout of per-layer FP arrays (see lattice.cu):
  int P;                // entries per plane
  int s_begin;          // first strip: strip s covers plane positions 3s, 3s+1, 3s+2
  int n_strips;
  const int16_t* strip_row;  // [n_strips] hexagon row (0..2W) of each strip
  const int32_t* row_off;    // [2W+1][4] offsets to rows r-2, r-1, r+1, r+2
  const int32_t* ppos;       // [A] plane position of each column
  const int32_t* pcol;       // [P] column at each plane position, -1 for zeros
  // the paired layout of the streamed solver (same fields; see lattice.cu)
  int P2, s_begin2, n_strips2;
  const int16_t* strip_row2;
  const int32_t* row_off2;
  const int32_t* ppos2;
  const int32_t* pcol2;
};

// The lattice as the streamed solver sees it: its paired plane layout in
// place of the compact one.
inline Lattice stream_view(const Lattice& l) {
  Lattice v = l;
  v.P = l.P2; v.s_begin = l.s_begin2; v.n_strips = l.n_strips2;
  v.strip_row = l.strip_row2; v.row_off = l.row_off2; v.ppos = l.ppos2; v.pcol = l.pcol2;
  return v;
}

// Host-side padded-row layout of one W (lattice.cu).
struct PlaneLayout {
  int P = 0, s_begin = 0, n_strips = 0;
  std::vector<int16_t> strip_row;
  std::vector<int32_t> row_off, ppos, pcol;
};
PlaneLayout make_layout(int W, bool paired = false);
// largest bulk-copy segment (entries, a multiple of 16) that a chunk of
// `pairs` strip pairs reads in one plane of the paired layout
int max_pair_segment(int W, int pairs);

// Plane positions [lo, hi) read by the strip at position b whose row has the
// offsets ro[0..3] (rows r-2, r-1, r+1, r+2): the runs of tiling.cuh.
__host__ __device__ inline void strip_span(int b, const int32_t* ro, int* lo, int* hi) {
  const int f0 = b + 1 + ro[0], d0 = b - 1 + ro[1], u0 = b - 2 + ro[2], e0 = b - 1 + ro[3], c0 = b - 1;
  int l = c0, h = c0 + 5;
  l = l < f0 ? l : f0; h = h > f0 + 3 ? h : f0 + 3;
  l = l < d0 ? l : d0; h = h > d0 + 6 ? h : d0 + 6;
  l = l < u0 ? l : u0; h = h > u0 + 6 ? h : u0 + 6;
  l = l < e0 ? l : e0; h = h > e0 + 3 ? h : e0 + 3;
  *lo = l; *hi = h;
}
void layout_fill(int W, int* P, int* s_begin, int* n_strips, int16_t* strip_row, int32_t* row_off,
                 int32_t* ppos, int32_t* pcol, bool paired = false);

// Plane positions [lo, hi) read by the strip pair at plane position b (= 6h,
// paired layout) whose row has the offsets ro[0..3] (rows r-2, r-1, r+1,
// r+2), with the 64-bit loads of the streamed sweep.
__host__ __device__ inline void pair_span(int b, const int32_t* ro, int* lo, int* hi) {
  const int fl = b + ro[0], dl = b - 2 + ro[1], ul = b - 2 + ro[2], el = b - 2 + ro[3], cl = b - 2;
  int l = cl, h = cl + 10;
  l = l < fl ? l : fl; h = h > fl + 8 ? h : fl + 8;
  l = l < dl ? l : dl; h = h > dl + 10 ? h : dl + 10;
  l = l < ul ? l : ul; h = h > ul + 10 ? h : ul + 10;
  l = l < el ? l : el; h = h > el + 8 ? h : el + 8;
  *lo = l; *hi = h;
}

// NVTX range over a host call (profilers group the call's launches under it)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// error reporting (thread-local message), defined in api.cu
void set_error(const std::string& msg);
pc_status cuda_fail(cudaError_t e, const char* what);

#define PC_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return pc::cuda_fail(e_, #call); \
  } while (0)

// Host-side lattice cache (lattice.cu).  Returns device tables for (W, L) on
// the current device; built once and kept until pc_shutdown().
pc_status get_lattice(int W, int L, Lattice* out);
void release_lattices();

int64_t n_columns(int W);

}  // namespace pc

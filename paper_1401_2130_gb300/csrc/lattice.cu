// lattice.cu -- per-W column tables of the fibre lattice (Sec. II.A, Fig. 1),
// built on the host once per device and cached.
//
// Column order: row-major over r = -W..W, q ascending within a row, keeping
// (q, r) with max(|q|, |r|, |q + r|) <= W.  For each column the table holds
// its 12 side-contact neighbour columns in the direction order of common.cuh
// (the sentinel value A marks a neighbour outside the hexagon) and its
// sublattice sigma = (q - r) mod 3.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace pc {

int64_t n_columns(int W) { return 3ll * W * (W + 1) + 1; }

// Padded-row plane layout of one tube layer (the FP arrays nu and deg).
// A zero zone of W + 8 entries opens the plane and stands for the rows -W-2,
// -W-1 outside the hexagon; rows r = -W..W follow in order, each preceded by
// 2 to 4 zeros chosen so that plane position mod 3 equals the sublattice
// (q - r) mod 3 of the column stored there; a second zero zone closes the
// plane and stands for the rows W+1, W+2.  Every neighbour of a column in
// rows r-2..r+2 then sits at a fixed offset from the column's own position
// -- position(q, r') = base(r') + q -- and inside the same plane.  P is a
// multiple of 16, so that every plane of the FP32 array and of the byte
// degree array starts on a 16-byte boundary (bulk copies).  Strips are
// triples of positions 3s, 3s+1, 3s+2 (sublattice 0, 1, 2); zero positions
// have degree 0, so a strip may cover zeros and simply writes zeros there.
// Fills the layout of radius W into caller buffers (any may be null) and
// returns P, s_begin, n_strips.  No allocation: usable from every entry point.
void layout_fill(int W, int* P_out, int* s_begin_out, int* n_strips_out, int16_t* strip_row,
                 int32_t* row_off, int32_t* ppos, int32_t* pcol) {
  const int nr = 2 * W + 1;  // W <= 255: at most 511 rows
  int start[511];
  auto qlo = [W](int ri) { const int r = ri - W; return r < 0 ? -W - r : -W; };
  auto len = [W](int ri) { const int r = ri - W; return 2 * W + 1 - (r < 0 ? -r : r); };
  const int Z = W + 8;
  int pos = Z;  // top zone [0, Z)
  for (int ri = 0; ri < nr; ++ri) {
    const int r = ri - W;
    const int want = ((qlo(ri) - r) % 3 + 3) % 3;
    int x = pos + 2;
    while (x % 3 != want) ++x;
    start[ri] = x;
    pos = x + len(ri);
  }
  const int zone = pos;                      // bottom zone [zone, zone + Z)
  const int P = (zone + Z + 15) & ~15;
  // base(row) = position(q, row) - q, for rows -W-2 .. W+2 (index ri + 2)
  auto base = [&](int ri_ext) -> int {
    if (ri_ext <= 1) return 3;                  // rows -W-2, -W-1: q in [-3, W+4]
    if (ri_ext >= nr + 2) return zone + W + 4;  // rows W+1, W+2: q in [-W-4, 3]
    return start[ri_ext - 2] - qlo(ri_ext - 2);
  };
  const int sb = start[0] / 3, se = (start[nr - 1] + len(nr - 1) + 2) / 3;
  if (P_out) *P_out = P;
  if (s_begin_out) *s_begin_out = sb;
  if (n_strips_out) *n_strips_out = se - sb;
  if (row_off) {
    const int dr[4] = {-2, -1, 1, 2};
    for (int ri = 0; ri < nr; ++ri)
      for (int k = 0; k < 4; ++k) row_off[ri * 4 + k] = base(ri + 2 + dr[k]) - base(ri + 2);
  }
  if (pcol) for (int k = 0; k < P; ++k) pcol[k] = -1;
  int a = 0;
  for (int ri = 0; ri < nr; ++ri)
    for (int j = 0; j < len(ri); ++j, ++a) {
      if (ppos) ppos[a] = start[ri] + j;
      if (pcol) pcol[start[ri] + j] = a;
    }
  if (strip_row) {
    // the row holding one of the strip's positions, else the row before it
    int ri = 0;
    for (int st = 0; st < se - sb; ++st) {
      const int p0 = 3 * (sb + st);
      while (ri + 1 < nr && start[ri + 1] <= p0 + 2) ++ri;
      strip_row[st] = (int16_t)ri;
    }
  }
}

// Plane positions [lo, hi) that the strips [k0, k1) read in one plane, for
// every chunk of `chunk` strips; returns the largest hi - lo (aligned to 16).
int max_segment(int W, int chunk) {
  const PlaneLayout L = make_layout(W);
  int best = 0;
  for (int k0 = 0; k0 < L.n_strips; k0 += chunk) {
    const int k1 = std::min(k0 + chunk, L.n_strips);
    int lo = 1 << 30, hi = -(1 << 30);
    for (int k = k0; k < k1; ++k) {
      int sl, sh;
      strip_span(3 * (L.s_begin + k), &L.row_off[4 * L.strip_row[k]], &sl, &sh);
      lo = std::min(lo, sl); hi = std::max(hi, sh);
    }
    lo &= ~15;
    hi = (hi + 15) & ~15;
    best = std::max(best, hi - lo);
  }
  return best;
}

PlaneLayout make_layout(int W) {
  PlaneLayout L;
  layout_fill(W, &L.P, &L.s_begin, &L.n_strips, nullptr, nullptr, nullptr, nullptr);
  L.strip_row.resize(L.n_strips);
  L.row_off.resize((size_t)(2 * W + 1) * 4);
  L.ppos.resize(n_columns(W));
  L.pcol.resize(L.P);
  layout_fill(W, nullptr, nullptr, nullptr, L.strip_row.data(), L.row_off.data(), L.ppos.data(),
              L.pcol.data());
  return L;
}

namespace {

struct Entry {
  int32_t* nbr = nullptr;
  int8_t* sigma = nullptr;
  int A = 0;
  int P = 0, s_begin = 0, n_strips = 0;
  int16_t* strip_row = nullptr;
  int32_t* row_off = nullptr;
  int32_t* ppos = nullptr;
  int32_t* pcol = nullptr;
};

std::mutex g_mu;
std::map<std::pair<int, int>, Entry> g_cache;  // (device, W) -> tables

int col_index(int W, int q, int r, const std::vector<int>& row_start) {
  if (r < -W || r > W) return -1;
  const int qlo = r < 0 ? -W - r : -W;
  const int qhi = r < 0 ? W : W - r;
  if (q < qlo || q > qhi) return -1;
  return row_start[r + W] + (q - qlo);
}

}  // namespace

pc_status get_lattice(int W, int L, Lattice* out) {
  int dev = 0;
  PC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  auto key = std::make_pair(dev, W);
  auto it = g_cache.find(key);
  if (it == g_cache.end()) {
    const int A = (int)n_columns(W);
    std::vector<int> row_start(2 * W + 1);
    std::vector<int> cq, cr;
    int a = 0;
    for (int r = -W; r <= W; ++r) {
      row_start[r + W] = a;
      const int qlo = r < 0 ? -W - r : -W;
      const int qhi = r < 0 ? W : W - r;
      for (int q = qlo; q <= qhi; ++q, ++a) { cq.push_back(q); cr.push_back(r); }
    }
    std::vector<int32_t> nbr((size_t)A * kLateral);
    std::vector<int8_t> sig(A);
    for (int c = 0; c < A; ++c) {
      sig[c] = (int8_t)(((cq[c] - cr[c]) % 3 + 3) % 3);
      for (int d = 0; d < kLateral; ++d) {
        const int j = col_index(W, cq[c] + dir_dq(d), cr[c] + dir_dr(d), row_start);
        nbr[(size_t)c * kLateral + d] = j < 0 ? A : j;
      }
    }
    Entry e;
    e.A = A;
    const PlaneLayout lay = make_layout(W);
    e.P = lay.P; e.s_begin = lay.s_begin; e.n_strips = lay.n_strips;
    PC_CUDA(cudaMalloc(&e.strip_row, sizeof(int16_t) * lay.strip_row.size()));
    PC_CUDA(cudaMalloc(&e.row_off, sizeof(int32_t) * lay.row_off.size()));
    PC_CUDA(cudaMalloc(&e.ppos, sizeof(int32_t) * lay.ppos.size()));
    PC_CUDA(cudaMalloc(&e.pcol, sizeof(int32_t) * lay.pcol.size()));
    PC_CUDA(cudaMemcpy(e.strip_row, lay.strip_row.data(), sizeof(int16_t) * lay.strip_row.size(), cudaMemcpyHostToDevice));
    PC_CUDA(cudaMemcpy(e.row_off, lay.row_off.data(), sizeof(int32_t) * lay.row_off.size(), cudaMemcpyHostToDevice));
    PC_CUDA(cudaMemcpy(e.ppos, lay.ppos.data(), sizeof(int32_t) * lay.ppos.size(), cudaMemcpyHostToDevice));
    PC_CUDA(cudaMemcpy(e.pcol, lay.pcol.data(), sizeof(int32_t) * lay.pcol.size(), cudaMemcpyHostToDevice));
    PC_CUDA(cudaMalloc(&e.nbr, nbr.size() * sizeof(int32_t)));
    PC_CUDA(cudaMalloc(&e.sigma, sig.size()));
    PC_CUDA(cudaMemcpy(e.nbr, nbr.data(), nbr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    PC_CUDA(cudaMemcpy(e.sigma, sig.data(), sig.size(), cudaMemcpyHostToDevice));
    it = g_cache.emplace(key, e).first;
  }
  const Entry& e = it->second;
  out->W = W;
  out->L = L;
  out->A = e.A;
  out->N = (int64_t)e.A * L;
  out->S = e.A + 1;
  out->TW = (L + 31) / 32;
  out->TWP = out->TW + 2;
  out->nbr = e.nbr;
  out->sigma = e.sigma;
  out->P = e.P; out->s_begin = e.s_begin; out->n_strips = e.n_strips;
  out->strip_row = e.strip_row; out->row_off = e.row_off; out->ppos = e.ppos; out->pcol = e.pcol;
  return PC_OK;
}

void release_lattices() {
  std::lock_guard<std::mutex> lk(g_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto& kv : g_cache) {
    cudaSetDevice(kv.first.first);
    cudaFree(kv.second.nbr);
    cudaFree(kv.second.sigma);
    cudaFree(kv.second.strip_row);
    cudaFree(kv.second.row_off);
    cudaFree(kv.second.ppos);
    cudaFree(kv.second.pcol);
  }
  cudaSetDevice(cur);
  g_cache.clear();
}

}  // namespace pc

// Host-side copy of the plane layout of radius W (diagnostics and tests).
extern "C" pc_status pc_lattice_layout(int32_t W, int32_t* P, int32_t* s_begin, int32_t* n_strips,
                                       int16_t* strip_row, int32_t* row_off, int32_t* ppos,
                                       int32_t* pcol) {
  if (W < 0 || W > 255) { pc::set_error("pc_lattice_layout: W must be in [0, 255]"); return PC_ERR_ARG; }
  const pc::PlaneLayout L = pc::make_layout(W);
  if (P) *P = L.P;
  if (s_begin) *s_begin = L.s_begin;
  if (n_strips) *n_strips = L.n_strips;
  if (strip_row) std::copy(L.strip_row.begin(), L.strip_row.end(), strip_row);
  if (row_off) std::copy(L.row_off.begin(), L.row_off.end(), row_off);
  if (ppos) std::copy(L.ppos.begin(), L.ppos.end(), ppos);
  if (pcol) std::copy(L.pcol.begin(), L.pcol.end(), pcol);
  return PC_OK;
}

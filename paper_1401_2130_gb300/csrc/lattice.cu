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

// Padded-row plane layouts of one tube layer (the FP arrays nu and deg).
// A zero zone opens the plane and stands for the rows -W-2, -W-1 outside the
// hexagon; rows r = -W..W follow in order, each preceded by at least 2
// zeros and placed so that plane position mod 3 equals the sublattice
// (q - r) mod 3 of the column stored there: a strip (positions 3s, 3s+1,
// 3s+2) then holds sublattices 0, 1, 2.  A second zero zone closes the plane
// and stands for the rows W+1, W+2.  Every neighbour of a column in rows
// r-2..r+2 sits at a fixed offset from the column's own position --
// position(q, r') = base(r') + q -- and inside the same plane.  P is a
// multiple of 16, so that every plane of the FP32 array and of the byte
// degree array starts on a 16-byte boundary (bulk copies).  Zero positions
// have degree 0, so a strip may cover zeros and simply writes zeros there.
//
// Two variants:
//   compact (resident solver): 2 to 4 zeros before each row, zones of W + 8;
//   paired (streamed solver): in addition base(r) is even for every row, so
//     every row offset is even and a strip pair (positions 6h .. 6h+5) reads
//     its runs with aligned 64-bit loads, and no strip pair holds columns of
//     two rows; zones of W + 20 hold every read of a strip pair, whose
//     positions may run up to five past its row's ends.
// Fills the layout of radius W into caller buffers (any may be null) and
// returns P, s_begin, n_strips.  No allocation: usable from every entry point.
void layout_fill(int W, int* P_out, int* s_begin_out, int* n_strips_out, int16_t* strip_row,
                 int32_t* row_off, int32_t* ppos, int32_t* pcol, bool paired) {
  const int nr = 2 * W + 1;  // W <= 255: at most 511 rows
  int start[511];
  auto qlo = [W](int ri) { const int r = ri - W; return r < 0 ? -W - r : -W; };
  auto len = [W](int ri) { const int r = ri - W; return 2 * W + 1 - (r < 0 ? -r : r); };
  const int Z = paired ? W + 20 : W + 8;
  int pos = Z;  // top zone [0, Z)
  for (int ri = 0; ri < nr; ++ri) {
    const int r = ri - W;
    const int want = ((qlo(ri) - r) % 3 + 3) % 3;
    int x = pos + 2;
    if (paired && ri > 0) {  // a new strip pair for the row's first column
      const int g = ((pos - 1) / 6 + 1) * 6;
      x = x > g ? x : g;
    }
    while (x % 3 != want || (paired && ((x - qlo(ri)) & 1))) ++x;
    start[ri] = x;
    pos = x + len(ri);
  }
  const int zone = pos;                      // bottom zone [zone, zone + Z)
  const int P = (zone + Z + 15) & ~15;
  // base(row) = position(q, row) - q, for rows -W-2 .. W+2 (index ri + 2).
  // Compact: rows -W-2, -W-1 are read at q in [-3, W+4], rows W+1, W+2 at q
  // in [-W-4, 3].  Paired: at q in [-8, W+8] and [-W-8, 9], with even bases.
  auto base = [&](int ri_ext) -> int {
    if (ri_ext <= 1) return paired ? 8 : 3;
    if (ri_ext >= nr + 2) return paired ? zone + W + 10 + ((zone + W) & 1) : zone + W + 4;
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

// Largest bulk-copy segment of a chunk of `pairs` strip pairs of the paired
// layout: plane positions [lo, hi) its pairs read, lo rounded down and hi up
// to 16 entries (16-byte aligned FP32 and byte copies).
int max_pair_segment(int W, int pairs) {
  const PlaneLayout L = make_layout(W, true);
  const int s_end = L.s_begin + L.n_strips;
  const int h_begin = L.s_begin >> 1, h_end = (s_end + 1) >> 1;
  int best = 0;
  for (int h0 = h_begin; h0 < h_end; h0 += pairs) {
    const int h1 = std::min(h0 + pairs, h_end);
    int lo = 1 << 30, hi = -(1 << 30);
    for (int h = h0; h < h1; ++h) {
      const int st = std::min(std::max(2 * h + 1, L.s_begin), s_end - 1);
      int sl, sh;
      pair_span(6 * h, &L.row_off[4 * L.strip_row[st - L.s_begin]], &sl, &sh);
      lo = std::min(lo, sl); hi = std::max(hi, sh);
    }
    lo &= ~15;
    hi = (hi + 15) & ~15;
    best = std::max(best, hi - lo);
  }
  return best;
}

PlaneLayout make_layout(int W, bool paired) {
  PlaneLayout L;
  layout_fill(W, &L.P, &L.s_begin, &L.n_strips, nullptr, nullptr, nullptr, nullptr, paired);
  L.strip_row.resize(L.n_strips);
  L.row_off.resize((size_t)(2 * W + 1) * 4);
  L.ppos.resize(n_columns(W));
  L.pcol.resize(L.P);
  layout_fill(W, nullptr, nullptr, nullptr, L.strip_row.data(), L.row_off.data(), L.ppos.data(),
              L.pcol.data(), paired);
  return L;
}

namespace {

struct DevLayout {
  int P = 0, s_begin = 0, n_strips = 0;
  int16_t* strip_row = nullptr;
  int32_t* row_off = nullptr;
  int32_t* ppos = nullptr;
  int32_t* pcol = nullptr;
};

struct Entry {
  int32_t* nbr = nullptr;
  int8_t* sigma = nullptr;
  int A = 0;
  DevLayout lay[2];  // compact (resident solver), paired (streamed solver)
};

pc_status upload_layout(const PlaneLayout& lay, DevLayout* d) {
  d->P = lay.P; d->s_begin = lay.s_begin; d->n_strips = lay.n_strips;
  PC_CUDA(cudaMalloc(&d->strip_row, sizeof(int16_t) * lay.strip_row.size()));
  PC_CUDA(cudaMalloc(&d->row_off, sizeof(int32_t) * lay.row_off.size()));
  PC_CUDA(cudaMalloc(&d->ppos, sizeof(int32_t) * lay.ppos.size()));
  PC_CUDA(cudaMalloc(&d->pcol, sizeof(int32_t) * lay.pcol.size()));
  PC_CUDA(cudaMemcpy(d->strip_row, lay.strip_row.data(), sizeof(int16_t) * lay.strip_row.size(), cudaMemcpyHostToDevice));
  PC_CUDA(cudaMemcpy(d->row_off, lay.row_off.data(), sizeof(int32_t) * lay.row_off.size(), cudaMemcpyHostToDevice));
  PC_CUDA(cudaMemcpy(d->ppos, lay.ppos.data(), sizeof(int32_t) * lay.ppos.size(), cudaMemcpyHostToDevice));
  PC_CUDA(cudaMemcpy(d->pcol, lay.pcol.data(), sizeof(int32_t) * lay.pcol.size(), cudaMemcpyHostToDevice));
  return PC_OK;
}

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
    for (int v = 0; v < 2; ++v) {
      const pc_status rc = upload_layout(make_layout(W, v == 1), &e.lay[v]);
      if (rc) return rc;
    }
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
  const DevLayout& c = e.lay[0];
  const DevLayout& d = e.lay[1];
  out->P = c.P; out->s_begin = c.s_begin; out->n_strips = c.n_strips;
  out->strip_row = c.strip_row; out->row_off = c.row_off; out->ppos = c.ppos; out->pcol = c.pcol;
  out->P2 = d.P; out->s_begin2 = d.s_begin; out->n_strips2 = d.n_strips;
  out->strip_row2 = d.strip_row; out->row_off2 = d.row_off; out->ppos2 = d.ppos; out->pcol2 = d.pcol;
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
    for (const DevLayout& d : kv.second.lay) {
      cudaFree(d.strip_row);
      cudaFree(d.row_off);
      cudaFree(d.ppos);
      cudaFree(d.pcol);
    }
  }
  cudaSetDevice(cur);
  g_cache.clear();
}

}  // namespace pc

namespace {
pc_status copy_layout(int32_t W, bool paired, int32_t* P, int32_t* s_begin, int32_t* n_strips,
                      int16_t* strip_row, int32_t* row_off, int32_t* ppos, int32_t* pcol) {
  if (W < 0 || W > 255) { pc::set_error("layout: W must be in [0, 255]"); return PC_ERR_ARG; }
  const pc::PlaneLayout L = pc::make_layout(W, paired);
  if (P) *P = L.P;
  if (s_begin) *s_begin = L.s_begin;
  if (n_strips) *n_strips = L.n_strips;
  if (strip_row) std::copy(L.strip_row.begin(), L.strip_row.end(), strip_row);
  if (row_off) std::copy(L.row_off.begin(), L.row_off.end(), row_off);
  if (ppos) std::copy(L.ppos.begin(), L.ppos.end(), ppos);
  if (pcol) std::copy(L.pcol.begin(), L.pcol.end(), pcol);
  return PC_OK;
}
}  // namespace

// Host-side copies of the plane layouts of radius W (diagnostics and tests).
extern "C" pc_status pc_lattice_layout(int32_t W, int32_t* P, int32_t* s_begin, int32_t* n_strips,
                                       int16_t* strip_row, int32_t* row_off, int32_t* ppos,
                                       int32_t* pcol) {
  return copy_layout(W, false, P, s_begin, n_strips, strip_row, row_off, ppos, pcol);
}

extern "C" pc_status pc_stream_layout(int32_t W, int32_t* P, int32_t* s_begin, int32_t* n_strips,
                                      int16_t* strip_row, int32_t* row_off, int32_t* ppos,
                                      int32_t* pcol) {
  return copy_layout(W, true, P, s_begin, n_strips, strip_row, row_off, ppos, pcol);
}

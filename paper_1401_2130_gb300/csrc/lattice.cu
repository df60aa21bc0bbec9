// lattice.cu -- per-W column tables of the fibre lattice (Sec. II.A, Fig. 1),
// built on the host once per device and cached.
//
// Column order: row-major over r = -W..W, q ascending within a row, keeping
// (q, r) with max(|q|, |r|, |q + r|) <= W.  For each column the table holds
// its 12 side-contact neighbour columns in the direction order of common.cuh
// (the sentinel value A marks a neighbour outside the hexagon) and its
// sublattice sigma = (q - r) mod 3.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace pc {

int64_t n_columns(int W) { return 3ll * W * (W + 1) + 1; }

namespace {

struct Entry {
  int32_t* nbr = nullptr;
  int8_t* sigma = nullptr;
  int A = 0;
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
  }
  cudaSetDevice(cur);
  g_cache.clear();
}

}  // namespace pc

// noalloc.cu -- pc_inspect_static: the resident inspection without any
// device-memory allocation.
//
// Some callers cannot allocate device memory at the point where they need an
// inspection: a process whose framework has reserved the whole device for
// its own pool allocator (a cudaMalloc there fails or fragments the pool),
// and latency-critical loops for which cudaMalloc / cudaFree are off limits
// because they can synchronise the whole device.  This entry point serves
// them: every piece of device scratch it needs -- the work and percolation
// counters, the lattice tables of the requested W, and the device staging of
// the per-configuration outputs -- lives in one file-scope static device
// array, g_static_scratch, of kStaticBytes bytes.  Every GPU that loads the
// library holds that array until the process exits.
//
// Limits: the lattice must fit the resident (shared-memory) solver and have
// at most kStaticMaxColumns columns; at most kStaticMaxConfigs configurations
// per call.  Larger requests are rejected with PC_ERR_ARG before any work.
//
// Sharing: all calls on a device use the same array and it keeps the last
// call's contents.  The counters are cleared at the start of every call and
// the tables rewritten, but two calls whose work overlaps on the GPU (for
// example on two streams) race on the array and corrupt each other's
// results; callers must serialise them.
//
// Set-up: the first call on a device looks up the array's device address
// with cudaGetSymbolAddress while that device is current, and caches it.
// Make that first call before any stream capture begins.  A device reset
// (cudaDeviceReset) invalidates the cached address; pc_shutdown() forgets it
// (with every other cached device object), and the next call looks it up
// again.
//
// Limits in practice: the resident solver holds the whole configuration in
// one CTA's shared memory (227 KB on GB300), which bounds the lattice long
// before the tables do: W <= 26 (at L = 1), W = 20 up to L = 8, W = 8 up to
// L = 74.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace pc {

namespace {

constexpr int kStaticMaxColumns = 8192;       // W <= 51
constexpr int kStaticMaxW = 51;
constexpr int kStaticMaxP = 9216;             // plane entries of the widest allowed lattice
constexpr int kStaticMaxStrips = kStaticMaxP / 3 + 2;
constexpr int kStaticMaxRows = 2 * kStaticMaxW + 1;
constexpr int64_t kStaticMaxConfigs = 1 << 18;
constexpr size_t kCtrBytes = 256;
constexpr size_t kNbrBytes = sizeof(int32_t) * kStaticMaxColumns * kLateral;
constexpr size_t kSigBytes = kStaticMaxColumns;
constexpr size_t kLayBytes = sizeof(int32_t) * (kStaticMaxColumns + kStaticMaxP + 4 * kStaticMaxRows) +
                             sizeof(int16_t) * kStaticMaxStrips;
constexpr size_t kOutBytes = (size_t)kStaticMaxConfigs * (1 + 4 + 4 + 4);
constexpr size_t kStaticBytes = kCtrBytes + kNbrBytes + kSigBytes + ((kLayBytes + 255) & ~(size_t)255) + kOutBytes;

// host staging of the layout tables (filled without allocation, then copied)
std::mutex g_host_mu;
int32_t h_ppos[kStaticMaxColumns];
int32_t h_pcol[kStaticMaxP];
int32_t h_roff[4 * kStaticMaxRows];
int16_t h_srow[kStaticMaxStrips];

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Address of g_static_scratch on the current device (set-up on first use).
pc_status static_scratch(unsigned char** out) {
  int dev = 0;
  PC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("pc_inspect_static: device ordinal out of range");
    return PC_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
    g_addr[dev] = (unsigned char*)p;
  }
  *out = g_addr[dev];
  return PC_OK;
}

// Lattice tables of radius W (same content as the host-built cache): for each
// column in row-major order its 12 side-contact neighbour columns (A when
// outside the hexagon) and its sublattice.
__global__ void static_tables_kernel(int W, int A, int32_t* nbr, int8_t* sigma) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= A) return;
  int r = -W, start = 0;
  for (; r <= W; ++r) {
    const int len = 2 * W + 1 - (r < 0 ? -r : r);
    if (a < start + len) break;
    start += len;
  }
  const int qlo = r < 0 ? -W - r : -W;
  const int q = qlo + (a - start);
  sigma[a] = (int8_t)(((q - r) % 3 + 3) % 3);
  for (int d = 0; d < kLateral; ++d) {
    const int qq = q + dir_dq(d), rr = r + dir_dr(d);
    int j = A;
    if (rr >= -W && rr <= W) {
      const int lo = rr < 0 ? -W - rr : -W, hi = rr < 0 ? W : W - rr;
      if (qq >= lo && qq <= hi) {
        int s = 0;
        for (int x = -W; x < rr; ++x) s += 2 * W + 1 - (x < 0 ? -x : x);
        j = s + (qq - lo);
      }
    }
    nbr[a * kLateral + d] = j;
  }
}

}  // namespace

// Forget the cached device addresses of the static array (pc_shutdown).
void release_static() {
  std::lock_guard<std::mutex> lk(g_mu);
  for (int d = 0; d < kMaxDevices; ++d) g_addr[d] = nullptr;
}

}  // namespace pc

using namespace pc;

extern "C" pc_status pc_inspect_static(int32_t W, int32_t L, double p, uint64_t seed,
                                       int64_t config_begin, int64_t n_configs,
                                       uint8_t* verdicts, int32_t* first_hit, float* mass,
                                       int32_t* m_stop, int64_t* n_percolating, double* Pi,
                                       void* cuda_stream) {
  NvtxRange nvtx_("pc_inspect_static");
  if (W < 0 || W > 255 || L < 1 || L >= (1 << 24)) { set_error("pc_inspect_static: bad W or L"); return PC_ERR_ARG; }
  if (!(p >= 0.0 && p <= 1.0)) { set_error("pc_inspect_static: p must be in [0, 1]"); return PC_ERR_ARG; }
  if (n_configs < 0 || config_begin < 0 || config_begin + n_configs > ((int64_t)1 << 32)) {
    set_error("pc_inspect_static: bad configuration range"); return PC_ERR_ARG;
  }
  if (n_configs > kStaticMaxConfigs) {
    set_error("pc_inspect_static: at most 262144 configurations per call"); return PC_ERR_ARG;
  }
  const int64_t A64 = n_columns(W);
  if (A64 > kStaticMaxColumns) {
    set_error("pc_inspect_static: at most 8192 columns (W <= 51)"); return PC_ERR_ARG;
  }
  const int A = (int)A64;
  if (!resident_fits(W, L)) {
    set_error("pc_inspect_static: lattice state exceeds one CTA's shared memory"); return PC_ERR_ARG;
  }
  if (n_configs > 0 && !verdicts) { set_error("pc_inspect_static: verdicts must not be NULL"); return PC_ERR_ARG; }
  // the layout's sizes are checked against the static tables before any
  // work is enqueued
  int P = 0, s_begin = 0, n_strips = 0;
  layout_fill(W, &P, &s_begin, &n_strips, nullptr, nullptr, nullptr, nullptr);
  if (P > kStaticMaxP || n_strips > kStaticMaxStrips) {
    set_error("pc_inspect_static: layout exceeds the static tables"); return PC_ERR_ARG;
  }
  unsigned char* base = nullptr;
  pc_status rc = static_scratch(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (n_configs == 0) {
    if (n_percolating) *n_percolating = 0;
    if (Pi) *Pi = 0.0;
    return PC_OK;
  }
  unsigned long long* work = (unsigned long long*)base;
  unsigned long long* n_perc = work + 1;
  int32_t* nbr = (int32_t*)(base + kCtrBytes);
  int8_t* sig = (int8_t*)(base + kCtrBytes + kNbrBytes);
  unsigned char* lay = base + kCtrBytes + kNbrBytes + kSigBytes;
  int32_t* d_ppos = (int32_t*)lay;
  int32_t* d_pcol = d_ppos + kStaticMaxColumns;
  int32_t* d_roff = d_pcol + kStaticMaxP;
  int16_t* d_srow = (int16_t*)(d_roff + 4 * kStaticMaxRows);
  unsigned char* o = lay + ((kLayBytes + 255) & ~(size_t)255);
  int32_t* d_fh = (int32_t*)o;
  float* d_mass = (float*)(o + 4 * (size_t)kStaticMaxConfigs);
  int32_t* d_ms = (int32_t*)(o + 8 * (size_t)kStaticMaxConfigs);
  uint8_t* d_v = (uint8_t*)(o + 12 * (size_t)kStaticMaxConfigs);

  PC_CUDA(cudaMemsetAsync(base, 0, kCtrBytes, st));
  static_tables_kernel<<<(A + 127) / 128, 128, 0, st>>>(W, A, nbr, sig);
  PC_CUDA(cudaGetLastError());
  {
    // pageable copies from static host tables: they synchronise, but allocate nothing
    std::lock_guard<std::mutex> lk(g_host_mu);
    layout_fill(W, nullptr, nullptr, nullptr, h_srow, h_roff, h_ppos, h_pcol);
    PC_CUDA(cudaMemcpyAsync(d_ppos, h_ppos, sizeof(int32_t) * A, cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaMemcpyAsync(d_pcol, h_pcol, sizeof(int32_t) * P, cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaMemcpyAsync(d_roff, h_roff, sizeof(int32_t) * 4 * (2 * W + 1), cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaMemcpyAsync(d_srow, h_srow, sizeof(int16_t) * n_strips, cudaMemcpyHostToDevice, st));
    PC_CUDA(cudaStreamSynchronize(st));
  }

  ResidentArgs a;
  a.lat.W = W; a.lat.L = L; a.lat.A = A; a.lat.N = (int64_t)A * L; a.lat.S = A + 1;
  a.lat.TW = (L + 31) / 32; a.lat.TWP = a.lat.TW + 2; a.lat.nbr = nbr; a.lat.sigma = sig;
  a.lat.P = P; a.lat.s_begin = s_begin; a.lat.n_strips = n_strips;
  a.lat.strip_row = d_srow; a.lat.row_off = d_roff; a.lat.ppos = d_ppos; a.lat.pcol = d_pcol;
  a.occ.k0 = (uint32_t)(seed & 0xffffffffu); a.occ.k1 = (uint32_t)(seed >> 32);
  a.occ.cfg = 0; a.occ.wl = (uint32_t)W | ((uint32_t)L << 8); a.occ.T = threshold_of(p);
  a.occ_bits = nullptr; a.words_per_cfg = (a.lat.N + 31) / 32;
  a.n_cfg = n_configs; a.cfg0 = (uint32_t)config_begin;
  a.verdict = d_v; a.first_hit = d_fh; a.mass = d_mass; a.m_stop = d_ms;
  a.n_perc = n_perc; a.work = work; a.prep_chunk = 8;
  if ((rc = launch_resident(a, resident_threads(A, L), st))) return rc;

  const size_t n = (size_t)n_configs;
  PC_CUDA(cudaMemcpyAsync(verdicts, d_v, n, cudaMemcpyDeviceToHost, st));
  if (first_hit) PC_CUDA(cudaMemcpyAsync(first_hit, d_fh, n * 4, cudaMemcpyDeviceToHost, st));
  if (mass) PC_CUDA(cudaMemcpyAsync(mass, d_mass, n * 4, cudaMemcpyDeviceToHost, st));
  if (m_stop) PC_CUDA(cudaMemcpyAsync(m_stop, d_ms, n * 4, cudaMemcpyDeviceToHost, st));
  unsigned long long cnt = 0;
  PC_CUDA(cudaMemcpyAsync(&cnt, n_perc, 8, cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaStreamSynchronize(st));
  if (n_percolating) *n_percolating = (int64_t)cnt;
  if (Pi) *Pi = (double)cnt / (double)n_configs;
  return PC_OK;
}

// api.cu -- the extern "C" entry points of libpercol (include/percol.h).
//
// Validates arguments, chooses the solver (shared-memory resident when the
// configuration's state fits one CTA, streamed otherwise), allocates the
// call's stream-ordered scratch and marshals host or device outputs.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "common.cuh"
#include "kernels.cuh"

namespace pc {

namespace {
thread_local std::string g_err;
}

void set_error(const std::string& msg) { g_err = msg; }

pc_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return PC_ERR_CUDA;
}

namespace {

pc_status check_lattice(int32_t W, int32_t L) {
  if (W < 0 || W > 255) { set_error("W must be in [0, 255]"); return PC_ERR_ARG; }
  if (L < 1 || L >= (1 << 24)) { set_error("L must be in [1, 2^24)"); return PC_ERR_ARG; }
  // per-layer arrays of the solvers have (L + 2) rows of A + 1 entries,
  // indexed with 32-bit integers
  const int64_t rows = (n_columns(W) + 1) * ((int64_t)L + 2);
  if (rows >= (int64_t)1 << 31) { set_error("lattice too large: (A + 1)(L + 2) >= 2^31"); return PC_ERR_ARG; }
  return PC_OK;
}

pc_status check_range(int64_t config_begin, int64_t n_configs) {
  if (n_configs < 0 || config_begin < 0 || config_begin + n_configs > ((int64_t)1 << 32)) {
    set_error("configurations must satisfy 0 <= begin, n >= 0, begin + n <= 2^32");
    return PC_ERR_ARG;
  }
  return PC_OK;
}

}  // namespace

bool resident_fits(int W, int L) {
  int dev = 0, max_smem = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int64_t A = n_columns(W);
  if (A > 32767) return false;
  Lattice lat = {};
  lat.W = W; lat.L = L; lat.A = (int)A;
  layout_fill(W, &lat.P, &lat.s_begin, &lat.n_strips, nullptr, nullptr, nullptr, nullptr);
  return resident_smem(lat) <= (size_t)max_smem;
}

int resident_threads(int A, int L) {
  // about one (strip, 16-layer chunk) item per thread; strips ~ A / 3
  const long long items = ((long long)A / 3 + 1) * ((L + 15) / 16);
  long long t = (items + 31) / 32 * 32;
  if (t < 128) t = 128;
  if (t > 640) t = 640;
  return (int)t;
}

namespace {

struct Scratch {
  unsigned long long* work = nullptr;
  unsigned long long* n_perc = nullptr;
  uint8_t* verdict = nullptr;
  int32_t* first_hit = nullptr;
  float* mass = nullptr;
  int32_t* m_stop = nullptr;
  char* base = nullptr;
};

// Shared implementation of pc_inspect / pc_inspect_occupancy.
pc_status inspect_impl(int32_t W, int32_t L, double p, uint64_t seed, int64_t cfg0,
                       const uint32_t* occ_bits, int64_t n, uint8_t* verdicts,
                       int32_t* first_hit, float* mass, int32_t* m_stop,
                       int64_t* n_percolating, double* Pi, int32_t flags, void* stream) {
  const bool dev_out = (flags & PC_OUT_DEVICE) != 0;
  if (flags & ~(PC_OUT_DEVICE | PC_MODE_RESIDENT | PC_MODE_STREAM | PC_BITS_ONLY | PC_VERDICT_FIRST)) {
    set_error("unknown flag bits"); return PC_ERR_ARG;
  }
  if (!verdicts && n > 0) { set_error("verdicts must not be NULL"); return PC_ERR_ARG; }
  if (dev_out && Pi) { set_error("Pi must be NULL with PC_OUT_DEVICE"); return PC_ERR_ARG; }
  if ((flags & PC_MODE_RESIDENT) && (flags & PC_MODE_STREAM)) { set_error("conflicting mode flags"); return PC_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) {
    if (n_percolating) {
      if (dev_out) PC_CUDA(cudaMemsetAsync(n_percolating, 0, sizeof(int64_t), st));
      else *n_percolating = 0;
    }
    if (Pi) *Pi = 0.0;
    return PC_OK;
  }
  Lattice lat;
  pc_status rc = get_lattice(W, L, &lat);
  if (rc) return rc;

  // call scratch: counters (+ device copies of host outputs)
  size_t bytes = 64;  // work counter, percolating counter, streamed-solver error flag
  if (!dev_out) bytes += (size_t)n * (1 + 4 + 4 + 4) + 64;
  Scratch s;
  PC_CUDA(cudaMallocAsync((void**)&s.base, bytes, st));
  s.work = (unsigned long long*)s.base;
  s.n_perc = s.work + 1;
  if (dev_out) {
    s.verdict = verdicts; s.first_hit = first_hit; s.mass = mass; s.m_stop = m_stop;
    if (n_percolating) s.n_perc = (unsigned long long*)n_percolating;
  } else {
    char* q = s.base + 64;
    s.first_hit = (int32_t*)q; q += (size_t)n * 4;
    s.mass = (float*)q; q += (size_t)n * 4;
    s.m_stop = (int32_t*)q; q += (size_t)n * 4;
    s.verdict = (uint8_t*)q;
    if (!first_hit) s.first_hit = nullptr;
    if (!mass) s.mass = nullptr;
    if (!m_stop) s.m_stop = nullptr;
  }
  rc = PC_OK;
  do {
    if (cudaMemsetAsync(s.base, 0, 64, st) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "memset"); break; }
    if (dev_out && n_percolating &&
        cudaMemsetAsync(n_percolating, 0, sizeof(int64_t), st) != cudaSuccess) {
      rc = cuda_fail(cudaGetLastError(), "memset"); break;
    }
    OccStream os;
    os.k0 = (uint32_t)(seed & 0xffffffffu);
    os.k1 = (uint32_t)(seed >> 32);
    os.cfg = 0;
    os.wl = (uint32_t)W | ((uint32_t)L << 8);
    os.T = occ_bits ? 0 : threshold_of(p);
    const int64_t wpc = (lat.N + 31) / 32;

    bool resident = resident_fits(W, L);
    if (flags & PC_MODE_STREAM) resident = false;
    if ((flags & PC_MODE_RESIDENT) && !resident) {
      set_error("PC_MODE_RESIDENT: lattice state exceeds shared memory"); rc = PC_ERR_OOM; break;
    }
    if (resident) {
      ResidentArgs a;
      a.lat = lat; a.occ = os; a.occ_bits = occ_bits; a.words_per_cfg = wpc;
      a.n_cfg = n; a.cfg0 = (uint32_t)cfg0;
      a.verdict = s.verdict; a.first_hit = s.first_hit; a.mass = s.mass; a.m_stop = s.m_stop;
      a.n_perc = s.n_perc; a.work = s.work; a.prep_chunk = 8;
      a.bits_only = (flags & PC_BITS_ONLY) ? 1 : 0;
      a.verdict_first = (flags & PC_VERDICT_FIRST) ? 1 : 0;
      rc = launch_resident(a, tuned_threads(lat, occ_bits ? 0.2 : p, seed, st), st);
    } else {
      StreamJob j;
      j.lat = lat; j.occ = os; j.occ_bits = occ_bits; j.words_per_cfg = wpc;
      j.n_cfg = n; j.cfg0 = (uint32_t)cfg0;
      j.out.verdict = s.verdict; j.out.first_hit = s.first_hit; j.out.mass = s.mass;
      j.out.m_stop = s.m_stop; j.out.n_perc = s.n_perc;
      j.bits_only = (flags & PC_BITS_ONLY) ? 1 : 0;
      j.error_out = (int*)(s.work + 2);
      rc = (!j.bits_only && (flags & PC_VERDICT_FIRST)) ? run_stream_verdict_first(j, st) : run_stream(j, st);
    }
    if (rc) break;
    if (!dev_out) {
      cudaError_t e = cudaMemcpyAsync(verdicts, s.verdict, (size_t)n, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && first_hit) e = cudaMemcpyAsync(first_hit, s.first_hit, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && mass) e = cudaMemcpyAsync(mass, s.mass, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && m_stop) e = cudaMemcpyAsync(m_stop, s.m_stop, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
      unsigned long long cnt = 0;
      int err = 0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, s.n_perc, 8, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&err, s.work + 2, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { rc = cuda_fail(e, "copy outputs"); break; }
      if (err & 2) { set_error("streamed solver: a bulk-copy wait timed out"); rc = PC_ERR_TIMEOUT; break; }
      if (err) { set_error("streamed solver: tick bound or device check failed"); rc = PC_ERR_INTERNAL; break; }
      if (n_percolating) *n_percolating = (int64_t)cnt;
      if (Pi) *Pi = (double)cnt / (double)n;
    }
  } while (0);
  cudaError_t fe = cudaFreeAsync(s.base, st);
  if (rc == PC_OK && fe != cudaSuccess) rc = cuda_fail(fe, "free scratch");
  if (rc == PC_OK) {
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) rc = cuda_fail(le, "launch");
  }
  return rc;
}

}  // namespace
}  // namespace pc

using namespace pc;

extern "C" {

pc_status pc_lattice_info(int32_t W, int32_t L, int64_t* n_columns_out, int64_t* n_sites) {
  pc_status rc = check_lattice(W, L);
  if (rc) return rc;
  const int64_t A = n_columns(W);
  if (n_columns_out) *n_columns_out = A;
  if (n_sites) *n_sites = A * (int64_t)L;
  return PC_OK;
}

pc_status pc_occupancy(int32_t W, int32_t L, double p, uint64_t seed, int64_t config_begin,
                       int64_t n_configs, uint32_t* occ_bits, void* cuda_stream) {
  NvtxRange nvtx_("pc_occupancy");
  pc_status rc = check_lattice(W, L);
  if (rc) return rc;
  if (!(p >= 0.0 && p <= 1.0)) { set_error("p must be in [0, 1]"); return PC_ERR_ARG; }
  if ((rc = check_range(config_begin, n_configs))) return rc;
  if (n_configs == 0) return PC_OK;
  if (!occ_bits) { set_error("occ_bits must not be NULL"); return PC_ERR_ARG; }
  Lattice lat;
  if ((rc = get_lattice(W, L, &lat))) return rc;
  OccStream os;
  os.k0 = (uint32_t)(seed & 0xffffffffu);
  os.k1 = (uint32_t)(seed >> 32);
  os.cfg = 0;
  os.wl = (uint32_t)W | ((uint32_t)L << 8);
  os.T = threshold_of(p);
  return launch_occupancy(lat, os, (uint32_t)config_begin, n_configs, occ_bits,
                          (cudaStream_t)cuda_stream);
}

pc_status pc_occupancy_fixed(int32_t W, int32_t L, int64_t n_metallic, uint64_t seed,
                             int64_t config_begin, int64_t n_configs, uint32_t* occ_bits,
                             void* cuda_stream) {
  NvtxRange nvtx_("pc_occupancy_fixed");
  pc_status rc = check_lattice(W, L);
  if (rc) return rc;
  const int64_t N = n_columns(W) * (int64_t)L;
  if (n_metallic < 0 || n_metallic > N) { set_error("n_metallic must be in [0, N]"); return PC_ERR_ARG; }
  if ((rc = check_range(config_begin, n_configs))) return rc;
  if (n_configs == 0) return PC_OK;
  if (!occ_bits) { set_error("occ_bits must not be NULL"); return PC_ERR_ARG; }
  Lattice lat;
  if ((rc = get_lattice(W, L, &lat))) return rc;
  OccStream os;
  os.k0 = (uint32_t)(seed & 0xffffffffu);
  os.k1 = (uint32_t)(seed >> 32);
  os.cfg = 0;
  os.wl = (uint32_t)W | ((uint32_t)L << 8);
  os.T = 0;
  return launch_occupancy_fixed(lat, os, (uint32_t)config_begin, n_configs, n_metallic, occ_bits,
                                (cudaStream_t)cuda_stream);
}

pc_status pc_inspect(int32_t W, int32_t L, double p, uint64_t seed, int64_t config_begin,
                     int64_t n_configs, uint8_t* verdicts, int32_t* first_hit, float* mass,
                     int32_t* m_stop, int64_t* n_percolating, double* Pi, int32_t flags,
                     void* cuda_stream) {
  NvtxRange nvtx_("pc_inspect");
  pc_status rc = check_lattice(W, L);
  if (rc) return rc;
  if (!(p >= 0.0 && p <= 1.0)) { set_error("p must be in [0, 1]"); return PC_ERR_ARG; }
  if ((rc = check_range(config_begin, n_configs))) return rc;
  return inspect_impl(W, L, p, seed, config_begin, nullptr, n_configs, verdicts, first_hit,
                      mass, m_stop, n_percolating, Pi, flags, cuda_stream);
}

pc_status pc_inspect_occupancy(int32_t W, int32_t L, const uint32_t* occ_bits, int64_t n_configs,
                               uint8_t* verdicts, int32_t* first_hit, float* mass,
                               int32_t* m_stop, int64_t* n_percolating, double* Pi,
                               int32_t flags, void* cuda_stream) {
  NvtxRange nvtx_("pc_inspect_occupancy");
  pc_status rc = check_lattice(W, L);
  if (rc) return rc;
  if ((rc = check_range(0, n_configs))) return rc;
  if (n_configs > 0 && !occ_bits) { set_error("occ_bits must not be NULL"); return PC_ERR_ARG; }
  return inspect_impl(W, L, 0.0, 0, 0, occ_bits, n_configs, verdicts, first_hit, mass, m_stop,
                      n_percolating, Pi, flags, cuda_stream);
}

pc_status pc_shutdown(void) {
  release_batches();
  release_lattices();
  release_static();
  return PC_OK;
}

const char* pc_last_error(void) { return g_err.c_str(); }

}  // extern "C"

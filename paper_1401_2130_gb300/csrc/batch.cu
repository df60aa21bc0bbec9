// batch.cu -- pc_batch_run (one GPU submission for many queries of mixed
// lattice sizes) and the autotuner of the resident solver's CTA size.
//
// A batch becomes one CUDA graph:
//   memset(counters) -> { at most three persistent resident launches, one per
//                         shared-memory class, over every query whose state
//                         fits shared memory, configurations taken from one
//                         list in decreasing lattice size (parallel graph
//                         branches, so the grids overlap and fill each other's
//                         tails) }
//                    -> { init -> WHILE(sweep, control) of the streamed solver
//                         over all remaining queries, sharing one slot pool }
// The instantiated graph and its device memory are cached per batch (same
// queries, output pointers and flags) and replayed by later calls.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "tune_file.h"

namespace pc {

// ---------------------------------------------------------------------------
// Autotuner: per (W, L, p bin), the resident CTA size with the lowest
// measured time on a sample of configurations; kept in memory and in
// PC_TUNE_FILE.  p matters: below the threshold configurations stop after a
// few short steps, above it they sweep the whole fibre, and the best CTA
// size differs between the two regimes.
// ---------------------------------------------------------------------------
namespace {

constexpr double kTunePBins = 40.0;  // p bins of width 0.025

std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
bool g_tune_loaded = false;

int p_bin(double p) { return (int)std::lround(p * kTunePBins); }

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = std::getenv("PC_TUNE_FILE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  tune_read(f, kResidentMaxThreads, g_tune);
  std::fclose(f);
}

void tune_save() {
  const char* path = std::getenv("PC_TUNE_FILE");
  if (!path) return;
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  tune_write(f, g_tune);
  std::fclose(f);
  std::rename(tmp.c_str(), path);
}

}  // namespace

int tuned_threads(const Lattice& lat, double p, uint64_t seed, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_load();
  const std::tuple<int, int, int> key{lat.W, lat.L, p_bin(p)};
  auto it = g_tune.find(key);
  if (it != g_tune.end()) return it->second;
  const int fallback = resident_threads(lat.A, lat.L);
  const int64_t n = 2048;
  char* mem = nullptr;
  if (cudaMallocAsync((void**)&mem, 64 + n * 13, st) != cudaSuccess) return fallback;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = fallback;
  float best_ms = 1e30f;
  const int cand[] = {128, 256, 384, 512, 640};
  for (int T : cand) {
    ResidentArgs a;
    a.lat = lat;
    a.occ.k0 = (uint32_t)(seed & 0xffffffffu); a.occ.k1 = (uint32_t)(seed >> 32);
    a.occ.cfg = 0; a.occ.wl = (uint32_t)lat.W | ((uint32_t)lat.L << 8); a.occ.T = threshold_of(p);
    a.occ_bits = nullptr; a.words_per_cfg = (lat.N + 31) / 32;
    a.n_cfg = n; a.cfg0 = 0x80000000u;  // a sample away from ordinary ranges
    a.verdict = (uint8_t*)(mem + 64); a.first_hit = (int32_t*)(mem + 64 + n);
    a.mass = (float*)(mem + 64 + 5 * n); a.m_stop = (int32_t*)(mem + 64 + 9 * n);
    a.n_perc = (unsigned long long*)(mem + 8); a.work = (unsigned long long*)mem;
    a.prep_chunk = 8;
    float ms = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 2 && ok; ++rep) {
      cudaMemsetAsync(mem, 0, 64, st);
      cudaEventRecord(e0, st);
      ok = launch_resident(a, T, st) == PC_OK;
      cudaEventRecord(e1, st);
      if (ok) ok = cudaEventSynchronize(e1) == cudaSuccess;
      if (ok) cudaEventElapsedTime(&ms, e0, e1);
    }
    if (ok && ms < best_ms) { best_ms = ms; best = T; }
    cudaGetLastError();  // a candidate that does not fit is simply skipped
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(mem, st);
  cudaStreamSynchronize(st);
  g_tune[key] = best;
  tune_save();
  return best;
}

// ---------------------------------------------------------------------------
// Batch graphs
// ---------------------------------------------------------------------------
namespace {

struct QueryPlan {
  int solver = 0;    // 0 resident, 1 streamed
  int threads = 0;
  unsigned long long* n_perc = nullptr;  // device counter
  uint8_t* v = nullptr; int32_t* fh = nullptr; float* mass = nullptr; int32_t* ms = nullptr;  // device outputs
};

struct BatchGraph {
  std::string key;
  int device = 0;
  char* mem = nullptr;       // counters + host-output staging
  size_t mem_bytes = 0;
  char* tab = nullptr;       // query tables of the persistent resident launches
  StreamPlan* plan = nullptr;
  std::vector<StreamJob> blocked;  // verdict-only streamed queries run after the batch graph (blocked.cu)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<QueryPlan> qp;
  // One replay at a time: a call holds mu from its launch to its last copy,
  // and every replay first waits (on its own stream) for the event the
  // previous replay recorded, so replays on different streams never overlap
  // on the device (they share the counters and the output staging).
  std::mutex mu;
  cudaEvent_t done = nullptr;
};

void destroy_batch(BatchGraph* b);
// The cache and every running call hold a reference; a batch evicted or
// released while a call still uses it is destroyed when that call drops it.
using BatchPtr = std::shared_ptr<BatchGraph>;

std::mutex g_batch_mu;
std::list<BatchPtr> g_batches;  // most recent first
constexpr size_t kMaxCached = 8;

void destroy_batch(BatchGraph* b) {
  if (!b) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->done) cudaEventDestroy(b->done);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->plan) stream_plan_release(b->plan, 0);
  if (b->mem) cudaFree(b->mem);
  if (b->tab) cudaFree(b->tab);
  cudaDeviceSynchronize();
  cudaSetDevice(cur);
  delete b;
}

std::string batch_key(const pc_query* q, int64_t n, int32_t flags, int dev) {
  std::string k((const char*)q, sizeof(pc_query) * (size_t)n);
  k.append((const char*)&flags, sizeof(flags));
  k.append((const char*)&dev, sizeof(dev));
  return k;
}

// A resident-size query of a batch: its arguments, index, autotuned CTA
// size and shared memory.
struct ResidentQuery {
  ResidentArgs a;
  int64_t index;
  int threads;
  size_t smem;
};

// The batch's resident-size queries as at most three persistent launches,
// one per shared-memory class (up to 1/4, 1/2 and all of an SM's shared
// memory: 4+, 2-3 and 1 CTA per SM), so that small lattices keep their
// occupancy.  Within a launch the queries are ordered by decreasing lattice
// size (sites), so the longest configurations start first and the shorter
// ones fill the tails; the CTA size is the autotuned one of the launch's
// heaviest query (sites x configurations).  work: 3 zeroed counters.
pc_status add_resident_launches(BatchGraph* b, std::vector<ResidentQuery>& rq, const pc_query* q,
                                unsigned long long* work, const cudaGraphNode_t* dep) {
  int dev = 0, smem_sm = 0;
  PC_CUDA(cudaGetDevice(&dev));
  PC_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  auto cls = [&](size_t sm) { return sm * 4 <= (size_t)smem_sm ? 0 : sm * 2 <= (size_t)smem_sm ? 1 : 2; };
  std::stable_sort(rq.begin(), rq.end(), [](const ResidentQuery& x, const ResidentQuery& y) {
    return x.a.lat.N > y.a.lat.N;
  });
  // device tables: per class ResidentArgs[] and item offsets[] (one allocation)
  const size_t n = rq.size();
  const size_t args_b = (sizeof(ResidentArgs) * n + 255) & ~(size_t)255;
  const size_t off_b = (sizeof(long long) * (n + 3) + 255) & ~(size_t)255;
  PC_CUDA(cudaMalloc((void**)&b->tab, 3 * (args_b + off_b)));
  for (int c = 0; c < 3; ++c) {
    std::vector<ResidentArgs> args;
    std::vector<long long> item0{0};
    size_t smem = 0;
    int threads = 0;
    double heavy = -1.0;
    for (const ResidentQuery& r : rq) {
      if (cls(r.smem) != c) continue;
      args.push_back(r.a);
      item0.push_back(item0.back() + r.a.n_cfg);
      smem = std::max(smem, r.smem);
      const double w = (double)r.a.lat.N * (double)r.a.n_cfg;
      if (w > heavy) { heavy = w; threads = r.threads; }
    }
    if (args.empty() || item0.back() == 0) continue;
    for (const ResidentQuery& r : rq)
      if (cls(r.smem) == c) b->qp[r.index].threads = threads;
    char* at = b->tab + c * (args_b + off_b);
    PC_CUDA(cudaMemcpy(at, args.data(), sizeof(ResidentArgs) * args.size(), cudaMemcpyHostToDevice));
    PC_CUDA(cudaMemcpy(at + args_b, item0.data(), sizeof(long long) * item0.size(), cudaMemcpyHostToDevice));
    ResidentBatch rb;
    rb.qs = (const ResidentArgs*)at;
    rb.item0 = (const long long*)(at + args_b);
    rb.nq = (int)args.size();
    rb.work = work + c;
    cudaGraphNode_t node;
    pc_status rc = resident_multi_add_node(rb, item0.back(), smem, threads, b->graph, dep, 1, &node);
    if (rc) return rc;
  }
  return PC_OK;
}

pc_status build_batch(const pc_query* q, int64_t nq, int32_t flags, cudaStream_t st, BatchGraph** out) {
  const bool dev_out = (flags & PC_OUT_DEVICE) != 0;
  BatchGraph* b = new BatchGraph();
  cudaGetDevice(&b->device);
  b->qp.resize(nq);
  // device memory: per query 2 counters, 3 class counters (+ staging of
  // host outputs)
  size_t bytes = 256 + (size_t)nq * 16 + 64;
  if (!dev_out)
    for (int64_t i = 0; i < nq; ++i) bytes += ((size_t)q[i].n_configs * 13 + 256) & ~(size_t)255;
  b->mem_bytes = bytes;
  cudaError_t e = cudaMalloc((void**)&b->mem, bytes);
  if (e != cudaSuccess) { delete b; return cuda_fail(e, "batch memory"); }
  if ((e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess) {
    destroy_batch(b);
    return cuda_fail(e, "batch event");
  }
  pc_status rc = PC_OK;
  std::vector<StreamQuery> sq;
  std::vector<ResidentQuery> rq;
  do {
    unsigned long long* ctr = (unsigned long long*)b->mem;  // [nq][2]: n_perc, work
    char* stage = b->mem + 256 + (size_t)nq * 16 + 64;
    if ((e = cudaGraphCreate(&b->graph, 0)) != cudaSuccess) { rc = cuda_fail(e, "graph create"); break; }
    cudaMemsetParams mp = {};
    mp.dst = b->mem; mp.value = 0; mp.elementSize = 1; mp.width = 256 + (size_t)nq * 16 + 64; mp.height = 1;
    mp.pitch = 0;
    cudaGraphNode_t n_zero;
    if ((e = cudaGraphAddMemsetNode(&n_zero, b->graph, nullptr, 0, &mp)) != cudaSuccess) { rc = cuda_fail(e, "memset node"); break; }
    for (int64_t i = 0; i < nq && rc == PC_OK; ++i) {
      QueryPlan& P = b->qp[i];
      P.n_perc = ctr + 2 * i;
      if (dev_out) {
        P.v = q[i].verdicts; P.fh = q[i].first_hit; P.mass = q[i].mass; P.ms = q[i].m_stop;
      } else {
        const size_t n = (size_t)q[i].n_configs;
        P.fh = (int32_t*)stage; P.mass = (float*)(stage + 4 * n); P.ms = (int32_t*)(stage + 8 * n);
        P.v = (uint8_t*)(stage + 12 * n);
        stage += (n * 13 + 256) & ~(size_t)255;
      }
      if (q[i].n_configs == 0) continue;
      Lattice lat;
      if ((rc = get_lattice(q[i].W, q[i].L, &lat))) break;
      OccStream os;
      os.k0 = (uint32_t)(q[i].seed & 0xffffffffu); os.k1 = (uint32_t)(q[i].seed >> 32);
      os.cfg = 0; os.wl = (uint32_t)q[i].W | ((uint32_t)q[i].L << 8); os.T = threshold_of(q[i].p);
      if (resident_fits(q[i].W, q[i].L)) {
        P.solver = 0;
        ResidentArgs a;
        a.lat = lat; a.occ = os; a.occ_bits = nullptr; a.words_per_cfg = (lat.N + 31) / 32;
        a.n_cfg = q[i].n_configs; a.cfg0 = (uint32_t)q[i].config_begin;
        a.verdict = P.v; a.first_hit = P.fh; a.mass = P.mass; a.m_stop = P.ms;
        a.n_perc = P.n_perc; a.work = ctr + 2 * i + 1; a.prep_chunk = 8;
        a.bits_only = (flags & PC_BITS_ONLY) ? 1 : 0;
        a.verdict_first = (flags & PC_VERDICT_FIRST) ? 1 : 0;
        if (!a.verdict) { set_error("verdicts buffer required"); rc = PC_ERR_ARG; break; }
        rq.push_back({a, i, tuned_threads(lat, q[i].p, q[i].seed, st), resident_smem(lat)});
      } else {
        P.solver = 1;
        StreamQuery s;
        s.lat = lat; s.occ = os; s.occ_bits = nullptr; s.words_per_cfg = (lat.N + 31) / 32;
        s.n_cfg = q[i].n_configs; s.cfg0 = (uint32_t)q[i].config_begin;
        s.out.verdict = P.v; s.out.first_hit = P.fh; s.out.mass = P.mass; s.out.m_stop = P.ms;
        s.out.n_perc = P.n_perc;
        s.bits_only = (flags & PC_BITS_ONLY) ? 1 : 0;
        if (!s.out.verdict) { set_error("verdicts buffer required"); rc = PC_ERR_ARG; break; }
        if (s.bits_only && !(flags & PC_ASYNC) && blocked_takes(lat)) {
          // verdicts only, and a cluster holds the cross-section: 32 steps
          // per visit of a slab, after the batch graph (in a graph of its own)
          P.solver = 2;
          StreamJob j;
          static_cast<StreamQuery&>(j) = s;
          // error flag in the counter area the graph zeroes (past the three
          // resident work counters)
          j.error_out = (int*)((char*)(ctr + 2 * nq) + 32);
          b->blocked.push_back(j);
          continue;
        }
        sq.push_back(s);
      }
    }
    if (rc) break;
    if (!rq.empty() && (rc = add_resident_launches(b, rq, q, ctr + 2 * nq, &n_zero)) != PC_OK) break;
    if (!sq.empty()) {
      // largest lattices first: long configurations start early
      std::stable_sort(sq.begin(), sq.end(), [](const StreamQuery& x, const StreamQuery& y) {
        return x.lat.N > y.lat.N;
      });
      if ((rc = stream_plan_create(sq.data(), (int)sq.size(), st, &b->plan))) break;
      cudaGraphNode_t last;
      if ((rc = stream_plan_add(b->plan, b->graph, &n_zero, 1, &last))) break;
    }
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) { rc = cuda_fail(e, "graph instantiate"); break; }
    // the plan's initialisation (on st) must be complete before any replay,
    // which may come on another stream
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { rc = cuda_fail(e, "batch build sync"); break; }
  } while (0);
  if (rc) { destroy_batch(b); return rc; }
  *out = b;
  return PC_OK;
}

}  // namespace

void release_batches() {
  std::list<BatchPtr> drop;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    drop.swap(g_batches);
  }
  // destroyed here, or by the last call still using one
}

}  // namespace pc

using namespace pc;

extern "C" pc_status pc_batch_run(const pc_query* q, int64_t nq, pc_result* out, int32_t flags,
                                  void* cuda_stream) {
  NvtxRange nvtx_("pc_batch_run");
  if (nq < 0 || (nq > 0 && !q)) { set_error("pc_batch_run: bad query array"); return PC_ERR_ARG; }
  if (flags & ~(PC_OUT_DEVICE | PC_ASYNC | PC_BITS_ONLY | PC_VERDICT_FIRST)) { set_error("pc_batch_run: unknown flag bits"); return PC_ERR_ARG; }
  const bool dev_out = (flags & PC_OUT_DEVICE) != 0, async = (flags & PC_ASYNC) != 0;
  if (async && (!dev_out || out)) { set_error("PC_ASYNC needs PC_OUT_DEVICE and out == NULL"); return PC_ERR_ARG; }
  for (int64_t i = 0; i < nq; ++i) {
    const pc_query& x = q[i];
    if (x.W < 0 || x.W > 255 || x.L < 1 || x.L >= (1 << 24)) { set_error("pc_batch_run: bad W or L"); return PC_ERR_ARG; }
    if ((n_columns(x.W) + 1) * ((int64_t)x.L + 2) >= ((int64_t)1 << 31)) { set_error("pc_batch_run: lattice too large"); return PC_ERR_ARG; }
    if (!(x.p >= 0.0 && x.p <= 1.0)) { set_error("pc_batch_run: p must be in [0, 1]"); return PC_ERR_ARG; }
    if (x.n_configs < 0 || x.config_begin < 0 || x.config_begin + x.n_configs > ((int64_t)1 << 32)) {
      set_error("pc_batch_run: bad configuration range"); return PC_ERR_ARG;
    }
    if (x.n_configs > 0 && !x.verdicts) { set_error("pc_batch_run: verdicts must not be NULL"); return PC_ERR_ARG; }
  }
  if (nq == 0) return PC_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  PC_CUDA(cudaGetDevice(&dev));
  const std::string key = batch_key(q, nq, flags, dev);
  BatchPtr b;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto it = g_batches.begin(); it != g_batches.end(); ++it)
      if ((*it)->key == key) { b = *it; g_batches.erase(it); g_batches.push_front(b); break; }
  }
  if (!b) {
    BatchGraph* raw = nullptr;
    pc_status rc = build_batch(q, nq, flags, st, &raw);
    if (rc) return rc;
    raw->key = key;
    b = BatchPtr(raw, destroy_batch);
    std::list<BatchPtr> evicted;
    {
      std::lock_guard<std::mutex> lk(g_batch_mu);
      g_batches.push_front(b);
      while (g_batches.size() > kMaxCached) { evicted.push_back(g_batches.back()); g_batches.pop_back(); }
    }
  }
  std::lock_guard<std::mutex> replay(b->mu);
  PC_CUDA(cudaStreamWaitEvent(st, b->done, 0));
  PC_CUDA(cudaGraphLaunch(b->exec, st));
  // verdict-only streamed queries on the blocked solver, after the graph
  // (which zeroes their counters), each in a graph of its own; not in
  // PC_ASYNC batches
  for (const StreamJob& j : b->blocked) {
    bool handled = false;
    pc_status rc = run_blocked(j, st, &handled);
    if (rc == PC_OK && !handled) rc = run_stream(j, st);  // the step-synchronous solver
    if (rc) return rc;
  }
  if (dev_out)
    for (int64_t i = 0; i < nq; ++i)
      if (q[i].n_percolating)
        PC_CUDA(cudaMemcpyAsync(q[i].n_percolating, b->qp[i].n_perc, 8, cudaMemcpyDeviceToDevice, st));
  if (async) {
    PC_CUDA(cudaEventRecord(b->done, st));
    return PC_OK;
  }
  int err = 0, err_b = 0;
  if (b->plan) PC_CUDA(cudaMemcpyAsync(&err, stream_plan_error(b->plan), sizeof(int), cudaMemcpyDeviceToHost, st));
  if (!b->blocked.empty()) PC_CUDA(cudaMemcpyAsync(&err_b, b->blocked[0].error_out, sizeof(int), cudaMemcpyDeviceToHost, st));
  std::vector<unsigned long long> cnt((size_t)nq);
  for (int64_t i = 0; i < nq; ++i) {
    const QueryPlan& P = b->qp[i];
    PC_CUDA(cudaMemcpyAsync(&cnt[i], P.n_perc, 8, cudaMemcpyDeviceToHost, st));
    if (!dev_out && q[i].n_configs > 0) {
      const size_t n = (size_t)q[i].n_configs;
      PC_CUDA(cudaMemcpyAsync(q[i].verdicts, P.v, n, cudaMemcpyDeviceToHost, st));
      if (q[i].first_hit) PC_CUDA(cudaMemcpyAsync(q[i].first_hit, P.fh, 4 * n, cudaMemcpyDeviceToHost, st));
      if (q[i].mass) PC_CUDA(cudaMemcpyAsync(q[i].mass, P.mass, 4 * n, cudaMemcpyDeviceToHost, st));
      if (q[i].m_stop) PC_CUDA(cudaMemcpyAsync(q[i].m_stop, P.ms, 4 * n, cudaMemcpyDeviceToHost, st));
    }
  }
  PC_CUDA(cudaEventRecord(b->done, st));
  PC_CUDA(cudaStreamSynchronize(st));
  if (err & 2) { set_error("streamed solver: a bulk-copy wait timed out"); return PC_ERR_TIMEOUT; }
  if (err) { set_error("streamed solver: tick bound or segment check failed"); return PC_ERR_INTERNAL; }
  if (err_b) { set_error("verdict-only solver: pass bound reached"); return PC_ERR_INTERNAL; }
  for (int64_t i = 0; i < nq; ++i) {
    if (!dev_out && q[i].n_percolating) *q[i].n_percolating = (int64_t)cnt[i];
    if (out) {
      out[i].n_percolating = (int64_t)cnt[i];
      out[i].Pi = q[i].n_configs ? (double)cnt[i] / (double)q[i].n_configs : 0.0;
      out[i].solver = b->qp[i].solver;
      out[i].threads = b->qp[i].threads;
    }
  }
  return PC_OK;
}

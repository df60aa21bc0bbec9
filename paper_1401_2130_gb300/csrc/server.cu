// server.cu -- pc_server_*: continuous-batching request loop.
//
// Queries (W, L, p, seed, configuration range) arrive at any time through
// pc_server_submit.  A worker thread admits them in arrival order as soon as
// their HBM footprint fits a device arena (first-fit allocator):
//   * a query whose configuration state fits one CTA's shared memory gets its
//     output buffers from the arena and one persistent resident-solver launch
//     on one of several side streams -- such launches run concurrently with
//     each other and with the streamed ticks;
//   * any other query gets its outputs plus k slots of streamed-solver state
//     (k <= free slots, bounded by what the arena holds) and the device binds
//     those slots to it; the engine runs chunks of ticks (sweep + control)
//     over all bound slots of all running queries, and a slot whose query has
//     configurations left refills itself on the device.
// Two chunks are kept in flight: while the device runs chunk c + 1, the
// worker reads chunk c's slot phases and per-query completion counts, copies
// finished queries' outputs out (on a separate stream), returns their memory
// and slots, and admits more queries, whose bindings land after the chunks
// already enqueued.  A status is trusted only for queries bound before its
// chunk.  The sweep's staging ring is sized for the widest streamed lattice
// the server accepts (max_W).  Latency = completion time - submission time.
// Results equal pc_inspect's: the occupancy stream is counter based and the
// per-configuration solve does not depend on what runs beside it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "arena.h"
#include "common.cuh"
#include "kernels.cuh"

namespace pc {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kResStreams = 4;

enum TicketState { T_PENDING, T_RUNNING, T_DONE, T_FAILED, T_CANCELLED };

struct Ticket {
  pc_query q;
  TicketState state = T_PENDING;
  pc_status status = PC_OK;
  Clock::time_point t_submit, t_done;
  pc_result result = {};
  // running state
  int kind = 0;                 // 0 resident, 1 streamed
  int stream_idx = 0;
  int qi = -1;                  // engine query index (streamed)
  size_t off_out = 0, bytes_out = 0, off_slots = 0, bytes_slots = 0;
  int nslots = 0;
  std::vector<int> slot_ids;    // slots reserved at admission (streamed)
  uint64_t start_seq = 0;       // first tick chunk enqueued after the query's binding
  cudaEvent_t ev = nullptr;
  unsigned long long* n_perc = nullptr;
  uint8_t* v = nullptr; int32_t* fh = nullptr; float* mass = nullptr; int32_t* ms = nullptr;
};

}  // namespace
}  // namespace pc

struct pc_server {
  pc_server_opts opts;
  int device = 0;
  cudaStream_t tick = nullptr;
  cudaStream_t copy = nullptr;  // output copies of finished streamed queries
  cudaStream_t res[pc::kResStreams] = {};
  int res_rr = 0;
  pc::ServerEngine* E = nullptr;
  char* arena_mem = nullptr;
  pc::Arena arena;
  std::vector<uint64_t> slot_owner;   // ticket id or 0
  std::vector<uint64_t> query_owner;  // engine query index -> ticket id or 0
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending;
  std::map<uint64_t, pc::Ticket> tickets;
  uint64_t next_ticket = 1;
  bool stop = false;
  // statistics
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, configs_done = 0;
  pc::Clock::time_point t_first, t_last;
  bool any = false;
};

namespace pc {
namespace {

size_t out_bytes(int64_t n) { return 256 + (size_t)n * 13 + 256; }

// Called with s->mu held for the ticket map; CUDA work outside the lock.
pc_status start_query(pc_server* s, uint64_t id, Ticket& t) {
  const pc_query& q = t.q;
  Lattice lat;
  pc_status rc = get_lattice(q.W, q.L, &lat);
  if (rc) return rc;
  const int64_t n = q.n_configs;
  char* o = s->arena.base + t.off_out;
  t.n_perc = (unsigned long long*)o;
  unsigned long long* work = t.n_perc + 1;
  char* d = o + 256;
  t.fh = (int32_t*)d; t.mass = (float*)(d + 4 * n); t.ms = (int32_t*)(d + 8 * n);
  t.v = (uint8_t*)(d + 12 * n);
  OccStream os;
  os.k0 = (uint32_t)(q.seed & 0xffffffffu); os.k1 = (uint32_t)(q.seed >> 32);
  os.cfg = 0; os.wl = (uint32_t)q.W | ((uint32_t)q.L << 8); os.T = threshold_of(q.p);
  if (t.kind == 0) {
    cudaStream_t st = s->res[t.stream_idx];
    PC_CUDA(cudaMemsetAsync(o, 0, 256, st));
    ResidentArgs a;
    a.lat = lat; a.occ = os; a.occ_bits = nullptr; a.words_per_cfg = (lat.N + 31) / 32;
    a.n_cfg = n; a.cfg0 = (uint32_t)q.config_begin;
    a.verdict = t.v; a.first_hit = t.fh; a.mass = t.mass; a.m_stop = t.ms;
    a.n_perc = t.n_perc; a.work = work; a.prep_chunk = 8;
    if ((rc = launch_resident(a, resident_threads(lat.A, lat.L), st))) return rc;
    PC_CUDA(cudaEventCreateWithFlags(&t.ev, cudaEventDisableTiming));
    PC_CUDA(cudaEventRecord(t.ev, st));
    return PC_OK;
  }
  cudaStream_t st = s->tick;
  if (t.slot_ids.empty()) { set_error("server: streamed query admitted without slots"); return PC_ERR_INTERNAL; }
  PC_CUDA(cudaMemsetAsync(o, 0, 256, st));
  StreamQuery sq;
  sq.lat = lat; sq.occ = os; sq.occ_bits = nullptr; sq.words_per_cfg = (lat.N + 31) / 32;
  sq.n_cfg = n; sq.cfg0 = (uint32_t)q.config_begin;
  sq.out.verdict = t.v; sq.out.first_hit = t.fh; sq.out.mass = t.mass; sq.out.m_stop = t.ms;
  sq.out.n_perc = t.n_perc;
  if ((rc = server_engine_set_query(s->E, t.qi, sq, st))) return rc;
  std::vector<int> slots, qs;
  std::vector<char*> bases;
  const size_t sb = stream_slot_bytes(lat.W, lat.L);
  for (size_t k = 0; k < t.slot_ids.size(); ++k) {
    slots.push_back(t.slot_ids[k]); qs.push_back(t.qi);
    bases.push_back(s->arena.base + t.off_slots + k * sb);
  }
  (void)id;
  // fresh slot memory: padding rows and sentinel columns must start zeroed
  PC_CUDA(cudaMemsetAsync(s->arena.base + t.off_slots, 0, t.bytes_slots, st));
  return server_engine_bind(s->E, slots.data(), qs.data(), bases.data(), (int)slots.size(), st);
}

// Copy a finished query's outputs to the caller, release its resources.
void finish_query(pc_server* s, uint64_t id, Ticket& t, cudaStream_t st) {
  const int64_t n = t.q.n_configs;
  unsigned long long cnt = 0;
  cudaError_t e = cudaMemcpyAsync(&cnt, t.n_perc, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && t.q.verdicts) e = cudaMemcpyAsync(t.q.verdicts, t.v, (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && t.q.first_hit) e = cudaMemcpyAsync(t.q.first_hit, t.fh, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && t.q.mass) e = cudaMemcpyAsync(t.q.mass, t.mass, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && t.q.m_stop) e = cudaMemcpyAsync(t.q.m_stop, t.ms, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  std::lock_guard<std::mutex> lk(s->mu);
  if (e != cudaSuccess) {
    t.state = T_FAILED;
    t.status = cuda_fail(e, "server: copy outputs");
  } else {
    t.state = T_DONE;
    t.result.n_percolating = (int64_t)cnt;
    t.result.Pi = n ? (double)cnt / (double)n : 0.0;
    t.result.solver = t.kind;
    t.result.threads = 0;
    if (t.q.n_percolating) *t.q.n_percolating = (int64_t)cnt;
  }
  t.t_done = Clock::now();
  const double ms = std::chrono::duration<double, std::milli>(t.t_done - t.t_submit).count();
  s->lat_ms.push_back(ms);
  s->completed += 1;
  s->configs_done += n;
  s->t_last = t.t_done;
  s->arena.release(t.off_out, t.bytes_out);
  if (t.bytes_slots) s->arena.release(t.off_slots, t.bytes_slots);
  for (auto& o : s->slot_owner) if (o == id) o = 0;
  if (t.qi >= 0) s->query_owner[t.qi] = 0;
  if (t.ev) { cudaEventDestroy(t.ev); t.ev = nullptr; }
  s->cv_done.notify_all();
}

void worker_main(pc_server* s) {
  cudaSetDevice(s->device);
  std::vector<uint64_t> running;
  cudaEvent_t ev[2] = {};
  for (int b = 0; b < 2; ++b) cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming);
  uint64_t next_seq = 0;  // sequence number of the next tick chunk
  int inflight = 0;       // chunks enqueued whose status has not been read
  for (;;) {
    // ---- admission (arrival order; stops at the first query that does not fit)
    std::vector<uint64_t> to_start;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) break;
      while (!s->pending.empty()) {
        const uint64_t id = s->pending.front();
        auto found = s->tickets.find(id);  // a cancelled ticket may already be polled away
        if (found == s->tickets.end() || found->second.state == T_CANCELLED) { s->pending.pop_front(); continue; }
        Ticket& t = found->second;
        const pc_query& q = t.q;
        const bool res = resident_fits(q.W, q.L);
        size_t off = 0;
        const size_t ob = out_bytes(q.n_configs);
        if (res) {
          if (!s->arena.alloc(ob, &off)) break;
          t.kind = 0; t.off_out = off; t.bytes_out = ob;
          t.stream_idx = s->res_rr; s->res_rr = (s->res_rr + 1) % kResStreams;
        } else {
          int qi = -1;
          for (size_t i = 0; i < s->query_owner.size(); ++i) if (!s->query_owner[i]) { qi = (int)i; break; }
          int free_slots = 0;
          for (auto o : s->slot_owner) free_slots += o == 0;
          if (qi < 0 || free_slots == 0) break;
          const size_t sb = stream_slot_bytes(q.W, q.L);
          if (!s->arena.alloc(ob, &off)) break;
          const size_t room = s->arena.largest();
          long long k = std::min<long long>(q.n_configs, free_slots);
          k = std::min<long long>(k, std::max(1, s->opts.max_slots_per_query));
          k = std::min<long long>(k, (long long)(room / (sb + 256)));
          size_t soff = 0;
          if (k < 1 || !s->arena.alloc((size_t)k * sb, &soff)) { s->arena.release(off, ob); break; }
          t.kind = 1; t.qi = qi; t.off_out = off; t.bytes_out = ob;
          t.off_slots = soff; t.bytes_slots = (size_t)k * sb; t.nslots = (int)k;
          s->query_owner[qi] = id;
          // reserve the slot indices now: later admissions in this pass must
          // not count them as free
          t.slot_ids.clear();
          for (size_t i = 0; i < s->slot_owner.size() && (long long)t.slot_ids.size() < k; ++i)
            if (!s->slot_owner[i]) { s->slot_owner[i] = id; t.slot_ids.push_back((int)i); }
        }
        t.state = T_RUNNING;
        s->pending.pop_front();
        to_start.push_back(id);
      }
    }
    for (uint64_t id : to_start) {
      Ticket* tp;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        tp = &s->tickets[id];
      }
      pc_status rc;
      {
        std::lock_guard<std::mutex> lk(s->mu);  // slot table
        rc = start_query(s, id, *tp);
      }
      if (rc) {
        std::lock_guard<std::mutex> lk(s->mu);
        tp->state = T_FAILED; tp->status = rc;
        s->arena.release(tp->off_out, tp->bytes_out);
        if (tp->bytes_slots) s->arena.release(tp->off_slots, tp->bytes_slots);
        for (auto& o : s->slot_owner) if (o == id) o = 0;
        if (tp->qi >= 0) s->query_owner[tp->qi] = 0;
        s->cv_done.notify_all();
      } else {
        tp->start_seq = next_seq;
        running.push_back(id);
      }
    }
    // ---- device work: keep two tick chunks in flight while streamed queries
    // run, so the host's bookkeeping for chunk c overlaps chunk c + 1 on the
    // device.  Work enqueued now (bindings) lands after the chunks in flight:
    // a status is trusted only for queries bound before its chunk.
    bool streamed = false;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (uint64_t id : running) if (s->tickets[id].kind == 1) streamed = true;
    }
    pc_status dev_rc = PC_OK;
    while (streamed && inflight < 2) {
      const int b = (int)(next_seq & 1);
      const int* ph = nullptr;
      const unsigned long long* qd = nullptr;
      if ((dev_rc = server_engine_run_chunk(s->E, s->tick)) ||
          (dev_rc = server_engine_status(s->E, s->tick, b, &ph, &qd))) break;
      const cudaError_t e = cudaEventRecord(ev[b], s->tick);
      if (e != cudaSuccess) { dev_rc = cuda_fail(e, "server: record tick event"); break; }
      ++next_seq;
      ++inflight;
    }
    if (dev_rc) {
      // the device loop cannot go on: every query still queued or running
      // fails with the CUDA error instead of waiting forever
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto& kv : s->tickets)
        if (kv.second.state == T_PENDING || kv.second.state == T_RUNNING) {
          kv.second.state = T_FAILED;
          kv.second.status = dev_rc;
        }
      s->pending.clear();
      s->stop = true;
      s->cv_done.notify_all();
      break;
    }
    const int* phases = nullptr;
    const unsigned long long* qdone = nullptr;
    uint64_t seen = 0;  // chunk whose status is read this iteration
    bool have_status = false;
    if (inflight > 0) {
      seen = next_seq - (uint64_t)inflight;
      const int b = (int)(seen & 1);
      cudaEventSynchronize(ev[b]);
      phases = s->E ? server_engine_phase_buffer(s->E, b) : nullptr;
      qdone = s->E ? server_engine_qdone_buffer(s->E, b) : nullptr;
      have_status = true;
      --inflight;
    }
    // ---- completions
    std::vector<uint64_t> still;
    for (uint64_t id : running) {
      Ticket* tp;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        tp = &s->tickets[id];
      }
      bool done = false;
      if (tp->kind == 0) done = cudaEventQuery(tp->ev) == cudaSuccess;
      else done = have_status && tp->start_seq <= seen && qdone[tp->qi] >= (unsigned long long)tp->q.n_configs;
      if (done) finish_query(s, id, *tp, tp->kind == 0 ? s->res[tp->stream_idx] : s->copy);
      else still.push_back(id);
    }
    // free slots of queries that have handed back (phase EMPTY) but run on
    if (have_status) {
      std::lock_guard<std::mutex> lk(s->mu);
      for (size_t i = 0; i < s->slot_owner.size(); ++i) {
        const uint64_t o = s->slot_owner[i];
        if (!o || phases[i] != 0) continue;
        auto it = s->tickets.find(o);
        // a slot bound after the chunk was enqueued still reads EMPTY there
        if (it != s->tickets.end() && it->second.start_seq > seen) continue;
        // keep the slot's memory with its query until the query finishes;
        // only the slot index is released for rebinding
        s->slot_owner[i] = 0;
      }
    }
    running.swap(still);
    if (running.empty() && inflight == 0) {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) break;
      if (s->pending.empty()) s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
    } else if (!streamed && inflight == 0) {
      std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
  }
  cudaStreamSynchronize(s->tick);
  for (int b = 0; b < 2; ++b) cudaEventDestroy(ev[b]);
}

}  // namespace
}  // namespace pc

using namespace pc;

extern "C" {

pc_status pc_server_create(const pc_server_opts* opts, pc_server** out) {
  if (!out) { set_error("pc_server_create: out is NULL"); return PC_ERR_ARG; }
  *out = nullptr;
  pc_server_opts o;
  o.hbm_budget_bytes = 8ull << 30;
  o.max_slots = 256;
  o.max_slots_per_query = 64;
  o.ticks_per_poll = 8;
  o.max_pending = 1 << 16;
  o.max_W = 255;
  if (opts) o = *opts;
  if (o.max_W == 0) o.max_W = 255;
  if (o.hbm_budget_bytes < (1u << 20) || o.max_slots < 1 || o.max_slots > 4096 || o.ticks_per_poll < 1 ||
      o.max_pending < 1 || o.max_slots_per_query < 1 || o.max_W < 0 || o.max_W > 255) {
    set_error("pc_server_create: bad options"); return PC_ERR_ARG;
  }
  pc_server* s = new pc_server();
  s->opts = o;
  cudaGetDevice(&s->device);
  cudaError_t e = cudaStreamCreateWithFlags(&s->tick, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
  for (int i = 0; i < kResStreams && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&s->res[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->arena_mem, o.hbm_budget_bytes);
  if (e != cudaSuccess) {
    pc_status rc = cuda_fail(e, "pc_server_create");
    if (s->arena_mem) cudaFree(s->arena_mem);
    if (s->tick) cudaStreamDestroy(s->tick);
    if (s->copy) cudaStreamDestroy(s->copy);
    for (auto r : s->res) if (r) cudaStreamDestroy(r);
    delete s;
    return rc == PC_ERR_CUDA && e == cudaErrorMemoryAllocation ? PC_ERR_OOM : rc;
  }
  s->arena.init(s->arena_mem, o.hbm_budget_bytes);
  const int max_queries = std::min(o.max_slots, 256);
  pc_status rc = server_engine_create(o.max_slots, max_queries, o.ticks_per_poll, o.max_W, s->tick, &s->E);
  if (rc) {
    cudaFree(s->arena_mem);
    cudaStreamDestroy(s->tick);
    cudaStreamDestroy(s->copy);
    for (auto r : s->res) cudaStreamDestroy(r);
    delete s;
    return rc;
  }
  s->slot_owner.assign(server_engine_slots(s->E), 0);
  s->query_owner.assign(max_queries, 0);
  s->worker = std::thread(worker_main, s);
  *out = s;
  return PC_OK;
}

pc_status pc_server_submit(pc_server* s, const pc_query* q, uint64_t* ticket) {
  if (!s || !q || !ticket) { set_error("pc_server_submit: NULL argument"); return PC_ERR_ARG; }
  if (q->W < 0 || q->W > 255 || q->L < 1 || q->L >= (1 << 24) ||
      (n_columns(q->W) + 1) * ((int64_t)q->L + 2) >= ((int64_t)1 << 31)) {
    set_error("pc_server_submit: bad W or L"); return PC_ERR_ARG;
  }
  if (!(q->p >= 0.0 && q->p <= 1.0) || q->n_configs < 1 || q->config_begin < 0 ||
      q->config_begin + q->n_configs > ((int64_t)1 << 32)) {
    set_error("pc_server_submit: bad p or configuration range"); return PC_ERR_ARG;
  }
  size_t need = out_bytes(q->n_configs);
  if (!resident_fits(q->W, q->L)) {
    if (q->W > s->opts.max_W) { set_error("pc_server_submit: lattice wider than the server's max_W"); return PC_ERR_ARG; }
    need += stream_slot_bytes(q->W, q->L) + 256;
  }
  if (need > s->opts.hbm_budget_bytes) {
    set_error("pc_server_submit: footprint exceeds the server's HBM budget"); return PC_ERR_OOM;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) { set_error("pc_server_submit: server is shutting down"); return PC_ERR_CANCELLED; }
  if ((int64_t)s->pending.size() >= s->opts.max_pending) { set_error("pc_server_submit: queue full"); return PC_ERR_BUSY; }
  const uint64_t id = s->next_ticket++;
  Ticket& t = s->tickets[id];
  t.q = *q;
  t.t_submit = Clock::now();
  if (!s->any) { s->any = true; s->t_first = t.t_submit; }
  s->submitted += 1;
  s->pending.push_back(id);
  *ticket = id;
  s->cv_work.notify_one();
  return PC_OK;
}

pc_status pc_server_poll(pc_server* s, uint64_t ticket, pc_result* out, int64_t timeout_ns) {
  if (!s) { set_error("pc_server_poll: NULL server"); return PC_ERR_ARG; }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) { set_error("pc_server_poll: unknown ticket"); return PC_ERR_ARG; }
  auto ready = [&] {
    const TicketState st = s->tickets[ticket].state;
    return st == T_DONE || st == T_FAILED || st == T_CANCELLED;
  };
  if (!ready()) {
    if (timeout_ns > 0) s->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), ready);
    if (!ready()) { set_error("pc_server_poll: not finished"); return PC_ERR_BUSY; }
  }
  Ticket& t = s->tickets[ticket];
  const pc_status st = t.state == T_DONE ? PC_OK : t.state == T_CANCELLED ? PC_ERR_CANCELLED : t.status;
  if (st == PC_ERR_CANCELLED) set_error("pc_server_poll: query cancelled");
  if (out && t.state == T_DONE) *out = t.result;
  s->tickets.erase(ticket);
  return st;
}

pc_status pc_server_cancel(pc_server* s, uint64_t ticket) {
  if (!s) { set_error("pc_server_cancel: NULL server"); return PC_ERR_ARG; }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) { set_error("pc_server_cancel: unknown ticket"); return PC_ERR_ARG; }
  if (it->second.state != T_PENDING) { set_error("pc_server_cancel: query already running"); return PC_ERR_BUSY; }
  it->second.state = T_CANCELLED;
  s->cv_done.notify_all();
  return PC_OK;
}

pc_status pc_server_get_stats(pc_server* s, pc_server_stats* out) {
  if (!s || !out) { set_error("pc_server_get_stats: NULL argument"); return PC_ERR_ARG; }
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->configs_completed = s->configs_done;
  std::vector<double> l = s->lat_ms;
  std::sort(l.begin(), l.end());
  auto pct = [&](double f) -> double {
    if (l.empty()) return 0.0;
    size_t i = (size_t)(f * (double)(l.size() - 1) + 0.5);
    return l[std::min(i, l.size() - 1)];
  };
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  double sum = 0;
  for (double v : l) sum += v;
  out->mean_ms = l.empty() ? 0.0 : sum / (double)l.size();
  const double span = s->completed ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
  out->configs_per_s = span > 0 ? (double)s->configs_done / span : 0.0;
  return PC_OK;
}

pc_status pc_server_destroy(pc_server* s) {
  if (!s) return PC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (uint64_t id : s->pending) {
      auto& t = s->tickets[id];
      if (t.state == T_PENDING) t.state = T_CANCELLED;
    }
    s->pending.clear();
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->tick);
  for (auto r : s->res) cudaStreamSynchronize(r);
  for (auto& kv : s->tickets) if (kv.second.ev) cudaEventDestroy(kv.second.ev);
  server_engine_destroy(s->E);
  cudaFree(s->arena_mem);
  cudaStreamDestroy(s->tick);
  cudaStreamDestroy(s->copy);
  for (auto r : s->res) cudaStreamDestroy(r);
  delete s;
  return PC_OK;
}

}  // extern "C"

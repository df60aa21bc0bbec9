// kernels.cuh -- launch interfaces between the C-ABI layer and the kernels.
#pragma once

#include "common.cuh"

namespace pc {

// Outputs of one inspection call (device pointers; optional ones may be null).
struct Outputs {
  uint8_t* verdict;
  int32_t* first_hit;
  float* mass;
  int32_t* m_stop;
  unsigned long long* n_perc;  // atomically incremented per percolating config
};

// Resident (shared-memory) solver, resident.cu.
struct ResidentArgs {
  Lattice lat;
  OccStream occ;             // occupancy stream (cfg field set per config)
  const uint32_t* occ_bits;  // caller occupancy [n_cfg][words_per_cfg] or null
  int64_t words_per_cfg;
  int64_t n_cfg;
  uint32_t cfg0;
  uint8_t* verdict;
  int32_t* first_hit;
  float* mass;
  int32_t* m_stop;
  unsigned long long* n_perc;
  unsigned long long* work;  // zeroed work counter
  int prep_chunk;            // layers prepared per lazy chunk (>= 3)
  int bits_only = 0;         // reached set only: no FP32 sweep, mass written 0
  int verdict_first = 0;     // reached set first, FP32 recursion only where it percolates
};
constexpr int kResidentMaxThreads = 640;  // resident CTA size limit: 20 warps at <= 96 registers
// Several queries in one persistent resident launch (device pointers): the
// configurations of query q are the items [item0[q], item0[q + 1]) of one
// list, counted by *work (zeroed).  Every query's own work field is unused.
struct ResidentBatch {
  const ResidentArgs* qs;   // [nq]
  const long long* item0;   // [nq + 1]
  int nq;
  unsigned long long* work;
};
size_t resident_smem(const Lattice& lat);
pc_status launch_resident(const ResidentArgs& args, int threads, cudaStream_t st);
pc_status resident_add_node(const ResidentArgs& args, int threads, cudaGraph_t g,
                            const cudaGraphNode_t* deps, size_t ndeps, cudaGraphNode_t* out);
// One persistent launch over several queries (graph node): dynamic shared
// memory smem (the largest query's), grid = CTAs that fit x SMs, capped at
// the item count.
pc_status resident_multi_add_node(const ResidentBatch& b, long long n_items, size_t smem, int threads,
                                  cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                                  cudaGraphNode_t* out);
// default CTA size of the resident solver (about 16 tube layers per thread)
int resident_threads(int A, int L);
// CTA size picked by the autotuner for (W, L, p bin) (batch.cu); times
// candidates on a miss, outside any stream capture
int tuned_threads(const Lattice& lat, double p, uint64_t seed, cudaStream_t st);
bool resident_fits(int W, int L);
void release_batches();
void release_static();  // noalloc.cu: forget the static array's cached addresses

// Streamed solver for lattices beyond shared memory, stream.cu.
struct StreamQuery {
  Lattice lat;
  OccStream occ;
  const uint32_t* occ_bits;
  int64_t words_per_cfg;
  int64_t n_cfg;
  uint32_t cfg0;
  Outputs out;
  int bits_only = 0;  // reached set only: no FP units, mass written 0
  // device list of n_cfg configurations (indices from 0 within the query) to
  // solve, outputs written at those indices; null = configurations 0..n_cfg-1
  const int64_t* sel = nullptr;
};
struct StreamJob : StreamQuery {
  int* error_out = nullptr;  // device int: 1 if the tick bound was hit
};
struct StreamPlan;
// Device resources for a set of queries (stream-ordered allocation on st).
pc_status stream_plan_create(const StreamQuery* qs, int nq, cudaStream_t st, StreamPlan** out);
// Adds [init -> WHILE(sweep, control)] to g after deps; *last = the WHILE node.
pc_status stream_plan_add(StreamPlan* P, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                          cudaGraphNode_t* last);
int* stream_plan_error(StreamPlan* P);
void stream_plan_release(StreamPlan* P, cudaStream_t st);
size_t stream_slot_bytes(int W, int L);
pc_status run_stream(const StreamJob& job, cudaStream_t st);
// PC_VERDICT_FIRST on the streamed path: a verdict-only solve of every
// configuration, then the full solve of the percolating ones (the host waits
// for the first to count them).
pc_status run_stream_verdict_first(const StreamJob& job, cudaStream_t st);
// Verdict-only solver with temporal blocking (blocked.cu): runs a PC_BITS_ONLY
// job when a thread-block cluster holds the lattice's cross-section
// (*handled = true), else leaves it to the step-synchronous solver.
pc_status run_blocked(const StreamJob& job, cudaStream_t st, bool* handled);
// Whether run_blocked takes PC_BITS_ONLY jobs of this lattice on this device.
bool blocked_takes(const Lattice& lat);

// Server engine (stream.cu): streamed-solver slots bound to queries by the host.
struct ServerEngine;
pc_status server_engine_create(int max_slots, int max_queries, int ticks_per_chunk, int max_W,
                               cudaStream_t st, ServerEngine** out);
void server_engine_destroy(ServerEngine* E);
int server_engine_slots(const ServerEngine* E);
pc_status server_engine_set_query(ServerEngine* E, int qi, const StreamQuery& q, cudaStream_t st);
pc_status server_engine_bind(ServerEngine* E, const int* slots, const int* queries, char* const* bases,
                             int n, cudaStream_t st);
pc_status server_engine_run_chunk(ServerEngine* E, cudaStream_t st);
// Enqueue a status read into host buffer buf (0 or 1): slot phases and
// per-query completion counts; the buffers are valid once the stream passes.
pc_status server_engine_status(ServerEngine* E, cudaStream_t st, int buf, const int** phases,
                               const unsigned long long** qdone);
const int* server_engine_phase_buffer(const ServerEngine* E, int buf);
const unsigned long long* server_engine_qdone_buffer(const ServerEngine* E, int buf);

// Standalone occupancy draw, occupancy.cu.
pc_status launch_occupancy(const Lattice& lat, const OccStream& os, uint32_t cfg0,
                           int64_t n_cfg, uint32_t* occ_bits, cudaStream_t st);
// Fixed-count occupancy (exactly n_metallic sites per configuration); waits
// for its own work on st (a convergence check).
pc_status launch_occupancy_fixed(const Lattice& lat, const OccStream& os, uint32_t cfg0, int64_t n_cfg,
                                 int64_t n_metallic, uint32_t* occ_bits, cudaStream_t st);

}  // namespace pc

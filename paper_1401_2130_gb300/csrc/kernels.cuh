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
};
size_t resident_smem(int A, int L);
pc_status launch_resident(const ResidentArgs& args, int threads, cudaStream_t st);

// Streamed solver for lattices beyond shared memory, stream.cu.
struct StreamJob {
  Lattice lat;
  OccStream occ;
  const uint32_t* occ_bits;
  int64_t words_per_cfg;
  int64_t n_cfg;
  uint32_t cfg0;
  Outputs out;
};
pc_status run_stream(const StreamJob& job, cudaStream_t st);

// Standalone occupancy draw, occupancy.cu.
pc_status launch_occupancy(const Lattice& lat, const OccStream& os, uint32_t cfg0,
                           int64_t n_cfg, uint32_t* occ_bits, cudaStream_t st);

}  // namespace pc

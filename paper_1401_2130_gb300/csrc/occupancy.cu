// occupancy.cu -- bit-packed occupancy of whole configurations (Sec. II.A:
// each site metallic with probability p), drawn from the Philox4x32-10
// stream.  One thread per output word: the 8 Philox blocks of 4 sites that
// make up 32 consecutive sites.  Integer ALU bound; written coalesced.
#include "common.cuh"
#include "kernels.cuh"

namespace pc {

__global__ void occupancy_kernel(OccStream os, uint32_t cfg0, int64_t n_cfg, int64_t N,
                                 int64_t wpc, uint32_t* __restrict__ out) {
  const int64_t total = n_cfg * wpc;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = g / wpc, w = g - c * wpc;
    OccStream s = os;
    s.cfg = cfg0 + (uint32_t)c;
    uint32_t word = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) word |= s.block_bits((uint32_t)(w * 8 + b)) << (4 * b);
    const int64_t first = w * 32;  // clear the bits past the last site
    if (first + 32 > N) word &= (N - first >= 32) ? 0xffffffffu : ((1u << (N - first)) - 1u);
    out[g] = word;
  }
}

pc_status launch_occupancy(const Lattice& lat, const OccStream& os, uint32_t cfg0,
                           int64_t n_cfg, uint32_t* occ_bits, cudaStream_t st) {
  const int64_t wpc = (lat.N + 31) / 32;
  const int64_t total = n_cfg * wpc;
  if (total <= 0) return PC_OK;
  int dev = 0, nsm = 0;
  PC_CUDA(cudaGetDevice(&dev));
  PC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  const int64_t cap = (int64_t)nsm * 8;
  if (blocks > cap) blocks = cap;
  occupancy_kernel<<<(unsigned)blocks, threads, 0, st>>>(os, cfg0, n_cfg, lat.N, wpc, occ_bits);
  PC_CUDA(cudaGetLastError());
  return PC_OK;
}

}  // namespace pc

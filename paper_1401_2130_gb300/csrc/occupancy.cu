// occupancy.cu -- bit-packed occupancy of whole configurations (Sec. II.A:
// each site metallic with probability p), drawn from the Philox4x32-10
// stream.  One thread per output word: the 8 Philox blocks of 4 sites that
// make up 32 consecutive sites.  Integer ALU bound; written coalesced.
#include <algorithm>

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

// ---------------------------------------------------------------------------
// Fixed-count occupancy (Sec. II.A: a random permutation of the N sites puts
// exactly Np of them metallic).  Site i carries the key (u_i << 32) | i, u_i
// its 32-bit word of the same Philox stream as the Bernoulli draw; the
// metallic sites are the Np smallest keys.  The Np-th smallest key is found
// per configuration by radix selection, 8 bits per pass from the top: a pass
// histograms the next digit of the keys that share the prefix found so far,
// and the selection step descends into the bin that holds the wanted rank.
// A configuration is resolved as soon as that bin holds a single key (keys
// are unique, so at most 8 passes).  Each pass recomputes the words from the
// stream instead of storing N keys per configuration.
// ---------------------------------------------------------------------------
namespace {

struct FcState {
  uint64_t prefix;  // high bits of the wanted key found so far
  int64_t rank;     // rank of the wanted key among the keys with that prefix
  int shift;        // bits below the prefix (64: no prefix yet)
  int resolved;     // 1: exactly one key has the prefix; -1: Np = 0 (no site)
};

__device__ __forceinline__ uint64_t fc_key(uint32_t u, int64_t i) { return ((uint64_t)u << 32) | (uint64_t)i; }

__global__ void fc_init_kernel(FcState* st, int64_t n_cfg, int64_t n_metallic) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cfg) return;
  FcState s;
  s.prefix = 0; s.shift = 64; s.rank = n_metallic - 1; s.resolved = n_metallic > 0 ? 0 : -1;
  st[c] = s;
}

// Histogram of the next 8-bit digit of the keys sharing the prefix.
__global__ void __launch_bounds__(256) fc_hist_kernel(OccStream os, uint32_t cfg0, int64_t n_cfg, int64_t N,
                                                      const FcState* __restrict__ st,
                                                      unsigned int* __restrict__ hist) {
  __shared__ unsigned int h[256];
  const int64_t nblk = (N + 3) / 4;
  for (int64_t c = blockIdx.y; c < n_cfg; c += gridDim.y) {
    const FcState s = st[c];
    if (s.resolved) continue;  // block-uniform
    for (int k = threadIdx.x; k < 256; k += blockDim.x) h[k] = 0u;
    __syncthreads();
    const int dshift = s.shift - 8;
    const uint32_t cfg = cfg0 + (uint32_t)c;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk;
         b += (int64_t)gridDim.x * blockDim.x) {
      const u32x4 r = philox4x32_10(u32x4{(uint32_t)b, cfg, os.wl, 0u}, os.k0, os.k1);
      const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t i = 4 * b + j;
        if (i >= N) break;
        const uint64_t key = fc_key(u[j], i);
        if (s.shift < 64 && (key >> s.shift) != s.prefix) continue;
        atomicAdd(&h[(key >> dshift) & 255u], 1u);
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 256; k += blockDim.x)
      if (h[k]) atomicAdd(&hist[c * 256 + k], h[k]);
    __syncthreads();
  }
}

// One warp per configuration: descend into the bin holding the wanted rank.
__global__ void fc_select_kernel(FcState* st, unsigned int* hist, int64_t n_cfg) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= n_cfg) return;
  FcState s = st[c];
  unsigned int* h = hist + c * 256;
  if (s.resolved) return;  // warp-uniform
  unsigned int v[8], sum = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) { v[k] = h[lane * 8 + k]; sum += v[k]; }
  // exclusive prefix of the per-lane sums
  unsigned int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  unsigned int run = incl - sum;
  int found = -1;
  unsigned int below = 0, cnt = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (found < 0 && (int64_t)run <= s.rank && s.rank < (int64_t)(run + v[k])) {
      found = lane * 8 + k; below = run; cnt = v[k];
    }
    run += v[k];
  }
  const unsigned int owner = __ballot_sync(0xffffffffu, found >= 0);
  const int src = owner ? __ffs(owner) - 1 : 0;
  found = __shfl_sync(0xffffffffu, found, src);
  below = __shfl_sync(0xffffffffu, below, src);
  cnt = __shfl_sync(0xffffffffu, cnt, src);
#pragma unroll
  for (int k = 0; k < 8; ++k) h[lane * 8 + k] = 0u;  // ready for the next pass
  if (lane == 0) {
    if (found < 0) {  // cannot happen: the ranks of the histogram cover rank
      s.resolved = 2;
    } else {
      s.prefix = (s.shift < 64 ? (s.prefix << 8) : 0ull) | (uint64_t)found;
      s.shift -= 8;
      s.rank -= below;
      if (cnt == 1 || s.shift == 0) s.resolved = 1;
    }
    st[c] = s;
  }
}

// Occupancy words: site metallic iff its key is among the Np smallest, i.e.
// key >> shift <= prefix (exactly one key has the prefix itself).
__global__ void fc_write_kernel(OccStream os, uint32_t cfg0, int64_t n_cfg, int64_t N, int64_t wpc,
                                const FcState* __restrict__ st, uint32_t* __restrict__ out,
                                int* __restrict__ error) {
  const int64_t total = n_cfg * wpc;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = g / wpc, w = g - c * wpc;
    const FcState s = st[c];
    uint32_t word = 0;
    if (s.resolved == 1) {
      const uint32_t cfg = cfg0 + (uint32_t)c;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int64_t blk = w * 8 + b;
        const u32x4 r = philox4x32_10(u32x4{(uint32_t)blk, cfg, os.wl, 0u}, os.k0, os.k1);
        const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int64_t i = 4 * blk + j;
          if (i < N && (fc_key(u[j], i) >> s.shift) <= s.prefix) word |= 1u << (4 * b + j);
        }
      }
    } else if (s.resolved != -1 && w == 0) {
      atomicOr(error, 1);  // the selection did not converge (never expected)
    }
    out[g] = word;
  }
}

}  // namespace

pc_status launch_occupancy_fixed(const Lattice& lat, const OccStream& os, uint32_t cfg0, int64_t n_cfg,
                                 int64_t n_metallic, uint32_t* occ_bits, cudaStream_t st) {
  const int64_t wpc = (lat.N + 31) / 32;
  if (n_cfg <= 0) return PC_OK;
  int dev = 0, nsm = 0;
  PC_CUDA(cudaGetDevice(&dev));
  PC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  char* mem = nullptr;
  const size_t st_bytes = ((size_t)n_cfg * sizeof(FcState) + 255) & ~(size_t)255;
  const size_t bytes = st_bytes + (size_t)n_cfg * 256 * sizeof(unsigned int) + 256;
  PC_CUDA(cudaMallocAsync((void**)&mem, bytes, st));
  FcState* s = (FcState*)mem;
  unsigned int* hist = (unsigned int*)(mem + st_bytes);
  int* error = (int*)(mem + bytes - 256);
  pc_status rc = PC_OK;
  do {
    cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)n_cfg * 256 * sizeof(unsigned int) + 256, st);
    if (e != cudaSuccess) { rc = cuda_fail(e, "fixed-count scratch"); break; }
    fc_init_kernel<<<(unsigned)((n_cfg + 255) / 256), 256, 0, st>>>(s, n_cfg, n_metallic);
    // site blocks per CTA row: enough CTAs to fill the device across configurations
    const int64_t nblk = (lat.N + 3) / 4;
    const int64_t gy = std::min<int64_t>(n_cfg, 65535);
    int64_t gx = (nblk + 255) / 256;
    const int64_t want = std::max<int64_t>(1, (int64_t)nsm * 8 / gy);
    if (gx > want) gx = want;
    for (int pass = 0; pass < 8; ++pass) {
      fc_hist_kernel<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(os, cfg0, n_cfg, lat.N, s, hist);
      fc_select_kernel<<<(unsigned)((n_cfg * 32 + 255) / 256), 256, 0, st>>>(s, hist, n_cfg);
    }
    const int64_t total = n_cfg * wpc;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)nsm * 8) blocks = (int64_t)nsm * 8;
    fc_write_kernel<<<(unsigned)blocks, 256, 0, st>>>(os, cfg0, n_cfg, lat.N, wpc, s, occ_bits, error);
    if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_fail(e, "fixed-count kernels"); break; }
    int err = 0;
    if ((e = cudaMemcpyAsync(&err, error, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      rc = cuda_fail(e, "fixed-count check"); break;
    }
    if (err) { set_error("fixed-count selection did not converge"); rc = PC_ERR_INTERNAL; }
  } while (0);
  cudaFreeAsync(mem, st);
  return rc;
}

}  // namespace pc

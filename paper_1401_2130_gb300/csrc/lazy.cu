// lazy.cu -- the lazy walk of the self-loop remark in Sec. II.B.
//
// Staying on the current site with probability s at every step, i.e. the
// chain s I + (1 - s) P, does not change whether the detector is ever
// reached, nor the first step at which it can be (the shortest spanning
// path needs a move at every step).  The probability of arriving exactly at
// that first step is the plain one times (1 - s)^first_hit, since each of the
// first_hit moves now happens with probability 1 - s.  So the variant's
// outputs come from the plain inspection's: verdicts, first_hit and m_stop
// unchanged, mass scaled here on the device.
#include "common.cuh"

namespace pc {
namespace {

__global__ void lazy_mass_kernel(const int32_t* __restrict__ first_hit, const float* __restrict__ mass,
                                 int64_t n, double keep, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t m = first_hit[i];
    out[i] = m > 0 ? (float)((double)mass[i] * pow(keep, (double)m)) : 0.f;
  }
}

pc_status launch_lazy_mass(const int32_t* fh, const float* mass, int64_t n, double keep, float* out,
                           cudaStream_t st) {
  int dev = 0, sms = 0;
  PC_CUDA(cudaGetDevice(&dev));
  PC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t want = (n + 255) / 256, cap = (int64_t)sms * 8;
  const int blocks = (int)(want < cap ? want : cap);
  lazy_mass_kernel<<<blocks, 256, 0, st>>>(fh, mass, n, keep, out);
  PC_CUDA(cudaGetLastError());
  return PC_OK;
}

}  // namespace
}  // namespace pc

using namespace pc;

extern "C" pc_status pc_lazy_mass(const int32_t* first_hit, const float* mass, int64_t n_configs,
                                  double hold, float* mass_lazy, int32_t flags, void* cuda_stream) {
  NvtxRange nvtx_("pc_lazy_mass");
  if (flags & ~PC_OUT_DEVICE) { set_error("pc_lazy_mass: unknown flag bits"); return PC_ERR_ARG; }
  if (!(hold >= 0.0 && hold < 1.0)) { set_error("pc_lazy_mass: hold must be in [0, 1)"); return PC_ERR_ARG; }
  if (n_configs < 0) { set_error("pc_lazy_mass: n_configs must be >= 0"); return PC_ERR_ARG; }
  if (n_configs == 0) return PC_OK;
  if (!first_hit || !mass || !mass_lazy) { set_error("pc_lazy_mass: NULL buffer"); return PC_ERR_ARG; }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double keep = 1.0 - hold;
  if (flags & PC_OUT_DEVICE) return launch_lazy_mass(first_hit, mass, n_configs, keep, mass_lazy, st);
  // host buffers: stage through one stream-ordered device allocation
  const size_t b4 = (size_t)n_configs * 4;
  char* d = nullptr;
  PC_CUDA(cudaMallocAsync((void**)&d, 3 * b4, st));
  int32_t* dfh = (int32_t*)d;
  float* dm = (float*)(d + b4);
  float* dout = (float*)(d + 2 * b4);
  pc_status rc = PC_OK;
  cudaError_t e = cudaMemcpyAsync(dfh, first_hit, b4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dm, mass, b4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) rc = cuda_fail(e, "pc_lazy_mass: copy in");
  if (rc == PC_OK) rc = launch_lazy_mass(dfh, dm, n_configs, keep, dout, st);
  if (rc == PC_OK) {
    e = cudaMemcpyAsync(mass_lazy, dout, b4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "pc_lazy_mass: copy out");
  }
  const cudaError_t fe = cudaFreeAsync(d, st);
  if (rc == PC_OK && fe != cudaSuccess) rc = cuda_fail(fe, "pc_lazy_mass: free");
  return rc;
}

// resident.cu -- shared-memory resident solver for lattices that fit in one
// CTA's shared memory (Sec. II.B, Eqs. (2)-(4) on the lattice of Sec. II.A).
//
// A persistent CTA pulls configurations from a work counter and keeps the
// whole state of one configuration in shared memory for its entire solve:
//   nu[2][(L+2) x S] FP32 : nu(i) = mu(i) / deg(i), the mass each site sends
//                           along each of its edges (ping-pong, rows t+1;
//                           rows 0 and L+1 and column A are always zero)
//   cf[L x S]        FP32 : 1/deg(i) for metallic sites, 0 otherwise
//   occw, R[2]       bits : occupancy and reached set; word (tw, a) holds the
//                           32 tube indices 32*tw .. 32*tw+31 of column a,
//                           stored row-major [tw + 1][a] (one zero pad row of
//                           words at each end, column A always zero)
// One step m of Eq. (3) in forward form, over the causal window t <= m:
//   mu_m(j) = sum over the 14 lattice neighbours i of j of nu_{m-1}(i)
//   nu_m(j) = cf(j) * mu_m(j)                         (Jacobi, FP32)
//   R_m     = R_{m-1} | (N(R_{m-1}) & occ)            (exact, bit-parallel)
// The verdict is decided by R only, so FP32 underflow cannot change it.  If a
// site of the end layer t = L-1 enters R at step m, the detector probability
// first becomes non-zero at step m+1 and equals sum_{t=L-1} nu_m (each end
// site sends nu along its detector edge).  If R does not grow, the
// configuration does not percolate.
// Layers are prepared lazily, a chunk at a time, as the window reaches them:
// occupancy drawn from the Philox stream (or read from caller bits), degrees
// and 1/deg computed, nu rows zeroed.  Layers the window never reaches are
// never drawn: their occupancy cannot influence any output.
#include "common.cuh"
#include "kernels.cuh"

namespace pc {

namespace {

constexpr uint32_t kGrow = 1u, kEnd = 2u;

struct Smem {
  float* nu[2];
  float* cf;
  uint32_t* occw;
  uint32_t* R[2];
  int16_t* nbr;
  int8_t* sig;
  uint32_t* flags;  // [3]
  float* redf;      // [32]
  long long* redi;  // [32]
  long long* scal;  // [4]
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t resident_smem_bytes(int A, int L) {
  const size_t S = (size_t)A + 1, TWP = (size_t)(L + 31) / 32 + 2;
  size_t b = 0;
  b += 2 * align16(sizeof(float) * (size_t)(L + 2) * S);
  b += align16(sizeof(float) * (size_t)L * S);
  b += 3 * align16(sizeof(uint32_t) * S * TWP);
  b += align16(sizeof(int16_t) * (size_t)A * kLateral);
  b += align16((size_t)A);
  b += align16(sizeof(uint32_t) * 4) + align16(sizeof(float) * 32) +
       align16(sizeof(long long) * 32) + align16(sizeof(long long) * 4);
  return b;
}

__device__ inline Smem carve(unsigned char* base, int A, int L) {
  const size_t S = (size_t)A + 1, TWP = (size_t)(L + 31) / 32 + 2;
  Smem s;
  size_t o = 0;
  auto take = [&](size_t bytes) { unsigned char* p = base + o; o += align16(bytes); return p; };
  s.nu[0] = (float*)take(sizeof(float) * (size_t)(L + 2) * S);
  s.nu[1] = (float*)take(sizeof(float) * (size_t)(L + 2) * S);
  s.cf = (float*)take(sizeof(float) * (size_t)L * S);
  s.occw = (uint32_t*)take(sizeof(uint32_t) * S * TWP);
  s.R[0] = (uint32_t*)take(sizeof(uint32_t) * S * TWP);
  s.R[1] = (uint32_t*)take(sizeof(uint32_t) * S * TWP);
  s.nbr = (int16_t*)take(sizeof(int16_t) * (size_t)A * kLateral);
  s.sig = (int8_t*)take((size_t)A);
  s.flags = (uint32_t*)take(sizeof(uint32_t) * 4);
  s.redf = (float*)take(sizeof(float) * 32);
  s.redi = (long long*)take(sizeof(long long) * 32);
  s.scal = (long long*)take(sizeof(long long) * 4);
  return s;
}

// Deterministic block reductions (fixed tree for a fixed block size).
__device__ inline float block_sum_f(float v, float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  if (warp == 0) {
    s = lane < nw ? red[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

__device__ inline long long block_sum_i(long long v, long long* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  long long s = 0;
  if (warp == 0) {
    s = lane < nw ? red[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// bit of a word array [tw + 1][S]: column col, tube tt (tt = -1 and tt >= L
// land in zero padding)
__device__ inline uint32_t bit_at(const uint32_t* w, int S, int col, int tt) {
  return (w[((tt >> 5) + 1) * S + col] >> (tt & 31)) & 1u;
}

// Word of R at tube offset dt, aligned to the word tw of the caller:
// bit b of the result = R(col, 32*tw + b + dt).
__device__ inline uint32_t shifted_word(const uint32_t* R, int S, int col, int tw, int dt) {
  const uint32_t w = R[(tw + 1) * S + col];
  if (dt == 0) return w;
  if (dt > 0) return (w >> 1) | (R[(tw + 2) * S + col] << 31);
  return (w << 1) | (R[tw * S + col] >> 31);
}

}  // namespace

size_t resident_smem(int A, int L) { return resident_smem_bytes(A, L); }

// One FP32 site-update sweep of unit (column a, phase ph) over t = ph, ph+P, ..
// up to tmax: nu_dst(a,t) = cf(a,t) * [nu(a,t-1) + nu(a,t+1) + sum_d nu(n_d, t+dt_d)]
__device__ __forceinline__ void sweep_unit(const float* __restrict__ src, float* __restrict__ dst,
                                           const float* __restrict__ cf, int a, int ph, int P,
                                           int tmax, int S, const int (&off)[kLateral]) {
  for (int t = ph; t <= tmax; t += P) {
    const int base = (t + 1) * S;
    float s = src[base - S + a] + src[base + S + a];
#pragma unroll
    for (int d = 0; d < kLateral; ++d) s += src[base + off[d]];
    dst[base + a] = cf[t * S + a] * s;
  }
}

// Lazy preparation of layers [F, Fnew): occupancy drawn up to layer Fnew (for
// the degrees of layer Fnew - 1), 1/deg of each site (Eq. (2); the detector
// edge adds one on t = L-1), nu rows zeroed in both buffers.  Block-uniform.
__device__ __forceinline__ void prepare_layers(const Smem& sm, const ResidentArgs& P, const OccStream& os,
                                            const uint32_t* cbits, int A, int L, int S,
                                            int& G, int& F, int Fnew) {
  const int tid = threadIdx.x, T = blockDim.x;
  const int Gnew = min(Fnew + 1, L);
  if (Gnew > G) {
    // resident lattices have N < 2^31: 32-bit site arithmetic
    const int i0 = G * A, i1 = Gnew * A;
    if (cbits) {
      const int w0 = i0 >> 5, w1 = (i1 - 1) >> 5;
      for (int wi = w0 + tid; wi <= w1; wi += T) {
        uint32_t w = cbits[wi];
        while (w) {
          const int b = __ffs(w) - 1;
          w &= w - 1;
          const int i = (wi << 5) + b;
          if (i < i0 || i >= i1) continue;
          const int t = i / A, a = i - t * A;
          atomicOr(&sm.occw[((t >> 5) + 1) * S + a], 1u << (t & 31));
        }
      }
    } else {
      const int b0 = i0 >> 2, b1 = (i1 - 1) >> 2;
      for (int bi = b0 + tid; bi <= b1; bi += T) {
        uint32_t bits = os.block_bits((uint32_t)bi);
        while (bits) {
          const int j = __ffs(bits) - 1;
          bits &= bits - 1;
          const int i = (bi << 2) + j;
          if (i < i0 || i >= i1) continue;
          const int t = i / A, a = i - t * A;
          atomicOr(&sm.occw[((t >> 5) + 1) * S + a], 1u << (t & 31));
        }
      }
    }
    G = Gnew;
    __syncthreads();
  }
  const int n = (Fnew - F) * S;
  for (int k = tid; k < n; k += T) {
    const int t = F + k / S, a = k % S;
    float c = 0.f;
    if (a < A && bit_at(sm.occw, S, a, t)) {
      const int sg = sm.sig[a];
      int deg = (int)bit_at(sm.occw, S, a, t - 1) + (int)bit_at(sm.occw, S, a, t + 1) + (t == L - 1);
#pragma unroll
      for (int d = 0; d < kLateral; ++d)
        deg += (int)bit_at(sm.occw, S, sm.nbr[a * kLateral + d], t + dir_dt(d, sg));
      c = deg ? __frcp_rn((float)deg) : 0.f;
    }
    sm.cf[t * S + a] = c;
    sm.nu[0][(t + 1) * S + a] = 0.f;
    sm.nu[1][(t + 1) * S + a] = 0.f;
  }
  F = Fnew;
  __syncthreads();
}

template <bool kOneUnit>
__global__ void __launch_bounds__(1024, 1) resident_kernel(ResidentArgs P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Lattice& lat = P.lat;
  const int A = lat.A, L = lat.L, S = lat.S, TWP = lat.TWP;
  const int tid = threadIdx.x, T = blockDim.x;
  Smem sm = carve(smem_raw, A, L);

  // tables into shared memory; zero the padding rows of nu
  // resident lattices have A < 2^15 (checked by the launcher): int16 in shared memory
  for (int k = tid; k < A * kLateral; k += T) sm.nbr[k] = (int16_t)lat.nbr[k];
  for (int k = tid; k < A; k += T) sm.sig[k] = lat.sigma[k];
  for (int k = tid; k < S; k += T) {
    sm.nu[0][k] = 0.f; sm.nu[1][k] = 0.f;
    sm.nu[0][(L + 1) * S + k] = 0.f; sm.nu[1][(L + 1) * S + k] = 0.f;
  }
  __syncthreads();

  // FP unit mapping: P_ph phases of A columns
  const int Pph = T >= A ? T / A : 1;
  const int n_units = A * Pph;
  int my_off[kLateral];
  int my_a = 0, my_ph = 0;
  if (kOneUnit && tid < n_units) {
    my_a = tid % A; my_ph = tid / A;
    const int sg = sm.sig[my_a];
#pragma unroll
    for (int d = 0; d < kLateral; ++d)
      my_off[d] = dir_dt(d, sg) * S + sm.nbr[my_a * kLateral + d];
  }

  const int CH = P.prep_chunk;
  const int n_words_col = S * TWP;

  for (;;) {
    if (tid == 0) sm.scal[0] = (long long)atomicAdd(P.work, 1ull);
    __syncthreads();
    const long long rel = sm.scal[0];
    if (rel >= P.n_cfg) break;
    const uint32_t cfg = P.cfg0 + (uint32_t)rel;

    // reset bit arrays and flags
    for (int k = tid; k < n_words_col; k += T) { sm.occw[k] = 0u; sm.R[0][k] = 0u; sm.R[1][k] = 0u; }
    if (tid < 3) sm.flags[tid] = 0u;
    __syncthreads();

    int G = 0, F = 0;  // layers with occupancy drawn / with cf + zeroed nu
    OccStream os = P.occ;
    os.cfg = cfg;
    const uint32_t* cbits = P.occ_bits ? P.occ_bits + (size_t)rel * P.words_per_cfg : nullptr;

    prepare_layers(sm, P, os, cbits, A, L, S, G, F, min(max(CH, 3), L));

    // ---- m = 0: start distribution on the metallic sites of t = 0 ----
    long long my_n0 = 0;
    for (int a = tid; a < A; a += T) {
      const uint32_t b = sm.occw[S + a] & 1u;
      sm.R[0][S + a] = b;
      my_n0 += b;
    }
    const long long n0 = block_sum_i(my_n0, sm.redi);
    int verdict = 0, fh = -1, mstop = 0;
    float mass = 0.f;
    if (n0 > 0) {
      const float inv_n0 = __frcp_rn((float)n0);
      for (int a = tid; a < A; a += T)
        sm.nu[0][S + a] = (sm.occw[S + a] & 1u) ? sm.cf[a] * inv_n0 : 0.f;
      __syncthreads();
      if (L == 1) {
        float part = 0.f;
        for (int a = tid; a < A; a += T) part += sm.nu[0][S + a];
        mass = block_sum_f(part, sm.redf);
        verdict = 1; fh = 1; mstop = 1;
      } else {
        for (int m = 1;; ++m) {
          const int tmax = min(m, L - 1);
          if (F < min(m + 3, L)) prepare_layers(sm, P, os, cbits, A, L, S, G, F, min(max(F + CH, m + 3), L));
          const bool odd = (m & 1) != 0;  // step m reads buffer (m-1)&1, writes m&1
          const float* __restrict__ src = odd ? sm.nu[0] : sm.nu[1];
          float* __restrict__ dst = odd ? sm.nu[1] : sm.nu[0];
          const uint32_t* Rs = odd ? sm.R[0] : sm.R[1];
          uint32_t* Rd = odd ? sm.R[1] : sm.R[0];
          // FP32 sweep
          if (kOneUnit) {
            if (tid < n_units) sweep_unit(src, dst, sm.cf, my_a, my_ph, Pph, tmax, S, my_off);
          } else {
            for (int u = tid; u < n_units; u += T) {
              const int a = u % A, ph = u / A, sg = sm.sig[a];
              int off[kLateral];
#pragma unroll
              for (int d = 0; d < kLateral; ++d) off[d] = dir_dt(d, sg) * S + sm.nbr[a * kLateral + d];
              sweep_unit(src, dst, sm.cf, a, ph, Pph, tmax, S, off);
            }
          }
          // exact reached-set step, 32 tubes per word
          const int nwin = (tmax >> 5) + 1;
          const int endw = (L - 1) >> 5, endb = (L - 1) & 31;
          uint32_t fl = 0;
          for (int u = tid; u < A * nwin; u += T) {
            const int tw = u / A, a = u - tw * A, sg = sm.sig[a];
            uint32_t acc = shifted_word(Rs, S, a, tw, -1) | shifted_word(Rs, S, a, tw, 1);
#pragma unroll
            for (int d = 0; d < kLateral; ++d)
              acc |= shifted_word(Rs, S, sm.nbr[a * kLateral + d], tw, dir_dt(d, sg));
            const int wi = (tw + 1) * S + a;
            const uint32_t old = Rs[wi];
            const uint32_t nw = old | (acc & sm.occw[wi]);
            Rd[wi] = nw;
            if (nw != old) fl |= kGrow;
            if (tw == endw && (((nw & ~old) >> endb) & 1u)) fl |= kEnd;
          }
          fl = __reduce_or_sync(0xffffffffu, fl);
          if ((tid & 31) == 0 && fl) atomicOr(&sm.flags[m % 3], fl);
          __syncthreads();
          const uint32_t f = sm.flags[m % 3];
          if (tid == 0) sm.flags[(m + 2) % 3] = 0u;
          if (f & kEnd) {
            float part = 0.f;
            for (int a = tid; a < A; a += T) part += dst[L * S + a];
            mass = block_sum_f(part, sm.redf);
            verdict = 1; fh = m + 1; mstop = m + 1;
            break;
          }
          if (!(f & kGrow)) { mstop = m; break; }
        }
      }
    }
    if (tid == 0) {
      P.verdict[rel] = (uint8_t)verdict;
      if (P.first_hit) P.first_hit[rel] = fh;
      if (P.mass) P.mass[rel] = mass;
      if (P.m_stop) P.m_stop[rel] = mstop;
      if (verdict && P.n_perc) atomicAdd(P.n_perc, 1ull);
    }
    __syncthreads();
  }
}

// Kernel, dynamic shared memory and grid of a resident launch.
static pc_status resident_config(const ResidentArgs& args, int threads, void** func, size_t* smem,
                                 long long* grid) {
  if (args.lat.A > 32767) {
    set_error("resident solver: more than 32767 columns");
    return PC_ERR_OOM;
  }
  *smem = resident_smem_bytes(args.lat.A, args.lat.L);
  const bool one = threads >= args.lat.A;
  auto kern = one ? resident_kernel<true> : resident_kernel<false>;
  PC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
  int dev = 0, nsm = 0, per_sm = 0;
  PC_CUDA(cudaGetDevice(&dev));
  PC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, *smem));
  if (per_sm < 1) {
    set_error("resident solver: lattice does not fit one CTA");
    return PC_ERR_OOM;
  }
  long long g = (long long)per_sm * nsm;
  if (g > args.n_cfg) g = args.n_cfg;
  *grid = g;
  *func = (void*)kern;
  return PC_OK;
}

pc_status resident_add_node(const ResidentArgs& args, int threads, cudaGraph_t g,
                            const cudaGraphNode_t* deps, size_t ndeps, cudaGraphNode_t* out) {
  void* func = nullptr;
  size_t smem = 0;
  long long grid = 0;
  pc_status rc = resident_config(args, threads, &func, &smem, &grid);
  if (rc) return rc;
  ResidentArgs a = args;
  void* params[] = {&a};
  cudaKernelNodeParams kp = {};
  kp.func = func;
  kp.gridDim = dim3((unsigned)(grid < 1 ? 1 : grid));
  kp.blockDim = dim3(threads);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = params;
  PC_CUDA(cudaGraphAddKernelNode(out, g, deps, ndeps, &kp));
  return PC_OK;
}

pc_status launch_resident(const ResidentArgs& args, int threads, cudaStream_t st) {
  if (args.lat.A > 32767) {
    set_error("resident solver: more than 32767 columns");
    return PC_ERR_OOM;
  }
  const size_t smem = resident_smem_bytes(args.lat.A, args.lat.L);
  const bool one = threads >= args.lat.A;
  auto kern = one ? resident_kernel<true> : resident_kernel<false>;
  PC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0, per_sm = 0;
  PC_CUDA(cudaGetDevice(&dev));
  PC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  if (per_sm < 1) {
    set_error("resident solver: lattice does not fit one CTA");
    return PC_ERR_OOM;
  }
  long long grid = (long long)per_sm * nsm;
  if (grid > args.n_cfg) grid = args.n_cfg;
  if (grid < 1) return PC_OK;
  kern<<<(unsigned)grid, threads, smem, st>>>(args);
  PC_CUDA(cudaGetLastError());
  return PC_OK;
}

}  // namespace pc

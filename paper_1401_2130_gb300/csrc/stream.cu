// stream.cu -- streamed solver for lattices whose state exceeds one CTA's
// shared memory (Sec. II.B, Eqs. (2)-(4) on the lattice of Sec. II.A).
//
// K "slots" each hold one configuration's state in HBM, laid out exactly as
// the resident solver lays it out in shared memory (nu ping-pong rows t+1,
// cf, occupancy and reached-set words [tw+1][a], column A an always-zero
// sentinel).  The host replays a CUDA graph of "ticks"; each tick is
//   sweep   : every CTA walks a global list of work units over all slots --
//             FP32 site updates of step m over the causal window, the exact
//             bit-parallel reached-set update, and lazy preparation of the
//             layers just ahead of the window (Philox draw of a word row,
//             1/deg rows, zeroing of nu and R rows);
//   control : one CTA per slot reads the step's grow/end flags, sums the
//             detector mass on a hit (deterministic block reduction), writes
//             the configuration's outputs and refills the slot from the work
//             counter (continuous refill: a slot never waits for the others).
// The unit plan of a slot is a pure function of its control record, computed
// identically by the sweep (to do the work) and by control (to advance G, F).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace pc {

namespace {

constexpr uint32_t kGrow = 1u, kEnd = 2u;
enum : int { PH_EMPTY = 0, PH_DRAW0 = 1, PH_PREP0 = 2, PH_STEP = 3 };
enum : int { U_FP = 0, U_BITS = 1, U_PREP = 2, U_DRAW = 3, U_KINDS = 4 };
constexpr int kCols = 256;   // columns per unit == threads per sweep CTA
constexpr int kRows = 16;    // layers (or word rows) per FP / BITS / PREP unit
constexpr int kMaxSlots = 64;

struct Ctl {
  long long rel;       // relative configuration index in the slot
  int phase;
  int m;               // next step to compute (PH_STEP)
  int G;               // layers with occupancy drawn (multiple of 32, or L)
  int F;               // layers with cf computed and nu / R rows cleaned
  unsigned int flags;  // grow / end of the step in flight
  int pad;
};

struct Ctx {
  Lattice lat;
  OccStream occ;
  const uint32_t* occ_bits;
  int64_t words_per_cfg;
  int64_t n_cfg;
  uint32_t cfg0;
  Outputs out;
  int K;
  Ctl* ctl;
  float* nu;           // [K][2][(L+2)*S]
  float* cf;           // [K][L*S]
  uint32_t* occw;      // [K][TWP*S]
  uint32_t* R;         // [K][2][TWP*S]
  unsigned long long* work;
  unsigned long long* n_done;
};

// Segments of work for one slot in the tick that starts from record c.
struct Plan {
  int lo[U_KINDS], hi[U_KINDS];  // row ranges per kind (layers, or word rows for BITS/DRAW)
  int G2, F2;                    // G and F after the tick
};

__host__ __device__ inline Plan make_plan(const Ctl& c, int L, int TW) {
  Plan p;
  for (int k = 0; k < U_KINDS; ++k) { p.lo[k] = 0; p.hi[k] = 0; }
  p.G2 = c.G; p.F2 = c.F;
  if (c.phase == PH_DRAW0) {
    const int rows = TW < 2 ? TW : 2;  // first 64 layers
    p.lo[U_DRAW] = 0; p.hi[U_DRAW] = rows;
    p.G2 = rows * 32 < L ? rows * 32 : L;
  } else if (c.phase == PH_PREP0) {
    p.lo[U_PREP] = 0; p.hi[U_PREP] = L < 5 ? L : 5;
    p.F2 = p.hi[U_PREP];
  } else if (c.phase == PH_STEP) {
    const int tmax = c.m < L - 1 ? c.m : L - 1;
    p.lo[U_FP] = 0; p.hi[U_FP] = tmax + 1;
    p.lo[U_BITS] = 0; p.hi[U_BITS] = (tmax >> 5) + 1;
    // prepare two layers per tick (the window grows by one); occupancy of
    // layer F2 must already be drawn: G >= min(F2 + 1, L)
    int F2 = c.F + 2 < L ? c.F + 2 : L;
    const int gneed = F2 + 1 < L ? F2 + 1 : L;
    if (c.G < gneed) F2 = c.F;  // cannot happen with the draw rule below
    p.lo[U_PREP] = c.F; p.hi[U_PREP] = F2;
    p.F2 = F2;
    // keep occupancy one word row ahead of the prepared layers
    if (c.G < L && c.G < F2 + 33) {
      p.lo[U_DRAW] = c.G >> 5; p.hi[U_DRAW] = (c.G >> 5) + 1;
      p.G2 = c.G + 32 < L ? c.G + 32 : L;
    }
  }
  return p;
}

__device__ inline int n_units_of(int kind, int lo, int hi, int A) {
  if (hi <= lo) return 0;
  const int ccol = (A + kCols - 1) / kCols;
  const int rows_per = (kind == U_DRAW) ? 1 : kRows;
  return ccol * ((hi - lo + rows_per - 1) / rows_per);
}

__device__ inline uint32_t bit_at(const uint32_t* w, int S, int col, int tt) {
  return (w[((tt >> 5) + 1) * S + col] >> (tt & 31)) & 1u;
}

__device__ inline uint32_t shifted_word(const uint32_t* R, int S, int col, int tw, int dt) {
  const uint32_t w = R[(tw + 1) * S + col];
  if (dt == 0) return w;
  if (dt > 0) return (w >> 1) | (R[(tw + 2) * S + col] << 31);
  return (w << 1) | (R[tw * S + col] >> 31);
}

__global__ void __launch_bounds__(kCols) sweep_kernel(Ctx x) {
  __shared__ Ctl s_ctl[kMaxSlots];
  __shared__ int s_pre[kMaxSlots * U_KINDS + 1];
  __shared__ uint32_t s_flag;
  const Lattice& lat = x.lat;
  const int A = lat.A, L = lat.L, S = lat.S, TWP = lat.TWP;
  const int tid = threadIdx.x;
  const int K = x.K;
  if (tid < K) s_ctl[tid] = x.ctl[tid];
  __syncthreads();
  if (tid < K) {
    const Plan p = make_plan(s_ctl[tid], L, lat.TW);
    for (int k = 0; k < U_KINDS; ++k) {
      s_pre[tid * U_KINDS + k] = n_units_of(k, p.lo[k], p.hi[k], A);
    }
  }
  __syncthreads();
  if (tid == 0) {  // exclusive prefix over (slot, kind)
    int acc = 0;
    for (int i = 0; i < K * U_KINDS; ++i) { const int v = s_pre[i]; s_pre[i] = acc; acc += v; }
    s_pre[K * U_KINDS] = acc;
  }
  __syncthreads();
  const int total = s_pre[K * U_KINDS];
  const int ccol = (A + kCols - 1) / kCols;
  const size_t nu_sz = (size_t)(L + 2) * S, w_sz = (size_t)TWP * S;

  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    // locate (slot, kind) by linear scan of the prefix
    int idx = 0;
    while (s_pre[idx + 1] <= u) ++idx;
    const int slot = idx / U_KINDS, kind = idx % U_KINDS;
    const int local = u - s_pre[idx];
    const int cchunk = local % ccol, rchunk = local / ccol;
    const int a = cchunk * kCols + tid;
    const Ctl& c = s_ctl[slot];
    float* nu0 = x.nu + (size_t)slot * 2 * nu_sz;
    float* nu1 = nu0 + nu_sz;
    float* cf = x.cf + (size_t)slot * L * S;
    uint32_t* occw = x.occw + (size_t)slot * w_sz;
    uint32_t* R0 = x.R + (size_t)slot * 2 * w_sz;
    uint32_t* R1 = R0 + w_sz;

    if (kind == U_FP) {
      const Plan p = make_plan(c, L, lat.TW);
      const int t0 = p.lo[U_FP] + rchunk * kRows;
      const int t1 = min(t0 + kRows, p.hi[U_FP]);
      const int m = c.m;
      const float* __restrict__ src = (m & 1) ? nu0 : nu1;
      float* __restrict__ dst = (m & 1) ? nu1 : nu0;
      if (a < A) {
        const int sg = lat.sigma[a];
        int off[kLateral];
#pragma unroll
        for (int d = 0; d < kLateral; ++d) off[d] = dir_dt(d, sg) * S + lat.nbr[a * kLateral + d];
        float below = src[t0 * S + a], here = src[(t0 + 1) * S + a];
        for (int t = t0; t < t1; ++t) {
          const int base = (t + 1) * S;
          const float above = src[base + S + a];
          float s = below + above;
#pragma unroll
          for (int d = 0; d < kLateral; ++d) s += src[base + off[d]];
          dst[base + a] = cf[t * S + a] * s;
          below = here; here = above;
        }
      }
    } else if (kind == U_BITS) {
      const Plan p = make_plan(c, L, lat.TW);
      const int w0 = p.lo[U_BITS] + rchunk * kRows;
      const int w1 = min(w0 + kRows, p.hi[U_BITS]);
      const int m = c.m;
      const int tmax = min(m, L - 1);
      const uint32_t* Rs = (m & 1) ? R0 : R1;
      uint32_t* Rd = (m & 1) ? R1 : R0;
      uint32_t fl = 0;
      if (a < A) {
        const int sg = lat.sigma[a];
        int nb[kLateral], dt[kLateral];
#pragma unroll
        for (int d = 0; d < kLateral; ++d) { nb[d] = lat.nbr[a * kLateral + d]; dt[d] = dir_dt(d, sg); }
        const int endw = (L - 1) >> 5, endb = (L - 1) & 31;
        for (int tw = w0; tw < w1; ++tw) {
          uint32_t acc = shifted_word(Rs, S, a, tw, -1) | shifted_word(Rs, S, a, tw, 1);
#pragma unroll
          for (int d = 0; d < kLateral; ++d) acc |= shifted_word(Rs, S, nb[d], tw, dt[d]);
          const int wi = (tw + 1) * S + a;
          const uint32_t old = Rs[wi];
          const uint32_t nw = old | (acc & occw[wi]);
          Rd[wi] = nw;
          if (nw != old) fl |= kGrow;
          if (tw == endw && (((nw & ~old) >> endb) & 1u)) fl |= kEnd;
        }
        (void)tmax;
      }
      fl = __reduce_or_sync(0xffffffffu, fl);
      if (tid == 0) s_flag = 0u;
      __syncthreads();
      if ((tid & 31) == 0 && fl) atomicOr(&s_flag, fl);
      __syncthreads();
      if (tid == 0 && s_flag) atomicOr(&x.ctl[slot].flags, s_flag);
    } else if (kind == U_PREP) {
      const Plan p = make_plan(c, L, lat.TW);
      const int t0 = p.lo[U_PREP] + rchunk * kRows;
      const int t1 = min(t0 + kRows, p.hi[U_PREP]);
      if (a < A) {
        const int sg = lat.sigma[a];
        int nb[kLateral];
#pragma unroll
        for (int d = 0; d < kLateral; ++d) nb[d] = lat.nbr[a * kLateral + d];
        for (int t = t0; t < t1; ++t) {
          float cval = 0.f;
          if (bit_at(occw, S, a, t)) {
            int deg = (int)bit_at(occw, S, a, t - 1) + (int)bit_at(occw, S, a, t + 1) + (t == L - 1);
#pragma unroll
            for (int d = 0; d < kLateral; ++d) deg += (int)bit_at(occw, S, nb[d], t + dir_dt(d, sg));
            cval = deg ? __frcp_rn((float)deg) : 0.f;
          }
          cf[t * S + a] = cval;
          nu0[(t + 1) * S + a] = 0.f;
          nu1[(t + 1) * S + a] = 0.f;
          // reached-set word rows are cleaned one row ahead of the layers
          if ((t & 31) == 0) {
            const int wr = (t >> 5) + 2;  // data word row (t>>5)+1
            R0[wr * S + a] = 0u; R1[wr * S + a] = 0u;
            if (t == 0) { R0[S + a] = 0u; R1[S + a] = 0u; }
          }
        }
      }
    } else {  // U_DRAW: one word row of occupancy, 32 tubes per word
      const Plan p = make_plan(c, L, lat.TW);
      const int tw = p.lo[U_DRAW] + rchunk;
      if (a < A) {
        uint32_t word = 0;
        const uint32_t cfg = x.cfg0 + (uint32_t)c.rel;
        if (x.occ_bits) {
          const uint32_t* cb = x.occ_bits + (size_t)c.rel * x.words_per_cfg;
          for (int b = 0; b < 32; ++b) {
            const int t = tw * 32 + b;
            if (t >= L) break;
            const int64_t i = (int64_t)t * A + a;
            word |= ((cb[i >> 5] >> (i & 31)) & 1u) << b;
          }
        } else {
          OccStream os = x.occ;
          os.cfg = cfg;
          for (int b = 0; b < 32; ++b) {
            const int t = tw * 32 + b;
            if (t >= L) break;
            const int64_t i = (int64_t)t * A + a;
            const u32x4 r = philox4x32_10(u32x4{(uint32_t)(i >> 2), cfg, os.wl, 0u}, os.k0, os.k1);
            const uint32_t v = (i & 3) == 0 ? r.x : (i & 3) == 1 ? r.y : (i & 3) == 2 ? r.z : r.w;
            word |= (uint32_t)((uint64_t)v < os.T) << b;
          }
        }
        occw[(tw + 1) * S + a] = word;
      }
    }
  }
}

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

// One CTA per slot.
__global__ void __launch_bounds__(kCols) control_kernel(Ctx x) {
  __shared__ float red[32];
  __shared__ int s_n0;
  const int slot = blockIdx.x, tid = threadIdx.x;
  const Lattice& lat = x.lat;
  const int A = lat.A, L = lat.L, S = lat.S;
  const size_t nu_sz = (size_t)(L + 2) * S, w_sz = (size_t)lat.TWP * S;
  Ctl c = x.ctl[slot];
  if (c.phase == PH_EMPTY) return;
  float* nu0 = x.nu + (size_t)slot * 2 * nu_sz;
  float* nu1 = nu0 + nu_sz;
  const float* cf = x.cf + (size_t)slot * L * S;
  const uint32_t* occw = x.occw + (size_t)slot * w_sz;
  uint32_t* R0 = x.R + (size_t)slot * 2 * w_sz;

  const Plan p = make_plan(c, L, lat.TW);
  bool finish = false;
  int verdict = 0, fh = -1, mstop = 0;
  float mass = 0.f;
  if (c.phase == PH_DRAW0) {
    c.G = p.G2; c.phase = PH_PREP0;
  } else if (c.phase == PH_PREP0) {
    c.F = p.F2;
    // m = 0: mu_0 uniform on the metallic sites of t = 0
    if (tid == 0) s_n0 = 0;
    __syncthreads();
    int cnt = 0;
    for (int a = tid; a < A; a += blockDim.x) cnt += (int)(occw[S + a] & 1u);
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if ((tid & 31) == 0 && cnt) atomicAdd(&s_n0, cnt);
    __syncthreads();
    const int n0 = s_n0;
    if (n0 == 0) {
      finish = true;
    } else {
      const float inv = __frcp_rn((float)n0);
      float part = 0.f;
      for (int a = tid; a < A; a += blockDim.x) {
        const uint32_t b = occw[S + a] & 1u;
        R0[S + a] = b;
        const float v = b ? cf[a] * inv : 0.f;
        nu0[S + a] = v;
        part += v;
      }
      if (L == 1) {
        mass = block_sum_f(part, red);
        finish = true; verdict = 1; fh = 1; mstop = 1;
      } else {
        c.phase = PH_STEP; c.m = 1; c.flags = 0u;
      }
    }
  } else if (c.phase == PH_STEP) {
    c.G = p.G2; c.F = p.F2;
    const unsigned f = c.flags;
    c.flags = 0u;
    if (f & kEnd) {
      const float* dst = (c.m & 1) ? nu1 : nu0;
      float part = 0.f;
      for (int a = tid; a < A; a += blockDim.x) part += dst[L * S + a];
      mass = block_sum_f(part, red);
      finish = true; verdict = 1; fh = c.m + 1; mstop = c.m + 1;
    } else if (!(f & kGrow)) {
      finish = true; mstop = c.m;
    } else {
      c.m += 1;
    }
  }
  if (finish) {
    if (tid == 0) {
      const long long rel = c.rel;
      x.out.verdict[rel] = (uint8_t)verdict;
      if (x.out.first_hit) x.out.first_hit[rel] = fh;
      if (x.out.mass) x.out.mass[rel] = mass;
      if (x.out.m_stop) x.out.m_stop[rel] = mstop;
      if (verdict && x.out.n_perc) atomicAdd(x.out.n_perc, 1ull);
      atomicAdd(x.n_done, 1ull);
      const unsigned long long nxt = atomicAdd(x.work, 1ull);
      Ctl n;
      n.rel = (long long)nxt; n.m = 0; n.G = 0; n.F = 0; n.flags = 0u; n.pad = 0;
      n.phase = (long long)nxt < x.n_cfg ? PH_DRAW0 : PH_EMPTY;
      x.ctl[slot] = n;
    }
  } else if (tid == 0) {
    x.ctl[slot] = c;
  }
}

__global__ void init_slots_kernel(Ctx x) {
  const int s = threadIdx.x;
  if (s < x.K) {
    Ctl n;
    n.rel = s; n.m = 0; n.G = 0; n.F = 0; n.flags = 0u; n.pad = 0;
    n.phase = s < x.n_cfg ? PH_DRAW0 : PH_EMPTY;
    x.ctl[s] = n;
  }
  if (s == 0) { *x.work = (unsigned long long)x.K; *x.n_done = 0ull; }
}

}  // namespace

size_t stream_slot_bytes(int A, int L) {
  const size_t S = (size_t)A + 1, TWP = (size_t)(L + 31) / 32 + 2;
  return sizeof(float) * (2 * (size_t)(L + 2) * S + (size_t)L * S) + sizeof(uint32_t) * 3 * TWP * S;
}

pc_status run_stream(const StreamJob& job, cudaStream_t st) {
  if (job.n_cfg <= 0) return PC_OK;
  const Lattice& lat = job.lat;
  const size_t slot_bytes = stream_slot_bytes(lat.A, lat.L);
  size_t free_b = 0, total_b = 0;
  PC_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t budget = free_b / 2;
  long long K = std::min<long long>(job.n_cfg, kMaxSlots);
  K = std::min<long long>(K, (long long)(budget / (slot_bytes + 1)));
  if (K < 1) {
    set_error("streamed solver: one configuration's state exceeds half the free device memory");
    return PC_ERR_OOM;
  }
  Ctx x;
  x.lat = lat; x.occ = job.occ; x.occ_bits = job.occ_bits; x.words_per_cfg = job.words_per_cfg;
  x.n_cfg = job.n_cfg; x.cfg0 = job.cfg0; x.out = job.out; x.K = (int)K;
  const size_t S = (size_t)lat.S, nu_sz = (size_t)(lat.L + 2) * S, w_sz = (size_t)lat.TWP * S;
  char* pool = nullptr;
  const size_t ctl_bytes = sizeof(Ctl) * kMaxSlots + 64;
  const size_t pool_bytes = ctl_bytes + (size_t)K * slot_bytes + 256;
  PC_CUDA(cudaMallocAsync((void**)&pool, pool_bytes, st));
  pc_status rc = PC_OK;
  unsigned long long* h_done = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  do {
    if (cudaMemsetAsync(pool, 0, pool_bytes, st) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "memset"); break; }
    char* q = pool;
    x.ctl = (Ctl*)q; q += sizeof(Ctl) * kMaxSlots;
    x.work = (unsigned long long*)q; q += 8;
    x.n_done = (unsigned long long*)q; q += 56;
    x.nu = (float*)q; q += sizeof(float) * K * 2 * nu_sz;
    x.cf = (float*)q; q += sizeof(float) * K * lat.L * S;
    x.occw = (uint32_t*)q; q += sizeof(uint32_t) * K * w_sz;
    x.R = (uint32_t*)q;
    init_slots_kernel<<<1, kMaxSlots, 0, st>>>(x);
    if (cudaGetLastError() != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "init_slots"); break; }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nsm * 8;
    // capture a chunk of ticks
    const int ticks = 32;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "stream"); break; }
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int i = 0; i < ticks; ++i) {
        sweep_kernel<<<grid, kCols, 0, cs>>>(x);
        control_kernel<<<(unsigned)K, kCols, 0, cs>>>(x);
      }
      e = cudaStreamEndCapture(cs, &graph);
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) { rc = cuda_fail(e, "graph capture"); break; }
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { rc = cuda_fail(e, "graph instantiate"); break; }
    if (cudaMallocHost(&h_done, sizeof(unsigned long long)) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "host alloc"); break; }
    *h_done = 0;
    // Each configuration needs at most N + 3 ticks (the reached set grows by
    // at least one site per step); bound the loop accordingly.
    const long long max_replays = (long long)((job.n_cfg + K - 1) / K) * ((lat.N + 8) / ticks + 2) + 16;
    long long replays = 0;
    for (;;) {
      e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) { rc = cuda_fail(e, "graph launch"); break; }
      e = cudaMemcpyAsync(h_done, x.n_done, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { rc = cuda_fail(e, "poll"); break; }
      if ((long long)*h_done >= job.n_cfg) break;
      if (++replays > max_replays) { set_error("streamed solver did not converge"); rc = PC_ERR_INTERNAL; break; }
    }
  } while (0);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (h_done) cudaFreeHost(h_done);
  cudaFreeAsync(pool, st);
  return rc;
}

}  // namespace pc

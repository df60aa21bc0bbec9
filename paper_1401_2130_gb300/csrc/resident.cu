// resident.cu -- shared-memory resident solver for lattices that fit in one
// CTA's shared memory (Sec. II.B, Eqs. (2)-(4) on the lattice of Sec. II.A).
//
// A persistent CTA pulls configurations from a work counter and keeps the
// whole state of one configuration in shared memory for its entire solve:
//   nu[2][(L+4) planes]  FP32: nu(i) = mu(i) / deg(i), the mass each site sends
//                        along each of its edges (ping-pong).  Layer t lives
//                        in plane t+2 of the padded-row layout (lattice.cu);
//                        planes 0, 1, L+2, L+3 and all padding are zero.
//   dg[L planes]         u8: deg(i) of metallic sites, 0 elsewhere (Eq. (2);
//                        the detector edge counts on t = L-1)
//   occw, R[2]           bits: occupancy and reached set; word (tw, a) holds
//                        the 32 tube indices 32*tw .. 32*tw+31 of column a,
//                        stored row-major [tw + 1][a] with zero pad rows and
//                        an always-zero column A
// One step m of Eq. (3) in forward form, over the causal window t <= m:
//   mu_m(j) = sum over the 14 lattice neighbours i of j of nu_{m-1}(i)
//   nu_m(j) = mu_m(j) / deg(j)                        (Jacobi, FP32)
//   R_m     = R_{m-1} | (N(R_{m-1}) & occ)            (exact, bit-parallel)
// The verdict is decided by R only, so FP32 underflow cannot change it.  If a
// site of the end layer t = L-1 enters R at step m, the detector probability
// first becomes non-zero at step m+1 and equals sum_{t=L-1} nu_m (each end
// site sends nu along its detector edge).  If R does not grow, the
// configuration does not percolate.
//
// The FP sweep is register tiled (strip_sweep, tiling.cuh): a thread owns a
// strip of 3 plane positions (sublattices 0, 1, 2) and walks a run of layers
// with the neighbour rows of layers t-1, t, t+1 in registers: 23 loads per
// layer for 3 outputs instead of 14 gathers per output; consecutive lanes
// read addresses 3 apart, which never share a shared-memory bank.
//
// Layers are prepared lazily, a chunk at a time, as the window reaches them:
// occupancy drawn from the Philox stream (or read from caller bits), degrees
// computed, nu planes zeroed.  Layers the window never reaches are never
// drawn: their occupancy cannot influence any output.
#include "common.cuh"
#include "kernels.cuh"
#include "tiling.cuh"

namespace pc {

namespace {

constexpr uint32_t kGrow = 1u, kEnd = 2u;
constexpr int kMaxThreads = kResidentMaxThreads;

struct Smem {
  float* nu[2];
  uint8_t* dg;
  uint32_t* occw;
  uint32_t* R[2];
  int16_t* nbr;
  int8_t* sig;
  int16_t* srow;
  int* roff;
  float* inv;       // [16]
  uint32_t* flags;  // [3]
  float* redf;      // [32]
  long long* redi;  // [32]
  long long* scal;  // [4]
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t smem_bytes(int W, int A, int L, int P, int n_strips) {
  const size_t S = (size_t)A + 1, TWP = (size_t)(L + 31) / 32 + 2;
  size_t b = 0;
  b += 2 * align16(sizeof(float) * (size_t)(L + 4) * P);
  b += align16((size_t)L * P);
  b += 3 * align16(sizeof(uint32_t) * S * TWP);
  b += align16(sizeof(int16_t) * (size_t)A * kLateral);
  b += align16((size_t)A);
  b += align16(sizeof(int16_t) * (size_t)n_strips);
  b += align16(sizeof(int) * 4 * (size_t)(2 * W + 1));
  b += align16(sizeof(float) * 16) + align16(sizeof(uint32_t) * 4) + align16(sizeof(float) * 32) +
       align16(sizeof(long long) * 32) + align16(sizeof(long long) * 4);
  return b;
}

__device__ inline Smem carve(unsigned char* base, int W, int A, int L, int P, int n_strips) {
  const size_t S = (size_t)A + 1, TWP = (size_t)(L + 31) / 32 + 2;
  Smem s;
  size_t o = 0;
  auto take = [&](size_t bytes) { unsigned char* p = base + o; o += align16(bytes); return p; };
  s.nu[0] = (float*)take(sizeof(float) * (size_t)(L + 4) * P);
  s.nu[1] = (float*)take(sizeof(float) * (size_t)(L + 4) * P);
  s.dg = (uint8_t*)take((size_t)L * P);
  s.occw = (uint32_t*)take(sizeof(uint32_t) * S * TWP);
  s.R[0] = (uint32_t*)take(sizeof(uint32_t) * S * TWP);
  s.R[1] = (uint32_t*)take(sizeof(uint32_t) * S * TWP);
  s.nbr = (int16_t*)take(sizeof(int16_t) * (size_t)A * kLateral);
  s.sig = (int8_t*)take((size_t)A);
  s.srow = (int16_t*)take(sizeof(int16_t) * (size_t)n_strips);
  s.roff = (int*)take(sizeof(int) * 4 * (size_t)(2 * W + 1));
  s.inv = (float*)take(sizeof(float) * 16);
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

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// bit of a word array [tw + 1][S]: column col, tube tt (tt = -1 and tt >= L
// land in zero padding)
__device__ inline uint32_t bit_at(const uint32_t* w, int S, int col, int tt) {
  return (w[((tt >> 5) + 1) * S + col] >> (tt & 31)) & 1u;
}

// Contacts of word tw of column col in the reached set R (words [tw + 1][S]):
// bit b of the result is set when some contact of the site at tube
// 32*tw + b is in R.  The end contacts are the own column at tubes t-1 and
// t+1; the 6 same-layer contacts share the tube index; the 3 up contacts
// are at tube t+1 when sigma = 2, the 3 down contacts at t-1 when
// sigma = 0.  Each group of three is ORed first and shifted once by a
// funnel shift selected by sigma, so no lane branches on its sublattice.
__device__ __forceinline__ uint32_t contact_word(const uint32_t* R, int S, int col, int tw,
                                                 const int (&nb)[kLateral], uint32_t sh_up,
                                                 uint32_t sh_dn) {
  const uint32_t* r0 = R + tw * S;  // word tw - 1
  const uint32_t* r1 = r0 + S;      // word tw
  const uint32_t* r2 = r1 + S;      // word tw + 1
  const uint32_t own = r1[col];
  uint32_t acc = ((own << 1) | (r0[col] >> 31)) | ((own >> 1) | (r2[col] << 31));
#pragma unroll
  for (int d = 0; d < 6; ++d) acc |= r1[nb[d]];
  const uint32_t up = r1[nb[6]] | r1[nb[7]] | r1[nb[8]];
  const uint32_t up_hi = r2[nb[6]] | r2[nb[7]] | r2[nb[8]];
  const uint32_t dn = r1[nb[9]] | r1[nb[10]] | r1[nb[11]];
  const uint32_t dn_lo = r0[nb[9]] | r0[nb[10]] | r0[nb[11]];
  return acc | __funnelshift_r(up, up_hi, sh_up) | __funnelshift_l(dn_lo, dn, sh_dn);
}

// Lazy preparation of layers [F, Fnew): occupancy drawn up to layer Fnew (for
// the degrees of layer Fnew - 1), degrees (Eq. (2), detector edge on t = L-1),
// nu planes zeroed in both buffers.  Block-uniform.
__device__ __forceinline__ void prepare_layers(const Smem& sm, const Lattice& lat, const OccStream& os,
                                               const uint32_t* cbits, int& G, int& F, int Fnew,
                                               bool bits_only) {
  const int tid = threadIdx.x, T = blockDim.x;
  const int A = lat.A, L = lat.L, S = lat.S, P = lat.P;
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
  const int n = bits_only ? 0 : (Fnew - F) * P;  // degrees and nu: FP sweep only
  for (int k = tid; k < n; k += T) {
    const int t = F + k / P, pos = k % P;
    const int a = __ldg(lat.pcol + pos);
    int deg = 0;
    if (a >= 0 && bit_at(sm.occw, S, a, t)) {
      const int sg = sm.sig[a];
      deg = (int)bit_at(sm.occw, S, a, t - 1) + (int)bit_at(sm.occw, S, a, t + 1) + (t == L - 1);
#pragma unroll
      for (int d = 0; d < kLateral; ++d)
        deg += (int)bit_at(sm.occw, S, sm.nbr[a * kLateral + d], t + dir_dt(d, sg));
    }
    sm.dg[t * P + pos] = (uint8_t)deg;
    sm.nu[0][(t + 2) * P + pos] = 0.f;
    sm.nu[1][(t + 2) * P + pos] = 0.f;
  }
  F = Fnew;
  __syncthreads();
}

}  // namespace

size_t resident_smem(const Lattice& lat) { return smem_bytes(lat.W, lat.A, lat.L, lat.P, lat.n_strips); }

// Per-query state of a CTA: the shared-memory carve of the query's lattice
// and, when the CTA has a thread per column, that thread's column tables.
struct QueryState {
  Smem sm;
  bool own_col;
  uint32_t my_nb[kLateral / 2];  // packed int16 pairs of neighbour columns
  int my_sg;
};

// Loads the lattice tables of query Pa into shared memory (resident
// lattices have A < 2^15: int16 columns) and zeroes the guard and boundary
// planes of nu.  Block-uniform.
__device__ __forceinline__ void setup_query(const ResidentArgs& Pa, unsigned char* smem_raw, QueryState& qs) {
  const Lattice& lat = Pa.lat;
  const int W = lat.W, A = lat.A, L = lat.L, P = lat.P, NS = lat.n_strips;
  const int tid = threadIdx.x, T = blockDim.x;
  qs.sm = carve(smem_raw, W, A, L, P, NS);
  const Smem& sm = qs.sm;
  for (int k = tid; k < A * kLateral; k += T) sm.nbr[k] = (int16_t)lat.nbr[k];
  for (int k = tid; k < A; k += T) sm.sig[k] = lat.sigma[k];
  for (int k = tid; k < NS; k += T) sm.srow[k] = lat.strip_row[k];
  for (int k = tid; k < 4 * (2 * W + 1); k += T) sm.roff[k] = lat.row_off[k];
  if (tid < 16) sm.inv[tid] = tid ? __frcp_rn((float)tid) : 0.f;
  for (int k = tid; k < 2 * P; k += T) {
    sm.nu[0][k] = 0.f; sm.nu[1][k] = 0.f;
    sm.nu[0][(size_t)(L + 2) * P + k] = 0.f; sm.nu[1][(size_t)(L + 2) * P + k] = 0.f;
  }
  __syncthreads();
  // a thread per column owns the column's reached-set words and keeps its
  // neighbour table
  qs.own_col = T >= A && tid < A;
  qs.my_sg = 0;
  if (qs.own_col) {
    qs.my_sg = sm.sig[tid];
#pragma unroll
    for (int d = 0; d < kLateral; d += 2)
      qs.my_nb[d >> 1] = (uint32_t)(uint16_t)sm.nbr[tid * kLateral + d] |
                         ((uint32_t)(uint16_t)sm.nbr[tid * kLateral + d + 1] << 16);
  }
}

// Inspects configuration rel of query Pa, whose tables setup_query loaded.
// Block-uniform; ends with a block barrier.
__device__ __forceinline__ void solve_config(const ResidentArgs& Pa, const QueryState& qst, long long rel) {
  const Lattice& lat = Pa.lat;
  const int A = lat.A, L = lat.L, S = lat.S, TWP = lat.TWP, P = lat.P;
  const int NS = lat.n_strips, SB = lat.s_begin;
  const int tid = threadIdx.x, T = blockDim.x;
  const Smem& sm = qst.sm;
  const bool own_col = qst.own_col;
  const int my_sg = qst.my_sg;
  const uint32_t (&my_nb)[kLateral / 2] = qst.my_nb;
  const int CH = Pa.prep_chunk;
  const bool bits_only = Pa.bits_only != 0;
  // verdict first: the reached set alone decides every configuration, and
  // the FP32 recursion runs afterwards, for exactly first_hit - 1 steps,
  // only on the configurations that percolate (the others' mass is 0)
  const bool vfirst = Pa.verdict_first != 0 && !bits_only && L > 1;
  const bool no_fp = bits_only || vfirst;  // no FP32 sweep in the first pass
  const int n_words_col = S * TWP;
  {
    const uint32_t cfg = Pa.cfg0 + (uint32_t)rel;

    // reset bit arrays and flags
    for (int k = tid; k < n_words_col; k += T) { sm.occw[k] = 0u; sm.R[0][k] = 0u; sm.R[1][k] = 0u; }
    if (tid < 3) sm.flags[tid] = 0u;
    __syncthreads();

    int G = 0, F = 0;  // layers with occupancy drawn / with degrees + zeroed nu
    OccStream os = Pa.occ;
    os.cfg = cfg;
    const uint32_t* cbits = Pa.occ_bits ? Pa.occ_bits + (size_t)rel * Pa.words_per_cfg : nullptr;

    prepare_layers(sm, lat, os, cbits, G, F, min(max(CH, 3), L), no_fp);

    // FP32 sweep of step m over the causal window: (strip, layer chunk)
    // items; K chunks per strip so that every thread gets at most one item
    // when the window allows.  The strip index is padded to a multiple of 32
    // per chunk (lanes past NS idle): a warp then never holds strips of two
    // chunks, whose planes lie whole planes apart and would share banks.
    auto fp_sweep = [&](int m, const float* src, float* dst) {
      const int nl = min(m, L - 1) + 1;
      const int NSp = (NS + 31) & ~31;
      const int K = T / NSp > 1 ? T / NSp : 1;
      int CL = (nl + K - 1) / K;
      CL = CL < 2 ? 2 : CL;
      const int nch = (nl + CL - 1) / CL;
      const uint32_t src_s = smem_addr(src), dg_s = smem_addr(sm.dg), inv_s = smem_addr(sm.inv);
      for (int it = tid; it < NSp * nch; it += T) {
        const int c = it / NSp, k = it - c * NSp;
        if (k >= NS) continue;
        const int t0 = c * CL, t1 = min(t0 + CL, nl);
        const int* ro = sm.roff + 4 * sm.srow[k];
        strip_sweep_s(src_s, dst, dg_s, inv_s, P, 3 * (SB + k), ro[0], ro[1], ro[2], ro[3], t0, t1);
      }
    };

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
      auto start_nu = [&]() {
        for (int a = tid; a < A; a += T) {
          const int pos = __ldg(lat.ppos + a);
          sm.nu[0][2 * P + pos] = (sm.occw[S + a] & 1u) ? sm.inv[sm.dg[pos]] * inv_n0 : 0.f;
        }
        __syncthreads();
      };
      if (!no_fp) start_nu();
      else __syncthreads();
      if (L == 1) {
        float part = 0.f;
        for (int k = tid; k < P; k += T) part += sm.nu[0][2 * P + k];
        mass = bits_only ? 0.f : block_sum_f(part, sm.redf);
        verdict = 1; fh = 1; mstop = 1;
      } else {
        for (int m = 1;; ++m) {
          const int tmax = min(m, L - 1);
          if (F < min(m + 3, L)) prepare_layers(sm, lat, os, cbits, G, F, min(max(F + CH, m + 3), L), no_fp);
          const bool odd = (m & 1) != 0;  // step m reads buffer (m-1)&1, writes m&1
          const float* __restrict__ src = odd ? sm.nu[0] : sm.nu[1];
          float* __restrict__ dst = odd ? sm.nu[1] : sm.nu[0];
          const uint32_t* Rs = odd ? sm.R[0] : sm.R[1];
          uint32_t* Rd = odd ? sm.R[1] : sm.R[0];
          if (!no_fp) fp_sweep(m, src, dst);
          // exact reached-set step, 32 tubes per word
          const int nwin = (tmax >> 5) + 1;
          const int endw = (L - 1) >> 5, endb = (L - 1) & 31;
          uint32_t fl = 0;
          if (own_col) {  // this thread's column, neighbour table in registers
            int nb[kLateral];
#pragma unroll
            for (int d = 0; d < kLateral; ++d) nb[d] = (my_nb[d >> 1] >> ((d & 1) * 16)) & 0xffff;
            const uint32_t sh_up = my_sg == 2 ? 1u : 0u, sh_dn = my_sg == 0 ? 1u : 0u;
            for (int tw = 0; tw < nwin; ++tw) {
              const uint32_t acc = contact_word(Rs, S, tid, tw, nb, sh_up, sh_dn);
              const int wi = (tw + 1) * S + tid;
              const uint32_t old = Rs[wi];
              const uint32_t nw = old | (acc & sm.occw[wi]);
              Rd[wi] = nw;
              if (nw != old) fl |= kGrow;
              if (tw == endw && (((nw & ~old) >> endb) & 1u)) fl |= kEnd;
            }
          } else if (T < A) {
            for (int u = tid; u < A * nwin; u += T) {
              const int tw = u / A, a = u - tw * A, sg = sm.sig[a];
              int nb[kLateral];
#pragma unroll
              for (int d = 0; d < kLateral; ++d) nb[d] = sm.nbr[a * kLateral + d];
              const uint32_t acc = contact_word(Rs, S, a, tw, nb, sg == 2 ? 1u : 0u, sg == 0 ? 1u : 0u);
              const int wi = (tw + 1) * S + a;
              const uint32_t old = Rs[wi];
              const uint32_t nw = old | (acc & sm.occw[wi]);
              Rd[wi] = nw;
              if (nw != old) fl |= kGrow;
              if (tw == endw && (((nw & ~old) >> endb) & 1u)) fl |= kEnd;
            }
          }
          fl = __reduce_or_sync(0xffffffffu, fl);
          if ((tid & 31) == 0 && fl) atomicOr(&sm.flags[m % 3], fl);
          __syncthreads();
          const uint32_t f = sm.flags[m % 3];
          if (tid == 0) sm.flags[(m + 2) % 3] = 0u;
          if (f & kEnd) {
            float part = 0.f;
            for (int k = no_fp ? P : tid; k < P; k += T) part += dst[(size_t)(L + 1) * P + k];
            mass = no_fp ? 0.f : block_sum_f(part, sm.redf);
            verdict = 1; fh = m + 1; mstop = m + 1;
            break;
          }
          if (!(f & kGrow)) { mstop = m; break; }
        }
        if (vfirst && verdict) {
          // second pass, FP32 only: degrees from layer 0 (the occupancy is
          // already drawn), nu_0, then steps 1 .. first_hit - 1 exactly as
          // the single pass runs them, so the mass is the same to the bit
          F = 0;
          prepare_layers(sm, lat, os, cbits, G, F, min(max(CH, 3), L), false);
          start_nu();
          for (int m = 1; m < fh; ++m) {
            if (F < min(m + 3, L)) prepare_layers(sm, lat, os, cbits, G, F, min(max(F + CH, m + 3), L), false);
            const bool odd = (m & 1) != 0;
            fp_sweep(m, odd ? sm.nu[0] : sm.nu[1], odd ? sm.nu[1] : sm.nu[0]);
            __syncthreads();
          }
          const float* last = ((fh - 1) & 1) ? sm.nu[1] : sm.nu[0];
          float part = 0.f;
          for (int k = tid; k < P; k += T) part += last[(size_t)(L + 1) * P + k];
          mass = block_sum_f(part, sm.redf);
        }
      }
    }
    if (tid == 0) {
      Pa.verdict[rel] = (uint8_t)verdict;
      if (Pa.first_hit) Pa.first_hit[rel] = fh;
      if (Pa.mass) Pa.mass[rel] = mass;
      if (Pa.m_stop) Pa.m_stop[rel] = mstop;
      if (verdict && Pa.n_perc) atomicAdd(Pa.n_perc, 1ull);
    }
    __syncthreads();
  }
}

// One query: every CTA takes configurations from the query's counter.
__global__ void __launch_bounds__(kMaxThreads, 1) resident_kernel(ResidentArgs Pa) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_item;
  QueryState qs;
  setup_query(Pa, smem_raw, qs);
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(Pa.work, 1ull);
    __syncthreads();
    const long long rel = s_item;
    if (rel >= Pa.n_cfg) break;
    solve_config(Pa, qs, rel);
  }
}

// Many queries in one persistent launch: their configurations form one
// list of items (query q owns [item0[q], item0[q + 1])), taken in order from
// one counter.  The host orders the queries by decreasing lattice size, so
// the longest configurations start first and the short ones fill the tails;
// a CTA reloads the lattice tables only when its next item belongs to
// another query.
__global__ void __launch_bounds__(kMaxThreads, 1) resident_multi_kernel(ResidentBatch B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long s_item;
  QueryState qs;
  int cur = -1;
  const long long n_items = B.item0[B.nq];
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(B.work, 1ull);
    __syncthreads();
    const long long item = s_item;
    if (item >= n_items) break;
    int lo = 0, hi = B.nq - 1;  // last q with item0[q] <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (B.item0[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const ResidentArgs& Pa = B.qs[lo];
    if (lo != cur) {
      setup_query(Pa, smem_raw, qs);
      cur = lo;
    }
    solve_config(Pa, qs, item - B.item0[lo]);
  }
}

// Kernel, dynamic shared memory and grid of a resident launch.
static pc_status resident_config(const ResidentArgs& args, int threads, void** func, size_t* smem,
                                 long long* grid) {
  if (args.lat.A > 32767) {
    set_error("resident solver: more than 32767 columns");
    return PC_ERR_OOM;
  }
  if (threads > kMaxThreads || threads < 32 || threads % 32) {
    set_error("resident solver: CTA size must be a multiple of 32 in [32, 640]");
    return PC_ERR_ARG;
  }
  *smem = resident_smem(args.lat);
  PC_CUDA(cudaFuncSetAttribute(resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
  int dev = 0, nsm = 0, per_sm = 0;
  PC_CUDA(cudaGetDevice(&dev));
  PC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resident_kernel, threads, *smem));
  if (per_sm < 1) {
    set_error("resident solver: lattice does not fit one CTA");
    return PC_ERR_OOM;
  }
  long long g = (long long)per_sm * nsm;
  if (g > args.n_cfg) g = args.n_cfg;
  *grid = g;
  *func = (void*)resident_kernel;
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

pc_status resident_multi_add_node(const ResidentBatch& b, long long n_items, size_t smem, int threads,
                                  cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                                  cudaGraphNode_t* out) {
  if (threads > kMaxThreads || threads < 32 || threads % 32) {
    set_error("resident solver: CTA size must be a multiple of 32 in [32, 640]");
    return PC_ERR_ARG;
  }
  PC_CUDA(cudaFuncSetAttribute(resident_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0, per_sm = 0;
  PC_CUDA(cudaGetDevice(&dev));
  PC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resident_multi_kernel, threads, smem));
  if (per_sm < 1) {
    set_error("resident solver: lattice does not fit one CTA");
    return PC_ERR_OOM;
  }
  long long grid = (long long)per_sm * nsm;
  if (grid > n_items) grid = n_items;
  ResidentBatch a = b;
  void* params[] = {&a};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)resident_multi_kernel;
  kp.gridDim = dim3((unsigned)(grid < 1 ? 1 : grid));
  kp.blockDim = dim3(threads);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = params;
  PC_CUDA(cudaGraphAddKernelNode(out, g, deps, ndeps, &kp));
  return PC_OK;
}

pc_status launch_resident(const ResidentArgs& args, int threads, cudaStream_t st) {
  void* func = nullptr;
  size_t smem = 0;
  long long grid = 0;
  pc_status rc = resident_config(args, threads, &func, &smem, &grid);
  if (rc) return rc;
  if (grid < 1) return PC_OK;
  resident_kernel<<<(unsigned)grid, threads, smem, st>>>(args);
  PC_CUDA(cudaGetLastError());
  return PC_OK;
}

}  // namespace pc

// blocked.cu -- the verdict-only (PC_BITS_ONLY) streamed solver with temporal
// blocking: 32 steps of the exact reached-set propagation per visit of a
// slab, the whole hexagonal cross-section held on chip by one thread-block
// cluster (Sec. II.B: only whether mass can reach a site matters, so the
// reached set R_m -- sites with nonzero mass at some step <= m -- decides
// the verdict; the first step that reaches the detector layer L-1 gives
// first_hit, the first step without growth m_stop).
//
// Why a cluster.  One step moves the reached set by at most one tube along
// the fibre, but across the cross-section the same-layer contacts jump two
// hexagon rows.  A tile of the cross-section would need a lateral halo of
// two rows per step, which at W = 64 (a hexagon 129 rows wide) leaves no
// useful interior after a few steps.  A cluster of up to 16 CTAs instead
// holds every column of the lattice (CTA r owns columns [r cpr, (r+1) cpr),
// one per thread), so the only halo is along t: one 32-tube word row above
// and below the slab, which 32 steps cannot cross.
//
// Slab ("tile") of a pass: valid word rows [w0, w0 + nw) plus the halo rows
// w0 - 1 and w0 + nw, in shared memory as quads: rows 4k .. 4k+3 of a column
// side by side in 16 bytes, [quad][cpr + 1] per array (entry cpr is the
// always-zero stand-in for contacts outside the hexagon), for the two
// reached-set buffers and the occupancy.  Each step reads a column's own
// words, its six same-layer contacts and the three up / three down contacts
// four rows at a time from the owning CTA's shared memory
// (ld.shared::cluster.v4: a warp's 32 columns stay one contiguous run, as
// distributed shared memory is served in 32-byte sectors), writes the new
// words to the other buffer, and ends with a cluster barrier.
// A step's growth and detector hit are ORed, per step, into a 32-bit mask of
// the configuration; valid rows of different slabs partition the layers, so
// the masks are exact.  After the pass the control kernel takes the first
// step that hit the detector or did not grow; the state after a terminating
// step is never used.
//
// Per configuration ("slot") in HBM: occupancy and two reached-set buffers,
// word [w][a] = tubes 32w .. 32w+31 of column a.  Rows are never cleaned: a
// pass starting after step m0 reads row w only if 32 w <= m0 (higher rows
// are empty at that step, whatever a previous configuration left there), and
// occupancy only up to the rows 32 steps can reach.  Occupancy is drawn
// lazily, one word row per pass, with the same Philox stream as every other
// path (counter (t A + a) >> 2, lane (t A + a) & 3).
//
// One tick = one pass kernel (persistent clusters taking slabs and draw
// rows from a counter) and one control kernel (one CTA per slot: masks ->
// outputs, refill, plan of the next pass).  The ticks run inside one CUDA
// graph's conditional WHILE node, whose condition the control kernel's last
// CTA sets, so the call stays asynchronous; with PC_STREAM_HOST_LOOP set the
// host launches them in chunks instead (profilers do not look inside graphs
// with conditional nodes).
#include <algorithm>
#include <cstdlib>

#include "blocked_plan.h"
#include "common.cuh"
#include "kernels.cuh"

namespace pc {

namespace {

constexpr int kSteps = kPassSteps;
constexpr int kMaxThreads = 800;  // columns per CTA: 80 registers a thread
constexpr int kMaxQuads = 9;      // slab rows / 4 in shared memory (valid rows + 2 halo rows)
constexpr int kCtlThreads = 256;
constexpr int kChunk = 16;       // ticks launched between reads of the completion count

inline size_t a256_host(size_t b) { return (b + 255) & ~(size_t)255; }

struct BSlot {
  long long item;    // configuration (index within the query)
  int phase;
  int m0;            // steps done
  int G;             // word rows of occupancy drawn
  int par;           // reached-set buffer holding step m0
  int tiles, draws;  // slabs and drawn rows of the pass in flight
  unsigned gmask;    // bit j: step m0 + 1 + j grew the reached set
  unsigned hmask;    // bit j: step m0 + 1 + j reached layer L - 1
};

struct BCtx {
  Lattice lat;
  OccStream occ;
  const uint32_t* occ_bits;
  int64_t words_per_cfg;
  int64_t n_cfg;
  uint32_t cfg0;
  Outputs out;
  int K;
  BSlot* slot;
  int* pre;                    // [K + 1] prefix of pass items over slots
  uint32_t* pool;              // per slot: occupancy, R0, R1 (TW x A words each)
  size_t slot_words;
  unsigned long long* work;    // next configuration
  unsigned long long* n_done;
  unsigned* next_item;
  unsigned* arrive;
  unsigned long long* ticks;   // passes run
  int cpr;                     // columns per CTA of a cluster
  int nrow;                    // slab rows in shared memory
  int nw;                      // valid rows per slab (nrow - 2)
  int use_cond;                // set the WHILE condition at the end of a pass
  int* error;                  // 1: the pass bound was reached (no correct run does)
  unsigned long long max_ticks;
  cudaGraphConditionalHandle cond;
  int cs;                      // CTAs per cluster the kernel was planned for
};

// --- cluster primitives (PTX ISA: mapa, ld.shared::cluster, barrier.cluster)
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster; orders shared-memory accesses
// before it against those after it, cluster-wide
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t map_rank(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t ldc(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

// Occupancy word (tubes 32 tw .. 32 tw + 31) of column a: the same stream as
// every other path draws.
__device__ inline uint32_t draw_word(const BCtx& x, long long rel, int tw, int a) {
  const int A = x.lat.A, L = x.lat.L;
  uint32_t word = 0;
  if (x.occ_bits) {
    const uint32_t* cb = x.occ_bits + (size_t)rel * x.words_per_cfg;
    for (int b = 0; b < 32; ++b) {
      const int t = tw * 32 + b;
      if (t >= L) break;
      const int64_t i = (int64_t)t * A + a;
      word |= ((cb[i >> 5] >> (i & 31)) & 1u) << b;
    }
  } else {
    const uint32_t cfg = x.cfg0 + (uint32_t)rel;
    for (int b = 0; b < 32; ++b) {
      const int t = tw * 32 + b;
      if (t >= L) break;
      const int64_t i = (int64_t)t * A + a;
      const u32x4 r = philox4x32_10(u32x4{(uint32_t)(i >> 2), cfg, x.occ.wl, 0u}, x.occ.k0, x.occ.k1);
      const uint32_t w = (i & 3) == 0 ? r.x : (i & 3) == 1 ? r.y : (i & 3) == 2 ? r.z : r.w;
      word |= (uint32_t)((uint64_t)w < x.occ.T) << b;
    }
  }
  return word;
}

// Items of a slot's next pass (slabs, then rows to draw).
__device__ inline void plan_slot(const BCtx& x, BSlot& c) {
  const PassItems p = pass_items(c.phase, c.m0, c.G, x.lat.TW, x.nw);
  c.tiles = p.tiles; c.draws = p.draws;
}

__device__ inline void take(const BCtx& x, BSlot& c, unsigned long long item) {
  c.item = (long long)item; c.m0 = 0; c.G = 0; c.par = 0; c.gmask = 0u; c.hmask = 0u;
  c.phase = (long long)item < x.n_cfg ? BP_DRAW0 : BP_EMPTY;
  plan_slot(x, c);
}

// Exclusive prefix over the slots of their pass items, by one block (each
// thread a contiguous run of slots, then a scan of the per-thread sums).
// Other CTAs wrote the slot records: they are read through L2 (__ldcg), not
// from a line this SM's L1 may hold from before.
__device__ void prefix_items(const BCtx& x) {
  __shared__ int s_part[32];
  const int tid = threadIdx.x, T = blockDim.x;
  const int per = (x.K + T - 1) / T;
  const int b0 = min(tid * per, x.K), b1 = min(b0 + per, x.K);
  int sum = 0;
  for (int s = b0; s < b1; ++s) sum += __ldcg(&x.slot[s].tiles) + __ldcg(&x.slot[s].draws);
  const int lane = tid & 31, warp = tid >> 5;
  int v = sum;  // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  if (lane == 31) s_part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int w = lane < (T >> 5) ? s_part[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += n;
    }
    s_part[lane] = w;
  }
  __syncthreads();
  int run = v - sum + (warp ? s_part[warp - 1] : 0);
  for (int s = b0; s < b1; ++s) {
    x.pre[s] = run;
    run += __ldcg(&x.slot[s].tiles) + __ldcg(&x.slot[s].draws);
  }
  if (tid == T - 1) x.pre[x.K] = run;
  __syncthreads();
}

__global__ void blocked_init_kernel(BCtx x) {
  for (int s = threadIdx.x; s < x.K; s += blockDim.x) {
    BSlot c;
    take(x, c, (unsigned long long)s);
    x.slot[s] = c;
  }
  __threadfence();  // the prefix reads the records through L2
  __syncthreads();
  prefix_items(x);
  if (threadIdx.x == 0) {
    *x.work = (unsigned long long)x.K;
    *x.n_done = 0ull; *x.next_item = 0u; *x.arrive = 0u; *x.ticks = 0ull; *x.error = 0;
  }
}

__device__ __forceinline__ uint4 ldc4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
  return v;
}
__device__ __forceinline__ uint4 lds4(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
  return v;
}
__device__ __forceinline__ void sts4(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" :: "r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ uint32_t lds_r(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ uint4 or4(uint4 a, uint4 b) { return make_uint4(a.x | b.x, a.y | b.y, a.z | b.z, a.w | b.w); }
__device__ __forceinline__ uint32_t q_at(const uint4& v, int r) { return r == 0 ? v.x : r == 1 ? v.y : r == 2 ? v.z : v.w; }

// One pass: every slab of every active slot (32 steps each) and the rows to
// draw.  Grid = whole clusters, persistent; items are taken cluster-wide.
//
// Shared memory of a CTA: three arrays (reached set, buffers 0 and 1, and
// occupancy), each [quad][column] of 16 bytes: slab rows 4k .. 4k+3 of a
// column side by side, so one 128-bit load brings four rows of a contact and
// a warp's 32 columns stay one contiguous run (distributed shared memory is
// served in 32-byte sectors).
__global__ void __launch_bounds__(kMaxThreads, 1) blocked_pass_kernel(BCtx x) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int s_item[2];
  __shared__ unsigned s_g, s_h;
  const int tid = threadIdx.x, nt = blockDim.x;
  {
    // launched without the planned cluster shape: no distributed shared
    // memory access; every CTA of the (same-sized) cluster returns here
    uint32_t ncta;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
    if ((int)ncta != x.cs) {
      if (tid == 0) atomicOr(x.error, 4);
      return;
    }
  }
  const uint32_t rank = cluster_rank();
  const int A = x.lat.A, L = x.lat.L, TW = x.lat.TW;
  const int stride = x.cpr + 1;                 // columns per quad row (column cpr: zero)
  const int nq = x.nrow >> 2;                   // quads per array
  const uint32_t qrow = (uint32_t)stride * 16u;  // bytes per quad row
  const uint32_t arr = (uint32_t)nq * qrow;      // bytes per array
  const int c0 = (int)rank * x.cpr;
  const int ncol = max(0, min(x.cpr, A - c0));
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(sm);
  for (int i = tid; i < 3 * nq; i += nt) sts4(base + (uint32_t)i * qrow + (uint32_t)x.cpr * 16u, make_uint4(0, 0, 0, 0));
  if (tid == 0) { s_g = 0u; s_h = 0u; }
  const bool own = tid < ncol;
  const int col = c0 + tid;
  const uint32_t me = base + (uint32_t)(own ? tid : x.cpr) * 16u;  // quad 0 of this column, buffer 0
  uint32_t nb[kLateral];  // cluster addresses of the contacts' quad 0, buffer 0
  int sg = 0;
  if (own) {
    sg = x.lat.sigma[col];
#pragma unroll
    for (int d = 0; d < kLateral; ++d) {
      // a contact outside the hexagon reads the zero column
      const int j = x.lat.nbr[col * kLateral + d];
      const int r = j >= A ? (int)rank : j / x.cpr;
      const int l = j >= A ? x.cpr : j - r * x.cpr;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(nb[d]) : "r"(base + (uint32_t)l * 16u), "r"((uint32_t)r));
    }
  } else {
#pragma unroll
    for (int d = 0; d < kLateral; ++d)
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(nb[d]) : "r"(me), "r"(rank));
  }
  // the up contacts reach tube t+1 from sigma = 2, the down contacts tube t-1
  // from sigma = 0: one funnel shift of their ORed words
  const uint32_t sh_up = sg == 2 ? 1u : 0u, sh_dn = sg == 0 ? 1u : 0u;
  const int endw = (L - 1) >> 5, endb = (L - 1) & 31;
  const uint32_t item_addr = map_rank(&s_item[0], 0u);
  cluster_sync_all();

  for (int it = 0;; ++it) {
    if (rank == 0 && tid == 0) s_item[it & 1] = (int)atomicAdd(x.next_item, 1u);
    cluster_sync_all();
    const int item = (int)ldc(item_addr + 4u * (uint32_t)(it & 1));
    if (item >= x.pre[x.K]) break;  // the same value in every CTA of the cluster
    int lo = 0, hi = x.K - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (x.pre[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const int s = lo;
    const BSlot c = x.slot[s];
    const int local = item - x.pre[s];
    // slot arrays: occupancy, then the reached-set buffers R0 and R1
    const size_t plane = (size_t)TW * A;

    if (local >= c.tiles) {  // one row of occupancy for the next pass
      const int tw = c.G + (local - c.tiles);
      if (own && tw < TW) x.pool[(size_t)s * x.slot_words + (size_t)tw * A + col] = draw_word(x, c.item, tw, col);
      continue;
    }

    // slab: local row i holds word row w0 - 1 + i
    const Slab sb = slab_of(local, c.m0, TW, x.nw, x.nrow);
    const int w0 = sb.w0, m0 = c.m0;
    const int n_eff = sb.n_eff;              // rows above the top row stay empty for 32 steps
    const int q_eff = (n_eff + 3) >> 2;      // quads computed (rows past n_eff loaded as zero)
    const int ivmax = sb.ivmax;              // valid rows 1 .. ivmax
    const int iend = endw - (w0 - 1);
    const bool end_here = iend >= 1 && iend <= ivmax;
    if (own) {
      const uint32_t* occw = x.pool + (size_t)s * x.slot_words;
      const uint32_t* Rs = occw + plane * (size_t)(1 + c.par);
      for (int k = 0; k < q_eff; ++k) {
        uint32_t rv[4], ov[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int i = 4 * k + r, wi = w0 - 1 + i;
          const bool in = wi >= 0 && i < n_eff;
          rv[r] = (in && wi * 32 <= m0) ? __ldcs(Rs + (size_t)wi * A + col) : 0u;
          ov[r] = in ? __ldcs(occw + (size_t)wi * A + col) : 0u;
        }
        sts4(me + (uint32_t)k * qrow, make_uint4(rv[0], rv[1], rv[2], rv[3]));
        sts4(me + 2u * arr + (uint32_t)k * qrow, make_uint4(ov[0], ov[1], ov[2], ov[3]));
      }
    }
    cluster_sync_all();
    for (int j = 0; j < kSteps; ++j) {
      const uint32_t so = (j & 1) ? arr : 0u, dso = (j & 1) ? 0u : arr;
      bool grow = false, hit = false;
      if (own) {
        uint32_t diff = 0u, prevw = 0u, dnl = 0u;
        uint4 cur = lds4(me + so);
        uint4 upc = or4(or4(ldc4(nb[6] + so), ldc4(nb[7] + so)), ldc4(nb[8] + so));
        for (int k = 0; k < q_eff; ++k) {
          const uint32_t ko = so + (uint32_t)k * qrow;
          uint4 ownn = make_uint4(0, 0, 0, 0), upn = make_uint4(0, 0, 0, 0);
          if (k + 1 < q_eff) {
            ownn = lds4(me + ko + qrow);
            upn = ldc4(nb[6] + ko + qrow);
            upn = or4(upn, ldc4(nb[7] + ko + qrow));
            upn = or4(upn, ldc4(nb[8] + ko + qrow));
          }
          uint4 dn = ldc4(nb[9] + ko);
          dn = or4(dn, ldc4(nb[10] + ko));
          dn = or4(dn, ldc4(nb[11] + ko));
          uint4 sl = ldc4(nb[0] + ko);
          sl = or4(sl, ldc4(nb[1] + ko));
          sl = or4(sl, ldc4(nb[2] + ko));
          sl = or4(sl, ldc4(nb[3] + ko));
          sl = or4(sl, ldc4(nb[4] + ko));
          sl = or4(sl, ldc4(nb[5] + ko));
          const uint4 oc = lds4(me + 2u * arr + (uint32_t)k * qrow);
          // rows of this quad that are valid (slab rows 1 .. ivmax)
          const int i0 = 4 * k;
          uint32_t out[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const uint32_t cw = q_at(cur, r);
            const uint32_t pw = r == 0 ? prevw : q_at(cur, r - 1);
            const uint32_t nw = r == 3 ? ownn.x : q_at(cur, r + 1);
            const uint32_t uh = r == 3 ? upn.x : q_at(upc, r + 1);
            const uint32_t dl = r == 0 ? dnl : q_at(dn, r - 1);
            // end contacts (tubes t-1, t+1), same-layer contacts, and the up /
            // down contacts at tube t+1 (sigma = 2) / t-1 (sigma = 0)
            uint32_t acc = __funnelshift_l(pw, cw, 1) | __funnelshift_r(cw, nw, 1) | q_at(sl, r);
            acc |= __funnelshift_r(q_at(upc, r), uh, sh_up) | __funnelshift_l(dl, q_at(dn, r), sh_dn);
            out[r] = cw | (acc & q_at(oc, r));
            const int i = i0 + r;
            if (i >= 1 && i <= ivmax) diff |= out[r] ^ cw;
          }
          sts4(me + dso + (uint32_t)k * qrow, make_uint4(out[0], out[1], out[2], out[3]));
          prevw = cur.w; dnl = dn.w; cur = ownn; upc = upn;
        }
        grow = diff != 0u;
        if (end_here) {  // the detector layer's word, before and after
          const uint32_t off = (uint32_t)(iend >> 2) * qrow + 4u * (uint32_t)(iend & 3);
          const uint32_t a = lds_r(me + so + off), b = lds_r(me + dso + off);
          hit = (((b & ~a) >> endb) & 1u) != 0u;
        }
      }
      if (__any_sync(0xffffffffu, grow) && (tid & 31) == 0) atomicOr(&s_g, 1u << j);
      if (__any_sync(0xffffffffu, hit) && (tid & 31) == 0) atomicOr(&s_h, 1u << j);
      cluster_sync_all();
    }
    // after an even number of steps the state is back in buffer 0
    if (own) {
      uint32_t* Rd = x.pool + (size_t)s * x.slot_words + plane * (size_t)(2 - c.par);
      for (int i = 1; i <= ivmax; ++i)
        Rd[(size_t)(w0 - 1 + i) * A + col] = lds_r(me + (uint32_t)(i >> 2) * qrow + 4u * (uint32_t)(i & 3));
    }
    if (tid == 0) {
      if (s_g) atomicOr(&x.slot[s].gmask, s_g);
      if (s_h) atomicOr(&x.slot[s].hmask, s_h);
      s_g = 0u; s_h = 0u;
    }
  }
  cluster_sync_all();  // no CTA leaves while another may still read its shared memory
}

// One CTA per slot: the pass's masks -> outputs or the next pass.
__global__ void __launch_bounds__(kCtlThreads) blocked_control_kernel(BCtx x) {
  __shared__ int s_n0;
  __shared__ bool s_last;
  const int s = blockIdx.x, tid = threadIdx.x;
  BSlot c = x.slot[s];
  if (c.phase != BP_EMPTY) {
    const int A = x.lat.A, L = x.lat.L, TW = x.lat.TW;
    uint32_t* occw = x.pool + (size_t)s * x.slot_words;
    uint32_t* R0 = occw + (size_t)TW * A;
    bool finish = false;
    int verdict = 0, fh = -1, mstop = 0;
    if (c.phase == BP_DRAW0) {
      c.G = c.draws;
      // m = 0: the metallic sites of layer 0
      if (tid == 0) s_n0 = 0;
      __syncthreads();
      int cnt = 0;
      for (int a = tid; a < A; a += blockDim.x) {
        const uint32_t b = occw[a] & 1u;
        R0[a] = b;
        cnt += (int)b;
      }
      cnt = __reduce_add_sync(0xffffffffu, cnt);
      if ((tid & 31) == 0 && cnt) atomicAdd(&s_n0, cnt);
      __syncthreads();
      if (s_n0 == 0) {
        finish = true;
      } else if (L == 1) {
        finish = true; verdict = 1; fh = 1; mstop = 1;
      } else {
        c.phase = BP_STEP; c.m0 = 0; c.par = 0; c.gmask = 0u; c.hmask = 0u;
      }
    } else {  // BP_STEP
      c.G += c.draws;
      // first step of the pass that reached the detector or did not grow
      const PassOutcome o = pass_outcome(c.gmask, c.hmask, c.m0);
      c.gmask = 0u; c.hmask = 0u;
      if (o.finish) {
        finish = true; verdict = o.verdict; fh = o.first_hit; mstop = o.m_stop;
      } else {
        c.m0 += kSteps; c.par ^= 1;
      }
    }
    if (tid == 0) {
      if (finish) {
        const long long rel = c.item;
        x.out.verdict[rel] = (uint8_t)verdict;
        if (x.out.first_hit) x.out.first_hit[rel] = fh;
        if (x.out.mass) x.out.mass[rel] = 0.f;
        if (x.out.m_stop) x.out.m_stop[rel] = mstop;
        if (verdict && x.out.n_perc) atomicAdd(x.out.n_perc, 1ull);
        atomicAdd(x.n_done, 1ull);
        take(x, c, atomicAdd(x.work, 1ull));
      } else {
        plan_slot(x, c);
      }
      x.slot[s] = c;
    }
  }
  // last CTA: prefix of the next pass's items
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(x.arrive, 1u) == (unsigned)(gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  prefix_items(x);
  if (tid == 0) {
    *x.arrive = 0u;
    *x.next_item = 0u;
    const unsigned long long t = *x.ticks + 1ull;
    *x.ticks = t;
    if (x.use_cond) {  // the loop ends when every configuration is done
      const bool more = __ldcg(x.n_done) < (unsigned long long)x.n_cfg;
      if (more && t >= x.max_ticks) *x.error = 1;
      cudaGraphSetConditional(x.cond, (more && t < x.max_ticks) ? 1u : 0u);
    }
  }
}

}  // namespace

struct Shape {
  int cs = 0, cpr = 0, threads = 0, nrow = 0, smem = 0, clusters = 0;
};

// Smallest cluster that holds the cross-section (at most 800 columns per
// CTA) with a slab of at least 3 quads (12 rows, 10 valid), and that the
// device can run.
bool pick_shape(const Lattice& lat, Shape* out) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  const int budget = optin - 64;  // static shared memory of the kernel
  if (cudaFuncSetAttribute(blocked_pass_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
    cudaGetLastError();
  for (int cs = 1; cs <= 16; cs *= 2) {
    const int cpr = (lat.A + cs - 1) / cs;
    if (cpr > kMaxThreads) continue;
    const int nq = std::min(kMaxQuads, budget / (48 * (cpr + 1)));
    if (nq < 3) continue;
    Shape s;
    s.cs = cs; s.cpr = cpr; s.threads = (cpr + 31) / 32 * 32; s.nrow = 4 * nq;
    s.smem = 48 * (cpr + 1) * nq;
    if (cudaFuncSetAttribute(blocked_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, s.smem) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cs; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)cs); cfg.blockDim = dim3((unsigned)s.threads);
    cfg.dynamicSmemBytes = (size_t)s.smem; cfg.attrs = at; cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, blocked_pass_kernel, &cfg) != cudaSuccess || n < 1) {
      cudaGetLastError();
      continue;
    }
    s.clusters = n;
    *out = s;
    return true;
  }
  return false;
}

bool blocked_takes(const Lattice& lat) {
  Shape sh;
  return !std::getenv("PC_BITS_STEPWISE") && pick_shape(lat, &sh);
}

pc_status run_blocked(const StreamJob& job, cudaStream_t st, bool* handled) {
  *handled = false;
  if (!job.bits_only || job.sel || job.n_cfg <= 0 || std::getenv("PC_BITS_STEPWISE")) return PC_OK;
  Shape sh;
  if (!pick_shape(job.lat, &sh)) return PC_OK;  // the step-synchronous solver takes it
  const Lattice& lat = job.lat;
  const size_t slot_words = 3 * (size_t)lat.TW * lat.A;
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  long long kmax = (long long)(free_b / 2 / (slot_words * 4 + 64));
  // enough slots that every cluster has slabs to take, as far as memory allows
  // as many configurations in flight as memory allows (short-lived ones
  // leave little work per pass otherwise)
  long long K = std::min<long long>(job.n_cfg, std::min<long long>(kmax, 4096));
  if (K < 1) { set_error("verdict-only solver: no memory for one configuration"); return PC_ERR_OOM; }

  const size_t head = 256 + a256_host(sizeof(BSlot) * (size_t)K) + a256_host(4 * (size_t)(K + 1));
  static_assert(sizeof(unsigned long long) * 3 + 4 * 3 <= 256, "counters fit the head");
  char* mem = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&mem, head + slot_words * 4 * (size_t)K, st);
  if (e != cudaSuccess) return cuda_fail(e, "verdict-only solver state");
  BCtx x;
  x.lat = lat; x.occ = job.occ; x.occ_bits = job.occ_bits; x.words_per_cfg = job.words_per_cfg;
  x.n_cfg = job.n_cfg; x.cfg0 = job.cfg0; x.out = job.out; x.K = (int)K;
  unsigned long long* ctr = (unsigned long long*)mem;
  x.work = ctr; x.n_done = ctr + 1; x.ticks = ctr + 2;
  x.next_item = (unsigned*)(ctr + 3); x.arrive = x.next_item + 1; x.error = (int*)(x.next_item + 2);
  x.slot = (BSlot*)(mem + 256);
  x.pre = (int*)(mem + 256 + a256_host(sizeof(BSlot) * (size_t)K));
  x.pool = (uint32_t*)(mem + head);
  x.slot_words = slot_words;
  x.cpr = sh.cpr; x.nrow = sh.nrow; x.nw = sh.nrow - 2;
  // a configuration needs at most (sites / 32 + 3) passes: the reached set
  // grows by at least one site per step until it stops
  const long long per_cfg = (long long)(lat.N / kSteps) + 3;
  const long long rounds = (job.n_cfg + K - 1) / K;
  x.max_ticks = (unsigned long long)std::min<long long>(per_cfg * rounds, 1ll << 40);
  x.use_cond = 0;
  x.cond = 0;
  x.cs = sh.cs;

  pc_status rc = PC_OK;
  const unsigned grid = (unsigned)(sh.cs * sh.clusters);
  if (std::getenv("PC_STREAM_HOST_LOOP")) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)sh.cs; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(grid); cfg.blockDim = dim3((unsigned)sh.threads);
    cfg.dynamicSmemBytes = (size_t)sh.smem; cfg.stream = st; cfg.attrs = at; cfg.numAttrs = 1;
    unsigned long long* done_h = nullptr;
    e = cudaMallocHost((void**)&done_h, sizeof(unsigned long long));
    if (e != cudaSuccess) { cudaFreeAsync(mem, st); return cuda_fail(e, "pinned count"); }
    *done_h = 0;
    blocked_init_kernel<<<1, 256, 0, st>>>(x);
    e = cudaGetLastError();
    unsigned long long ticks = 0;
    while (e == cudaSuccess && *done_h < (unsigned long long)job.n_cfg) {
      for (int i = 0; i < kChunk && e == cudaSuccess; ++i) {
        e = cudaLaunchKernelEx(&cfg, blocked_pass_kernel, x);
        if (e == cudaSuccess) {
          blocked_control_kernel<<<x.K, kCtlThreads, 0, st>>>(x);
          e = cudaGetLastError();
        }
      }
      ticks += kChunk;
      if (e == cudaSuccess) e = cudaMemcpyAsync(done_h, x.n_done, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e == cudaSuccess && ticks > x.max_ticks && *done_h < (unsigned long long)job.n_cfg) {
        set_error("verdict-only solver did not converge");
        rc = PC_ERR_INTERNAL;
        break;
      }
    }
    int err = 0;
    if (e == cudaSuccess && rc == PC_OK) {
      e = cudaMemcpyAsync(&err, x.error, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "verdict-only solver");
    else if (err) { set_error("verdict-only solver: device check failed"); rc = PC_ERR_INTERNAL; }
    cudaFreeHost(done_h);
    cudaFreeAsync(mem, st);
    *handled = true;
    return rc;
  }
  // init -> WHILE(pass, control), one graph
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  do {
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) break;
    if ((e = cudaGraphConditionalHandleCreate(&x.cond, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    x.use_cond = 1;
    void* args[] = {&x};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)blocked_init_kernel;
    kp.gridDim = dim3(1); kp.blockDim = dim3(256); kp.kernelParams = args;
    cudaGraphNode_t n_init, n_while, n_pass, n_ctl;
    if ((e = cudaGraphAddKernelNode(&n_init, g, nullptr, 0, &kp)) != cudaSuccess) break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = x.cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&n_while, g, &n_init, nullptr, 1, &cp)) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaKernelNodeParams pp = {};
    pp.func = (void*)blocked_pass_kernel;
    pp.gridDim = dim3(grid); pp.blockDim = dim3((unsigned)sh.threads);
    pp.sharedMemBytes = (unsigned)sh.smem; pp.kernelParams = args;
    if ((e = cudaGraphAddKernelNode(&n_pass, body, nullptr, 0, &pp)) != cudaSuccess) break;
    cudaKernelNodeAttrValue cv = {};
    cv.clusterDim.x = (unsigned)sh.cs; cv.clusterDim.y = 1; cv.clusterDim.z = 1;
    if ((e = cudaGraphKernelNodeSetAttribute(n_pass, cudaLaunchAttributeClusterDimension, &cv)) != cudaSuccess) break;
    cudaKernelNodeParams cpk = {};
    cpk.func = (void*)blocked_control_kernel;
    cpk.gridDim = dim3((unsigned)x.K); cpk.blockDim = dim3(kCtlThreads); cpk.kernelParams = args;
    if ((e = cudaGraphAddKernelNode(&n_ctl, body, &n_pass, 1, &cpk)) != cudaSuccess) break;
    if ((e = cudaGraphInstantiate(&ex, g, 0)) != cudaSuccess) break;
    if ((e = cudaGraphLaunch(ex, st)) != cudaSuccess) break;
    if (job.error_out) e = cudaMemcpyAsync(job.error_out, x.error, sizeof(int), cudaMemcpyDeviceToDevice, st);
  } while (0);
  if (e != cudaSuccess) rc = cuda_fail(e, "verdict-only solver graph");
  if (ex) cudaGraphExecDestroy(ex);  // an in-flight executable is freed on completion
  if (g) cudaGraphDestroy(g);
  cudaFreeAsync(mem, st);
  *handled = true;
  return rc;
}

}  // namespace pc

extern "C" pc_status pc_bits_blocked_shape(int32_t W, int32_t* cluster_size, int32_t* columns_per_cta,
                                           int32_t* slab_rows, int32_t* clusters) {
  if (W < 0 || W > 255) { pc::set_error("pc_bits_blocked_shape: W must be in [0, 255]"); return PC_ERR_ARG; }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return pc::cuda_fail(e, "pc_bits_blocked_shape");
  pc::Lattice lat{};
  lat.W = W; lat.A = 3 * W * (W + 1) + 1;
  pc::Shape s;
  if (!pc::pick_shape(lat, &s)) {
    pc::set_error("pc_bits_blocked_shape: no cluster of this device holds the cross-section");
    return PC_ERR_ARG;
  }
  if (cluster_size) *cluster_size = s.cs;
  if (columns_per_cta) *columns_per_cta = s.cpr;
  if (slab_rows) *slab_rows = s.nrow;
  if (clusters) *clusters = s.clusters;
  return PC_OK;
}

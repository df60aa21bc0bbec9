// stream.cu -- streamed solver for lattices whose state exceeds one CTA's
// shared memory (Sec. II.B, Eqs. (2)-(4) on the lattice of Sec. II.A), for one
// or many queries (W, L, p, seed, configuration range) at once.
//
// K "slots" each hold one configuration's state in HBM:
//   nu[2][(L+4) planes] FP32  nu = mu / deg (ping-pong), layer t in plane t+2
//                          of the padded-row layout (lattice.cu); planes 0, 1,
//                          L+2, L+3 and all padding zero
//   dg[L planes]     u8    deg(i) for metallic sites (Eq. (2), detector edge
//                          included on t = L-1), 0 elsewhere
//   occw, R[2]       bits  occupancy and reached set, words [tw+1][a] of 32
//                          consecutive tube indices of column a
// A slot takes configurations from a global work list (all queries, largest
// lattices first) and is refilled as soon as its configuration finishes.
// The device runs "ticks" inside one CUDA graph conditional WHILE node:
//   sweep   : a persistent grid takes work units over all slots from a
//             per-tick counter -- FP32 site updates of step m over the causal
//             window t <= m (a chunk of 256 strips walks up 128 layers; the
//             plane segment and degree bytes the chunk reads are staged into
//             shared memory by bulk copies (TMA) through a ring of up to 6
//             slots, freed two layers at a time), the exact bit-parallel
//             reached-set update, and lazy preparation of the layers just
//             ahead of the window (Philox draw of a word row, degrees,
//             zeroing of nu and R rows);
//   control : one CTA per slot reads the step's grow / end flags, sums the
//             detector mass on a hit (deterministic block reduction), writes
//             the outputs, refills the slot and plans its next tick; the last
//             CTA to finish prefix-sums the plans and sets the loop condition.
// No host round trip between ticks; the loop ends when every configuration is
// done or after a tick bound that no correct run reaches (then an error flag
// is raised for the host).
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "plan.h"
#include "tiling.cuh"
#include "tma.cuh"

namespace pc {

namespace {

constexpr uint32_t kGrow = 1u, kEnd = 2u;
constexpr int kCols = 256;    // columns per unit == threads per sweep CTA
constexpr int kRows = 16;     // word rows per BITS unit
constexpr int kBitsCols = 2;  // columns per thread of a BITS unit
constexpr int kRowsFP = 128;  // layers per FP unit (the ring prologue is paid once per unit)
constexpr int kMaxRing = 6;  // ring slots: planes in flight ahead of the compute (deeper rings cost L1)
// shared memory the ring may take per CTA: at least two sweep CTAs fit on an
// SM (at W = 64 six slots take 39.4 KB, and three CTAs fit)
constexpr int kRingBudget = 104 * 1024;
constexpr int kMaxSlots = 4096;

// ring depth for slots of cap entries (4 B of nu + 1 B of degree each): as
// deep as the budget allows, at least 3 (a layer reads two planes and needs
// one in flight)
inline int ring_depth(int cap) {
  const int n = kRingBudget / (cap * (int)(sizeof(float) + 1));
  return n < 3 ? 3 : n > kMaxRing ? kMaxRing : n;
}

// dynamic shared memory of the sweep kernel: the ring (nring slots of cap
// FP32 entries, then nring of cap degree bytes) and the tick's unit prefix
// over the K slots (K + 1 ints)
__host__ __device__ inline int ring_bytes(int cap, int nring) { return (nring * cap * (int)(sizeof(float) + 1) + 15) & ~15; }
inline int sweep_smem_bytes(int cap, int nring, int K) { return ring_bytes(cap, nring) + 4 * (K + 1); }

struct QDev {
  Lattice lat;
  OccStream occ;
  const uint32_t* occ_bits;
  int64_t words_per_cfg;
  int64_t n_cfg;
  uint32_t cfg0;
  Outputs out;
  long long item0;  // first global work item of this query
  int bits_only;    // reached set only: no FP units, mass written 0
  const int64_t* sel;  // item i of the query solves configuration sel[i] (null: configuration i)
};

// configuration (index within its query) that work item i of query Q solves
__device__ inline long long config_of(const QDev& Q, long long i) { return Q.sel ? Q.sel[i] : i; }

struct __align__(16) Ctl {
  long long item;       // global work item in the slot
  int q;                // query of that item
  int phase;
  int m;                // step being computed (PH_STEP)
  int G;                // layers with occupancy drawn (multiple of 32, or L)
  int F;                // layers with degrees and cleaned nu / R rows
  unsigned int flags;   // grow / end of the step in flight
  int units[U_KINDS];   // this tick's units per kind
};

struct Ctx {
  const QDev* qs;
  int nq;
  long long n_items;
  int K;
  Ctl* ctl;
  int* pre;                    // [K + 1] exclusive prefix of units over slots
  char* pool;
  size_t slot_bytes;
  unsigned long long* work;    // next work item
  unsigned long long* n_done;  // finished configurations
  unsigned int* ticks;
  unsigned int* arrive;        // control blocks finished this tick
  unsigned int* next_unit;     // next unit of this tick's sweep
  int* error;
  unsigned int max_ticks;
  cudaGraphConditionalHandle cond;
  int seg_cap;                  // floats per shared-memory ring slot of the FP units
  int nring;                    // ring slots (3 .. kMaxRing)
  int fp;                       // some query runs the FP32 recursion (else: the bits-only kernel)
  int use_cond;                 // set the WHILE condition at the end of a tick
  int server;                   // 1: slots are bound to a query by the host
  char** slot_base;             // [K] state of each slot (server mode)
  unsigned long long* qnext;    // [nq] next configuration of a query (server mode)
  unsigned long long* qdone;    // [nq] finished configurations (server mode)
};


// items along the plane / column axis of one unit row, per kind: strip pairs
// for FP, plane positions for PREP and CLEAN, columns for BITS and DRAW
__host__ __device__ inline int width_of(int kind, const Lattice& lat) {
  if (kind == U_FP) {  // strip pairs of the paired layout
    const int s_end = lat.s_begin + lat.n_strips;
    return ((s_end + 1) >> 1) - (lat.s_begin >> 1);
  }
  return (kind == U_PREP || kind == U_CLEAN) ? lat.P : lat.A;
}

// items of one unit row per kind (a BITS unit thread takes kBitsCols columns)
__host__ __device__ inline int unit_width(int kind) { return kind == U_BITS ? kCols * kBitsCols : kCols; }

__host__ __device__ inline int units_of(int kind, int lo, int hi, const Lattice& lat) {
  if (hi <= lo) return 0;
  const int ccol = (width_of(kind, lat) + unit_width(kind) - 1) / unit_width(kind);
  const int per = (kind == U_DRAW || kind == U_CLEAN) ? 1 : kind == U_FP ? kRowsFP : kind == U_PREP ? 32 : kRows;
  return ccol * ((hi - lo + per - 1) / per);
}

// Sub-arrays of a slot for lattice lat.
struct SlotView {
  float* nu0; float* nu1; uint8_t* dg; uint32_t* occw; uint32_t* R0; uint32_t* R1;
};

__host__ __device__ inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

__host__ __device__ inline size_t slot_bytes_of(int A, int L, int P) {
  const size_t S = (size_t)A + 1, TWP = (size_t)(L + 31) / 32 + 2;
  return 2 * a256(sizeof(float) * (size_t)(L + 4) * P) + a256((size_t)L * P) +
         3 * a256(sizeof(uint32_t) * TWP * S);
}

__device__ inline SlotView view_of(const Ctx& x, int slot, const Lattice& lat) {
  const size_t S = (size_t)lat.S;
  char* b = x.server ? x.slot_base[slot] : x.pool + (size_t)slot * x.slot_bytes;
  SlotView v;
  const size_t nu_b = a256(sizeof(float) * (size_t)(lat.L + 4) * lat.P);
  const size_t w_b = a256(sizeof(uint32_t) * (size_t)lat.TWP * S);
  v.nu0 = (float*)b; b += nu_b;
  v.nu1 = (float*)b; b += nu_b;
  v.dg = (uint8_t*)b; b += a256((size_t)lat.L * lat.P);
  v.occw = (uint32_t*)b; b += w_b;
  v.R0 = (uint32_t*)b; b += w_b;
  v.R1 = (uint32_t*)b;
  return v;
}

__device__ inline uint32_t bit_at(const uint32_t* w, int S, int col, int tt) {
  return (w[((tt >> 5) + 1) * S + col] >> (tt & 31)) & 1u;
}

// query of a global work item (queries are few; linear scan)
__device__ inline int query_of(const Ctx& x, long long item) {
  int q = 0;
  while (q + 1 < x.nq && x.qs[q + 1].item0 <= item) ++q;
  return q;
}

__device__ inline void fill_plan(Ctl& c, const QDev& Q) {
  const Plan p = make_plan(c.phase, c.m, c.G, c.F, Q.lat.L, Q.lat.TW);
  for (int k = 0; k < U_KINDS; ++k) c.units[k] = units_of(k, p.lo[k], p.hi[k], Q.lat);
  if (Q.bits_only) c.units[U_FP] = 0;
}

__device__ inline void assign(const Ctx& x, Ctl& c, unsigned long long item) {
  c.item = (long long)item; c.m = 0; c.G = 0; c.F = 0; c.flags = 0u;
  for (int k = 0; k < U_KINDS; ++k) c.units[k] = 0;
  if ((long long)item < x.n_items) {
    c.q = query_of(x, (long long)item);
    c.phase = PH_DRAW0;
    fill_plan(c, x.qs[c.q]);
  } else {
    c.q = 0; c.phase = PH_EMPTY;
  }
}

// exclusive prefix over slots of the unit totals, by one block
__device__ void plan_prefix(const Ctx& x) {
  __shared__ int s_part[32];
  const int tid = threadIdx.x, T = blockDim.x;
  const int per = (x.K + T - 1) / T;
  const int b0 = tid * per, b1 = min(b0 + per, x.K);
  int sum = 0;
  // other blocks wrote these records: read through L2, not a stale L1 line
  for (int s = b0; s < b1; ++s) {
    const int4 u = __ldcg((const int4*)x.ctl[s].units);
    sum += u.x + u.y + u.z + u.w + __ldcg(&x.ctl[s].units[4]);
  }
  // block exclusive scan of per-thread sums (warp shuffles + 32 partials)
  const int lane = tid & 31, warp = tid >> 5;
  int v = sum;
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
    const int4 u = __ldcg((const int4*)x.ctl[s].units);
    run += u.x + u.y + u.z + u.w + __ldcg(&x.ctl[s].units[4]);
  }
  if (tid == T - 1) x.pre[x.K] = run;
  __syncthreads();
}

// Query table upload through kernel parameters: asynchronous, and no
// pageable host copy (which would synchronise the caller's stream).
constexpr int kQChunk = 16;
struct QChunk {
  int n, base;
  QDev q[kQChunk];
};

__global__ void upload_queries_kernel(QDev* dst, QChunk c) {
  if ((int)threadIdx.x < c.n) dst[c.base + threadIdx.x] = c.q[threadIdx.x];
}

__global__ void __launch_bounds__(1024) stream_init_kernel(Ctx x) {
  for (int s = threadIdx.x; s < x.K; s += blockDim.x) {
    Ctl c;
    assign(x, c, (unsigned long long)s);
    x.ctl[s] = c;
  }
  if (threadIdx.x == 0) {
    *x.work = (unsigned long long)x.K;
    *x.n_done = 0ull;
    *x.ticks = 0u;
    *x.arrive = 0u;
    *x.next_unit = 0u;
    *x.error = 0;
  }
  __threadfence();
  __syncthreads();
  plan_prefix(x);
}


// Ring state carried across the FP units of one CTA.  Planes are copied
// and consumed strictly in order, round robin over the nring slots, across
// units too, so the slot of the next plane to consume and the parity of its
// barrier's phase follow from one cursor, and the slot of the next plane to
// copy from another.  Every thread keeps both (they are identical in all
// threads); the copies are issued by lane 0 of the warps in turn.  Every
// plane a unit issues is consumed by the same unit.
struct Ring {
  int slot;       // slot of the next plane to consume
  uint32_t par;   // parity of that slot's current phase (flips once per round)
  int wslot;      // slot of the next plane to copy
  int pending;    // planes copied and not yet consumed
  int turn;       // warp that issues the next copy
  bool dead;      // this thread saw a wait expire: no further waits or copies
};

constexpr int kWarps = kCols / 32;

__device__ __forceinline__ void ring_next(int& slot, uint32_t& par, int nring) {
  if (++slot == nring) { slot = 0; par ^= 1u; }
}

// One FP unit: strip pairs [k0, k0 + kCols) (one per thread, 6 plane
// positions each) over layers [t0, t1).  Layer t reads planes t+2, t+3 of nu and layer t of the degrees
// (planes t+1 and older are already in registers).  The segment [lo, hi) of
// each plane the chunk touches, and the same byte range of the degree layer
// three planes below it, are copied into the next ring slot (cp.async.bulk;
// an mbarrier per slot counts the bytes).  After each pair of layers a block
// barrier frees the slots of the two planes the pair is done with, and they
// are refilled nring planes further on, so the copies run nring-2 planes
// ahead of their use.  The copies go to the warps in turn: a warp that
// issues one starts the next pair a few instructions late, and the pair's
// barrier waits for it, so no warp should carry them all.  A wait that expires sets error
// bit 2 and *abort; the thread then skips all further waits and copies, and
// the kernel drains the copies in flight and returns after the unit.
__device__ __forceinline__ void fp_unit_staged(const Ctx& x, const Lattice& lat, const SlotView& v, bool odd,
                                               int k0, int t0, int t1, float* ring, uint8_t* dring,
                                               uint64_t* full, Ring& rg, int* abort, const float* inv,
                                               int* s_red) {
  const int tid = threadIdx.x, P = lat.P, cap = x.seg_cap, nring = x.nring;
  const int warp = tid >> 5;
  // strip pair h = positions 6h .. 6h+5 (paired layout: one row, even row
  // offsets); threads past the last pair repeat it: they write the same
  // values to the same addresses, and the layer loop needs no branch
  const int s_end = lat.s_begin + lat.n_strips;
  const int h_begin = lat.s_begin >> 1, h_end = (s_end + 1) >> 1;
  const int h = min(h_begin + k0 + tid, h_end - 1);
  const int st = min(max(2 * h + 1, lat.s_begin), s_end - 1);  // a strip of the pair holding its row
  int lo, hi;
  const int b = 6 * h;
  const int32_t* ro = lat.row_off + 4 * lat.strip_row[st - lat.s_begin];
  const int r0 = __ldg(ro), r1 = __ldg(ro + 1), r2 = __ldg(ro + 2), r3 = __ldg(ro + 3);
  {
    const int32_t rr[4] = {r0, r1, r2, r3};
    pair_span(b, rr, &lo, &hi);
  }
  // segment of the chunk: block min / max
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (tid == 0) { s_red[0] = 0x7fffffff; s_red[1] = -0x7fffffff; }
  __syncthreads();
  if ((tid & 31) == 0) { atomicMin(&s_red[0], lo); atomicMax(&s_red[1], hi); }
  __syncthreads();
  // 16-entry alignment: 16-byte aligned copies of both the FP32 and the byte planes
  const int lo_al = s_red[0] & ~15;
  int seg = ((s_red[1] + 15) & ~15) - lo_al;
  if (seg > cap) {  // cannot happen: the host sized the ring for every lattice
    if (tid == 0) atomicOr(x.error, 4);
    seg = cap;
  }
  const float* src = odd ? v.nu0 : v.nu1;
  float* dst = odd ? v.nu1 : v.nu0;
  // copy the next plane (and the degree layer three below it) into its
  // slot: lane 0 of warp rg.turn issues, every thread advances the cursor
  int next_pl = t0 + 1;
  const int last = t1 + 2;
  auto issue = [&]() {
    if (next_pl > last) return;
    if (warp == rg.turn && (tid & 31) == 0 && !rg.dead) {
      const int sl = rg.wslot;
      const int lay = next_pl - 3;
      const bool with_dg = lay >= t0;
      fence_proxy_async_shared();
      mbar_arrive_expect_tx(&full[sl], (unsigned)seg * (with_dg ? 5u : 4u));
      bulk_g2s(ring + (size_t)sl * cap, src + (size_t)next_pl * P + lo_al, (unsigned)seg * 4u, &full[sl]);
      if (with_dg) bulk_g2s(dring + (size_t)sl * cap, v.dg + (size_t)lay * P + lo_al, (unsigned)seg, &full[sl]);
    }
    ++next_pl;
    ++rg.pending;
    if (++rg.wslot == nring) rg.wslot = 0;
    if (++rg.turn == kWarps) rg.turn = 0;
  };
  // consume the next plane: wait for its slot; returns the slot.  After an
  // expired wait the cursor stays on that slot, where the drain starts.
  auto consume = [&]() -> int {
    const int sl = rg.slot;
    if (!rg.dead) {
      if (mbar_wait(&full[sl], rg.par)) {
        ring_next(rg.slot, rg.par, nring);
        --rg.pending;
      } else {
        rg.dead = true; *abort = 1; atomicOr(x.error, 2);
      }
    }
    return sl;
  };
  // shared byte offsets within a slot of this pair's 64-bit-aligned reads:
  // rows r+1, r-1, r, r+2 from position b - 2, row r-2 from b; degrees at b
  const uint32_t ou = 4u * (uint32_t)(b - 2 + r2 - lo_al), od = 4u * (uint32_t)(b - 2 + r1 - lo_al);
  const uint32_t oc = 4u * (uint32_t)(b - 2 - lo_al), oe = 4u * (uint32_t)(b - 2 + r3 - lo_al);
  const uint32_t of = 4u * (uint32_t)(b + r0 - lo_al), og = (uint32_t)(b - lo_al);
  // shared addresses (bytes): slot s of the FP32 ring at ring_s + s * cap4,
  // of the degree ring at dring_s + s * cap
  const uint32_t ring_s = smem_u32(ring), dring_s = smem_u32(dring), inv_s = smem_u32(inv);
  const uint32_t cap4 = 4u * (uint32_t)cap;

  for (int i = 0; i < nring; ++i) issue();
  const int s1 = consume();  // plane t0 + 1
  const int s2 = consume();  // plane t0 + 2
  // layer t-1 values of the pair: U[2], D[2] of each strip, C[0..6]
  float pu[2], pd[2], pcv[7];
  PairRuns A, B;
  {
    PairRuns T;
    const uint32_t p1 = ring_s + (uint32_t)s1 * cap4;
    load_pair_runs(T, p1 + ou, p1 + od, p1 + oc);
    pu[0] = T.u[2]; pu[1] = T.u[5]; pd[0] = T.d[2]; pd[1] = T.d[5];
#pragma unroll
    for (int i = 0; i < 7; ++i) pcv[i] = T.c[i];
    const uint32_t q2 = ring_s + (uint32_t)s2 * cap4;
    load_pair_runs(A, q2 + ou, q2 + od, q2 + oc);
  }
  __syncthreads();  // plane t0 + 1's slot is free
  issue();
  // output plane of layer t (global stores, bypassing L1)
  float* out = dst + (size_t)(t0 + 2) * P + b;
  // layers in pairs: one block barrier frees the two planes the pair is done with
  int t = t0;
  // shared byte address of the slot of plane t + 2
  uint32_t p2 = ring_s + (uint32_t)s2 * cap4;
  for (;;) {
    {
      const int s3 = consume();  // plane t + 3
      const uint32_t p3 = ring_s + (uint32_t)s3 * cap4;
      load_pair_runs(B, p3 + ou, p3 + od, p3 + oc);
      pair_emit(A, B, pu, pd, pcv, p2 + oe, p2 + of, dring_s + (uint32_t)s3 * (uint32_t)cap + og, inv_s, out);
      pu[0] = A.u[2]; pu[1] = A.u[5]; pd[0] = A.d[2]; pd[1] = A.d[5];
#pragma unroll
      for (int i = 0; i < 7; ++i) pcv[i] = A.c[i];
      p2 = p3;
      out += P;
    }
    if (++t >= t1) {
      __syncthreads();
      issue();
      break;
    }
    {
      const int s3 = consume();
      const uint32_t p3 = ring_s + (uint32_t)s3 * cap4;
      load_pair_runs(A, p3 + ou, p3 + od, p3 + oc);
      pair_emit(B, A, pu, pd, pcv, p2 + oe, p2 + of, dring_s + (uint32_t)s3 * (uint32_t)cap + og, inv_s, out);
      pu[0] = B.u[2]; pu[1] = B.u[5]; pd[0] = B.d[2]; pd[1] = B.d[5];
#pragma unroll
      for (int i = 0; i < 7; ++i) pcv[i] = B.c[i];
      p2 = p3;
      out += P;
    }
    __syncthreads();  // planes t + 1 and t + 2 are free
    issue();
    issue();
    if (++t >= t1) break;
  }
}

// kFP = false: a plan without FP32 work (every query PC_BITS_ONLY) -- no
// ring, no FP units, fewer registers and more CTAs per SM for the
// latency-bound bit units.
template <bool kFP>
__global__ void __launch_bounds__(kCols, kFP ? 2 : 4) sweep_kernel(Ctx x) {
  // x.nring slots of x.seg_cap floats (nu planes), then x.nring of x.seg_cap
  // bytes (degrees), then the tick's unit prefix over the slots
  extern __shared__ __align__(128) float ring[];
  uint8_t* dring = reinterpret_cast<uint8_t*>(ring + (size_t)x.nring * x.seg_cap);
  int* s_pre = reinterpret_cast<int*>(reinterpret_cast<char*>(ring) + ring_bytes(x.seg_cap, x.nring));
  __shared__ float inv_deg[16];
  __shared__ uint32_t s_flag;
  __shared__ int s_red[2];
  __shared__ __align__(8) uint64_t bars[kMaxRing];  // one per ring slot
  __shared__ int s_abort;
  const int tid = threadIdx.x;
  if (tid < 16) inv_deg[tid] = tid ? __frcp_rn((float)tid) : 0.f;
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < x.nring; ++i) mbar_init(&bars[i], 1);  // one arrival plus the bytes
    mbar_fence_init();
  }
  // the tick's unit prefix, searched for every unit: staged once per CTA
  for (int s = tid; s <= x.K; s += blockDim.x) s_pre[s] = x.pre[s];
  __syncthreads();
  Ring rg{0, 0u, 0, 0, 0, false};
  const int total = s_pre[x.K];
  // units are taken from a tick-wide counter (double-buffered broadcast: one
  // block barrier per unit).  A CTA asks for its next unit only when it is
  // free: reserving one ahead holds back long units at the end of a tick.
  __shared__ int s_unit[2];
  for (int it = 0;; ++it) {
    if (tid == 0) s_unit[it & 1] = (int)atomicAdd(x.next_unit, 1u);
    __syncthreads();
    const int u = s_unit[it & 1];
    if (u >= total) break;
    // slot: last s with pre[s] <= u (binary search)
    int lo = 0, hi = x.K - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_pre[mid] <= u) lo = mid; else hi = mid - 1;
    }
    const int slot = lo;
    const Ctl c = x.ctl[slot];
    // a slot's units in the order preparation, draw, FP, bits, clean: the
    // occasional long preparation and draw units start early in the tick
    // instead of lengthening its end
    constexpr int kOrder[U_KINDS] = {U_PREP, U_DRAW, U_FP, U_BITS, U_CLEAN};
    // (unrolled: constant indices keep the slot's control block in registers)
    int local = u - s_pre[slot], kind = -1;
#pragma unroll
    for (int i = 0; i < U_KINDS; ++i) {
      const int n = c.units[kOrder[i]];
      if (kind < 0) {
        if (local < n) kind = kOrder[i];
        else local -= n;
      }
    }
    const QDev& Q = x.qs[c.q];
    const Lattice& lat = Q.lat;
    const int A = lat.A, L = lat.L, S = lat.S, P = lat.P;
    const int ccol = (width_of(kind, lat) + unit_width(kind) - 1) / unit_width(kind);
    const int cchunk = local % ccol, rchunk = local / ccol;
    const int a = cchunk * unit_width(kind) + tid;  // column, strip pair or plane position
    const Plan p = make_plan(c.phase, c.m, c.G, c.F, L, lat.TW);
    const SlotView v = view_of(x, slot, lat);

    if (kFP && kind == U_FP) {
      const int t0 = p.lo[U_FP] + rchunk * kRowsFP;
      const int t1 = min(t0 + kRowsFP, p.hi[U_FP]);
      fp_unit_staged(x, lat, v, (c.m & 1) != 0, cchunk * kCols, t0, t1, ring, dring, bars, rg, &s_abort,
                     inv_deg, s_red);
      __syncthreads();
      if (s_abort) {  // a wait expired: let the copies in flight land (bounded), then stop
        if (tid == 0)
          for (; rg.pending > 0; --rg.pending) {
            mbar_wait(&bars[rg.slot], rg.par);
            ring_next(rg.slot, rg.par, x.nring);
          }
        return;
      }
    } else if (kind == U_BITS) {
      // columns a and a + kCols (kBitsCols per thread) and two word rows
      // per iteration: four independent load chains in flight per thread
      const int w0 = p.lo[U_BITS] + rchunk * kRows;
      const int w1 = min(w0 + kRows, p.hi[U_BITS]);
      const bool odd = (c.m & 1) != 0;
      // Rs and occw are only read during a sweep (no unit of this tick writes
      // the rows read here): read-only cache path
      const uint32_t* __restrict__ Rs = odd ? v.R0 : v.R1;
      uint32_t* __restrict__ Rd = odd ? v.R1 : v.R0;
      const uint32_t* __restrict__ occw = v.occw;
      const int endw = (L - 1) >> 5, endb = (L - 1) & 31;
      uint32_t fl = 0;
      int col[kBitsCols], nb[kBitsCols][kLateral];
      uint32_t sh_up[kBitsCols], sh_dn[kBitsCols];
#pragma unroll
      for (int k = 0; k < kBitsCols; ++k) {
        // a thread past the last column takes the sentinel column A: its
        // words are zero and its contacts the sentinel again, so it reads in
        // bounds and writes nothing
        col[k] = a + k * kCols < A ? a + k * kCols : A;
        const int cc = col[k] < A ? col[k] : 0;
        const int sg = lat.sigma[cc];
#pragma unroll
        for (int d = 0; d < kLateral; ++d) nb[k][d] = col[k] < A ? lat.nbr[cc * kLateral + d] : A;
        // the up contacts reach tube t+1 from sigma = 2, the down contacts
        // tube t-1 from sigma = 0: one funnel shift of their ORed words
        sh_up[k] = sg == 2 ? 1u : 0u;
        sh_dn[k] = sg == 0 ? 1u : 0u;
      }
#pragma unroll 2
      for (int tw = w0; tw < w1; ++tw) {
        const uint32_t* r0 = Rs + (size_t)tw * S;  // word tw - 1
        const uint32_t* r1 = r0 + S;               // word tw
        const uint32_t* r2 = r1 + S;               // word tw + 1
#pragma unroll
        for (int k = 0; k < kBitsCols; ++k) {
          const int ak = col[k];
          const uint32_t old = __ldg(r1 + ak);
          // end contacts: tubes t-1 and t+1 of the own column
          uint32_t acc = ((old << 1) | (__ldg(r0 + ak) >> 31)) | ((old >> 1) | (__ldg(r2 + ak) << 31));
          // same-layer contacts (d = 0..5): same tube index
#pragma unroll
          for (int d = 0; d < 6; ++d) acc |= __ldg(r1 + nb[k][d]);
          const uint32_t up = __ldg(r1 + nb[k][6]) | __ldg(r1 + nb[k][7]) | __ldg(r1 + nb[k][8]);
          const uint32_t up_hi = __ldg(r2 + nb[k][6]) | __ldg(r2 + nb[k][7]) | __ldg(r2 + nb[k][8]);
          const uint32_t dn = __ldg(r1 + nb[k][9]) | __ldg(r1 + nb[k][10]) | __ldg(r1 + nb[k][11]);
          const uint32_t dn_lo = __ldg(r0 + nb[k][9]) | __ldg(r0 + nb[k][10]) | __ldg(r0 + nb[k][11]);
          // bit b of the result = contact at tube 32 tw + b (+1 for up, -1 for down)
          acc |= __funnelshift_r(up, up_hi, sh_up[k]) | __funnelshift_l(dn_lo, dn, sh_dn[k]);
          const int wi = (tw + 1) * S + ak;
          const uint32_t nw = old | (acc & __ldg(occw + wi));
          if (ak < A) {
            Rd[wi] = nw;
            if (nw != old) fl |= kGrow;
            if (tw == endw && (((nw & ~old) >> endb) & 1u)) fl |= kEnd;
          }
        }
      }
      fl = __reduce_or_sync(0xffffffffu, fl);
      if (tid == 0) s_flag = 0u;
      __syncthreads();
      if ((tid & 31) == 0 && fl) atomicOr(&s_flag, fl);
      __syncthreads();
      if (tid == 0 && s_flag) atomicOr(&x.ctl[slot].flags, s_flag);
    } else if (kind == U_PREP) {
      // one word row (32 layers, t0 a multiple of 32) of plane position a:
      // degrees counted for 32 tubes at once -- each contact's occupancy
      // word, shifted to the row by the contact's tube offset, added into a
      // 4-bit counter held as four bit planes (at most 14 contacts) -- then
      // written one byte per layer, the nu planes zeroed, and the
      // reached-set word row after this one cleaned
      const int t0 = p.lo[U_PREP] + rchunk * 32;
      const int t1 = min(t0 + 32, p.hi[U_PREP]);
      const int pos = a;
      if (pos < P) {
        const int col = __ldg(lat.pcol + pos);
        const int w = t0 >> 5;
        uint32_t cnt0 = 0u, cnt1 = 0u, cnt2 = 0u, cnt3 = 0u, own = 0u;
        if (col >= 0 && !Q.bits_only) {
          const int sg = lat.sigma[col];
          const uint32_t* o0 = v.occw + (size_t)w * S;  // word w - 1
          const uint32_t* o1 = o0 + S;                  // word w
          const uint32_t* o2 = o1 + S;                  // word w + 1
          auto add = [&](uint32_t x) {  // bit-sliced counter += x
            uint32_t c = cnt0 & x; cnt0 ^= x;
            uint32_t c2 = cnt1 & c; cnt1 ^= c;
            c = cnt2 & c2; cnt2 ^= c2;
            cnt3 ^= c;
          };
          own = o1[col];
          add((own << 1) | (o0[col] >> 31));  // tube t-1
          add((own >> 1) | (o2[col] << 31));  // tube t+1
          const uint32_t sh_up = sg == 2 ? 1u : 0u, sh_dn = sg == 0 ? 1u : 0u;
#pragma unroll
          for (int d = 0; d < kLateral; ++d) {
            const int nb = lat.nbr[col * kLateral + d];
            if (d < 6) add(o1[nb]);
            else if (d < 9) add(__funnelshift_r(o1[nb], o2[nb], sh_up));
            else add(__funnelshift_l(o0[nb], o1[nb], sh_dn));
          }
        }
        for (int t = t0; t < t1; ++t) {
          const int b = t - t0;
          int deg = 0;
          if ((own >> b) & 1u)
            deg = (int)(((cnt0 >> b) & 1u) | (((cnt1 >> b) & 1u) << 1) | (((cnt2 >> b) & 1u) << 2) |
                        (((cnt3 >> b) & 1u) << 3)) + (t == L - 1);
          if (!Q.bits_only) {
            v.dg[(size_t)t * P + pos] = (uint8_t)deg;
            v.nu0[(size_t)(t + 2) * P + pos] = 0.f;
            v.nu1[(size_t)(t + 2) * P + pos] = 0.f;
          }
        }
        if (col >= 0) {  // reached-set word rows cleaned one row ahead
          v.R0[(w + 2) * S + col] = 0u; v.R1[(w + 2) * S + col] = 0u;
          if (w == 0) { v.R0[S + col] = 0u; v.R1[S + col] = 0u; }
        }
      }
    } else if (kind == U_CLEAN) {
      // zero planes 0, 1, L+2, L+3 of nu, pad rows 0 and TW+1 of the bit arrays
      if (a < P) {
        const size_t hi0 = (size_t)(L + 2) * P;
        v.nu0[a] = 0.f; v.nu0[P + a] = 0.f; v.nu0[hi0 + a] = 0.f; v.nu0[hi0 + P + a] = 0.f;
        v.nu1[a] = 0.f; v.nu1[P + a] = 0.f; v.nu1[hi0 + a] = 0.f; v.nu1[hi0 + P + a] = 0.f;
      }
      if (a <= A) {
        const int top = (lat.TW + 1) * S + a;
        v.occw[a] = 0u; v.R0[a] = 0u; v.R1[a] = 0u;
        v.occw[top] = 0u; v.R0[top] = 0u; v.R1[top] = 0u;
      }
      if (cchunk == 0)  // the sentinel column A of every word row
        for (int r = tid; r < lat.TWP; r += kCols) {
          v.occw[r * S + A] = 0u; v.R0[r * S + A] = 0u; v.R1[r * S + A] = 0u;
        }
    } else {  // U_DRAW: one word row of occupancy, 32 tubes per word
      const int tw = p.lo[U_DRAW] + rchunk;
      if (a < A) {
        const long long rel = x.server ? c.item : config_of(Q, c.item - Q.item0);
        uint32_t word = 0;
        if (Q.occ_bits) {
          const uint32_t* cb = Q.occ_bits + (size_t)rel * Q.words_per_cfg;
          for (int b = 0; b < 32; ++b) {
            const int t = tw * 32 + b;
            if (t >= L) break;
            const int64_t i = (int64_t)t * A + a;
            word |= ((cb[i >> 5] >> (i & 31)) & 1u) << b;
          }
        } else {
          const uint32_t cfg = Q.cfg0 + (uint32_t)rel;
          for (int b = 0; b < 32; ++b) {
            const int t = tw * 32 + b;
            if (t >= L) break;
            const int64_t i = (int64_t)t * A + a;
            const u32x4 r = philox4x32_10(u32x4{(uint32_t)(i >> 2), cfg, Q.occ.wl, 0u}, Q.occ.k0, Q.occ.k1);
            const uint32_t w = (i & 3) == 0 ? r.x : (i & 3) == 1 ? r.y : (i & 3) == 2 ? r.z : r.w;
            word |= (uint32_t)((uint64_t)w < Q.occ.T) << b;
          }
        }
        v.occw[(tw + 1) * S + a] = word;
      }
    }
  }
}

// The sweep kernel a plan launches.
inline const void* sweep_fn(const Ctx& x) {
  return x.fp ? (const void*)sweep_kernel<true> : (const void*)sweep_kernel<false>;
}

// Persistent sweep grid: as many CTAs as fit on the device at once (units
// are fetched dynamically, so more CTAs would only add start-up work).
int sweep_grid(const Ctx& x) {
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_fn(x), kCols,
                                                    sweep_smem_bytes(x.seg_cap, x.nring, x.K)) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return nsm * per_sm;
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

// One CTA per slot; the last CTA to finish plans the next tick.
__global__ void __launch_bounds__(kCols) control_kernel(Ctx x) {
  __shared__ float red[32];
  __shared__ int s_n0;
  __shared__ bool s_last;
  const int slot = blockIdx.x, tid = threadIdx.x;
  Ctl c = x.ctl[slot];
  if (c.phase != PH_EMPTY) {
    const QDev& Q = x.qs[c.q];
    const Lattice& lat = Q.lat;
    const int A = lat.A, L = lat.L, S = lat.S;
    const SlotView v = view_of(x, slot, lat);
    const Plan p = make_plan(c.phase, c.m, c.G, c.F, L, lat.TW);
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
      for (int a = tid; a < A; a += blockDim.x) cnt += (int)(v.occw[S + a] & 1u);
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
          const uint32_t b = v.occw[S + a] & 1u;
          v.R0[S + a] = b;
          if (Q.bits_only) continue;
          const int pos = __ldg(lat.ppos + a);
          const int d = v.dg[pos];
          const float val = b ? (d ? __frcp_rn((float)d) : 0.f) * inv : 0.f;
          v.nu0[(size_t)2 * lat.P + pos] = val;
          part += val;
        }
        if (L == 1) {
          mass = Q.bits_only ? 0.f : block_sum_f(part, red);
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
        const float* dst = (c.m & 1) ? v.nu1 : v.nu0;
        float part = 0.f;
        for (int k = Q.bits_only ? lat.P : tid; k < lat.P; k += blockDim.x)
          part += dst[(size_t)(L + 1) * lat.P + k];
        mass = Q.bits_only ? 0.f : block_sum_f(part, red);
        finish = true; verdict = 1; fh = c.m + 1; mstop = c.m + 1;
      } else if (!(f & kGrow)) {
        finish = true; mstop = c.m;
      } else {
        c.m += 1;
      }
    }
    if (tid == 0) {
      if (finish) {
        const long long rel = x.server ? c.item : config_of(Q, c.item - Q.item0);
        Q.out.verdict[rel] = (uint8_t)verdict;
        if (Q.out.first_hit) Q.out.first_hit[rel] = fh;
        if (Q.out.mass) Q.out.mass[rel] = mass;
        if (Q.out.m_stop) Q.out.m_stop[rel] = mstop;
        if (verdict && Q.out.n_perc) atomicAdd(Q.out.n_perc, 1ull);
        atomicAdd(x.n_done, 1ull);
        if (x.server) {
          // the slot stays with its query while it has configurations left
          atomicAdd(&x.qdone[c.q], 1ull);
          const unsigned long long nxt = atomicAdd(&x.qnext[c.q], 1ull);
          const int q = c.q;
          c.item = (long long)nxt; c.m = 0; c.G = 0; c.F = 0; c.flags = 0u;
          for (int k = 0; k < U_KINDS; ++k) c.units[k] = 0;
          if ((long long)nxt < x.qs[q].n_cfg) { c.phase = PH_DRAW0; fill_plan(c, x.qs[q]); }
          else c.phase = PH_EMPTY;
        } else {
          assign(x, c, atomicAdd(x.work, 1ull));
        }
      } else {
        fill_plan(c, Q);
      }
      x.ctl[slot] = c;
    }
  }
  // last block: prefix of the next tick's units, loop condition
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(x.arrive, 1u) == (unsigned)(gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  plan_prefix(x);
  if (tid == 0) {
    *x.arrive = 0u;
    *x.next_unit = 0u;
    const unsigned t = *x.ticks + 1u;
    *x.ticks = t;
    // an error bit (expired wait, failed check) ends the loop at once
    const bool more = *x.n_done < (unsigned long long)x.n_items && *x.error == 0;
    if (x.use_cond) {
      if (more && t >= x.max_ticks) *x.error = 1;
      cudaGraphSetConditional(x.cond, (more && t < x.max_ticks) ? 1u : 0u);
    }
  }
}

}  // namespace

size_t stream_slot_bytes(int W, int L) {
  int P = 0;
  layout_fill(W, &P, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, true);
  return slot_bytes_of((int)n_columns(W), L, P);
}

struct StreamPlan {
  Ctx x;
  char* mem = nullptr;   // one allocation: queries, ctl, prefix, counters, pool
  int grid = 0;
  int* error_dev = nullptr;
};

pc_status stream_plan_create(const StreamQuery* qs, int nq, cudaStream_t st, StreamPlan** out) {
  *out = nullptr;
  long long n_items = 0;
  size_t slot = 0;
  unsigned long long max_steps = 0;
  std::vector<QDev> h(nq);
  for (int i = 0; i < nq; ++i) {
    h[i].lat = stream_view(qs[i].lat); h[i].occ = qs[i].occ; h[i].occ_bits = qs[i].occ_bits;
    h[i].words_per_cfg = qs[i].words_per_cfg; h[i].n_cfg = qs[i].n_cfg; h[i].cfg0 = qs[i].cfg0;
    h[i].out = qs[i].out; h[i].item0 = n_items; h[i].bits_only = qs[i].bits_only; h[i].sel = qs[i].sel;
    n_items += qs[i].n_cfg;
    slot = std::max(slot, slot_bytes_of(qs[i].lat.A, qs[i].lat.L, qs[i].lat.P2));
    max_steps = std::max<unsigned long long>(max_steps, (unsigned long long)qs[i].lat.N + 4);
  }
  size_t free_b = 0, total_b = 0;
  PC_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t budget = free_b / 2;
  long long K = std::min<long long>(n_items, kMaxSlots);
  // PC_STREAM_MAX_SLOTS caps the pool (tests use it to force slot reuse)
  if (const char* cap = std::getenv("PC_STREAM_MAX_SLOTS")) {
    const long long c = std::atoll(cap);
    if (c > 0) K = std::min<long long>(K, c);
  }
  K = std::min<long long>(K, (long long)(budget / (slot + 1)));
  if (n_items > 0 && K < 1) {
    set_error("streamed solver: one configuration's state exceeds half the free device memory");
    return PC_ERR_OOM;
  }
  if (K < 1) K = 1;
  const size_t hdr = a256(sizeof(QDev) * nq) + a256(sizeof(Ctl) * K) + a256(sizeof(int) * (K + 1)) + 256;
  StreamPlan* P = new StreamPlan();
  cudaError_t e = cudaMallocAsync((void**)&P->mem, hdr + (size_t)K * slot + 256, st);
  if (e != cudaSuccess) { delete P; return cuda_fail(e, "stream plan alloc"); }
  char* q = P->mem;
  Ctx& x = P->x;
  x.qs = (const QDev*)q; q += a256(sizeof(QDev) * nq);
  x.nq = nq; x.n_items = n_items; x.K = (int)K;
  x.ctl = (Ctl*)q; q += a256(sizeof(Ctl) * K);
  x.pre = (int*)q; q += a256(sizeof(int) * (K + 1));
  x.work = (unsigned long long*)q;
  x.n_done = x.work + 1;
  x.ticks = (unsigned int*)(x.work + 2);
  x.arrive = x.ticks + 1;
  x.error = (int*)(x.ticks + 2);
  x.next_unit = x.ticks + 3;
  q += 256;
  x.pool = q;
  x.slot_bytes = slot;
  x.use_cond = 0; x.server = 0; x.slot_base = nullptr; x.qnext = nullptr; x.qdone = nullptr;
  x.fp = 0;
  for (int i = 0; i < nq; ++i) x.fp |= qs[i].bits_only ? 0 : 1;
  {
    int cap = 16;
    for (int i = 0; i < nq; ++i) cap = std::max(cap, max_pair_segment(qs[i].lat.W, kCols) + 16);
    x.seg_cap = x.fp ? cap : 0;
    x.nring = x.fp ? ring_depth(cap) : 0;
    const int bytes = sweep_smem_bytes(x.seg_cap, x.nring, x.K);
    cudaError_t ea = cudaFuncSetAttribute(sweep_fn(x), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (ea != cudaSuccess) { cudaFreeAsync(P->mem, st); delete P; return cuda_fail(ea, "sweep smem"); }
  }
  // every configuration needs at most N + 3 ticks; slots run concurrently
  const unsigned long long waves = (unsigned long long)((n_items + K - 1) / K);
  const unsigned long long bound = waves * (max_steps + 4) + 64;
  x.max_ticks = (unsigned int)std::min<unsigned long long>(bound, 0xffffff00ull);
  P->error_dev = x.error;
  for (int b = 0; b < nq && e == cudaSuccess; b += kQChunk) {
    QChunk ch;
    ch.base = b;
    ch.n = std::min(kQChunk, nq - b);
    for (int i = 0; i < ch.n; ++i) ch.q[i] = h[b + i];
    upload_queries_kernel<<<1, kQChunk, 0, st>>>((QDev*)x.qs, ch);
    e = cudaGetLastError();
  }
  // pool must start zeroed: padding rows / sentinel columns are never written
  if (e == cudaSuccess) e = cudaMemsetAsync(x.pool, 0, (size_t)K * slot, st);
  if (e != cudaSuccess) { cudaFreeAsync(P->mem, st); delete P; return cuda_fail(e, "stream plan init"); }
  P->grid = sweep_grid(x);
  *out = P;
  return PC_OK;
}

// Adds [init kernel -> WHILE(sweep, control)] to graph g after deps.
pc_status stream_plan_add(StreamPlan* P, cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps,
                          cudaGraphNode_t* last) {
  Ctx& x = P->x;
  PC_CUDA(cudaGraphConditionalHandleCreate(&x.cond, g, 1, cudaGraphCondAssignDefault));
  x.use_cond = 1;
  void* args[] = {&x};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)stream_init_kernel;
  kp.gridDim = dim3(1); kp.blockDim = dim3(1024); kp.sharedMemBytes = 0; kp.kernelParams = args;
  cudaGraphNode_t n_init;
  PC_CUDA(cudaGraphAddKernelNode(&n_init, g, deps, ndeps, &kp));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = x.cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t n_while;
  PC_CUDA(cudaGraphAddNode(&n_while, g, &n_init, nullptr, 1, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaKernelNodeParams sp = {};
  sp.func = const_cast<void*>(sweep_fn(x));
  sp.gridDim = dim3(P->grid); sp.blockDim = dim3(kCols); sp.kernelParams = args;
  sp.sharedMemBytes = (unsigned)sweep_smem_bytes(x.seg_cap, x.nring, x.K);
  cudaGraphNode_t n_sweep, n_ctl;
  PC_CUDA(cudaGraphAddKernelNode(&n_sweep, body, nullptr, 0, &sp));
  cudaKernelNodeParams cpk = {};
  cpk.func = (void*)control_kernel;
  cpk.gridDim = dim3(x.K); cpk.blockDim = dim3(kCols); cpk.kernelParams = args;
  PC_CUDA(cudaGraphAddKernelNode(&n_ctl, body, &n_sweep, 1, &cpk));
  *last = n_while;
  return PC_OK;
}

int* stream_plan_error(StreamPlan* P) { return P->error_dev; }

void stream_plan_release(StreamPlan* P, cudaStream_t st) {
  if (!P) return;
  if (P->mem) cudaFreeAsync(P->mem, st);
  delete P;
}

// ---------------------------------------------------------------------------
// Server engine: the same ticks, with slots bound to queries by the host
// (continuous batching).  The host uploads query entries, binds free slots to
// admitted queries, runs chunks of ticks and reads back slot phases and
// per-query completion counts between chunks.
// ---------------------------------------------------------------------------
namespace {

constexpr int kBindChunk = 64;
struct BindList {
  int n;
  int slot[kBindChunk];
  int query[kBindChunk];
  char* base[kBindChunk];
};

__global__ void __launch_bounds__(1024) server_bind_kernel(Ctx x, BindList b) {
  if ((int)threadIdx.x < b.n) {
    const int s = b.slot[threadIdx.x], q = b.query[threadIdx.x];
    x.slot_base[s] = b.base[threadIdx.x];
    Ctl c;
    const unsigned long long nxt = atomicAdd(&x.qnext[q], 1ull);
    c.item = (long long)nxt; c.q = q; c.m = 0; c.G = 0; c.F = 0; c.flags = 0u;
    for (int k = 0; k < U_KINDS; ++k) c.units[k] = 0;
    if ((long long)nxt < x.qs[q].n_cfg) { c.phase = PH_DRAW0; fill_plan(c, x.qs[q]); }
    else c.phase = PH_EMPTY;
    x.ctl[s] = c;
  }
  __threadfence();
  __syncthreads();
  plan_prefix(x);
}

__global__ void server_reset_kernel(Ctx x) {
  for (int s = threadIdx.x; s < x.K; s += blockDim.x) {
    Ctl c;
    c.item = 0; c.q = 0; c.phase = PH_EMPTY; c.m = 0; c.G = 0; c.F = 0; c.flags = 0u;
    for (int k = 0; k < U_KINDS; ++k) c.units[k] = 0;
    x.ctl[s] = c;
    x.pre[s] = 0;
  }
  if (threadIdx.x == 0) { x.pre[x.K] = 0; *x.arrive = 0u; *x.next_unit = 0u; *x.ticks = 0u; *x.n_done = 0ull; }
}

__global__ void server_status_kernel(Ctx x, int* phases) {
  for (int s = threadIdx.x; s < x.K; s += blockDim.x) phases[s] = x.ctl[s].phase;
}

}  // namespace

struct ServerEngine {
  Ctx x;
  char* mem = nullptr;
  int* d_phase = nullptr;
  int* h_phase[2] = {};                 // pinned [K], one per status buffer
  unsigned long long* h_qdone[2] = {};  // pinned [nq]
  cudaGraphExec_t chunk = nullptr;
  int max_queries = 0;
};

pc_status server_engine_create(int max_slots, int max_queries, int ticks_per_chunk, int max_W,
                               cudaStream_t st, ServerEngine** out) {
  *out = nullptr;
  ServerEngine* E = new ServerEngine();
  Ctx& x = E->x;
  const int K = std::max(1, std::min(max_slots, kMaxSlots));
  const int nq = std::max(1, max_queries);
  const size_t bytes = a256(sizeof(QDev) * nq) + a256(sizeof(Ctl) * K) + a256(sizeof(int) * (K + 1)) +
                       a256(sizeof(char*) * K) + 2 * a256(sizeof(unsigned long long) * nq) +
                       a256(sizeof(int) * K) + 256;
  cudaError_t e = cudaMalloc((void**)&E->mem, bytes);
  if (e != cudaSuccess) { delete E; return cuda_fail(e, "server engine alloc"); }
  char* q = E->mem;
  x = Ctx{};
  x.qs = (const QDev*)q; q += a256(sizeof(QDev) * nq);
  x.nq = nq; x.n_items = 0; x.K = K;
  x.ctl = (Ctl*)q; q += a256(sizeof(Ctl) * K);
  x.pre = (int*)q; q += a256(sizeof(int) * (K + 1));
  x.slot_base = (char**)q; q += a256(sizeof(char*) * K);
  x.qnext = (unsigned long long*)q; q += a256(sizeof(unsigned long long) * nq);
  x.qdone = (unsigned long long*)q; q += a256(sizeof(unsigned long long) * nq);
  E->d_phase = (int*)q; q += a256(sizeof(int) * K);
  x.work = (unsigned long long*)q;
  x.n_done = x.work + 1;
  x.ticks = (unsigned int*)(x.work + 2);
  x.arrive = x.ticks + 1;
  x.error = (int*)(x.ticks + 2);
  x.next_unit = x.ticks + 3;
  x.pool = nullptr; x.slot_bytes = 0; x.max_ticks = 0xffffffffu;
  x.use_cond = 0; x.server = 1; x.fp = 1;  // served queries may run the FP32 recursion
  x.seg_cap = max_pair_segment(max_W, kCols) + 16;  // any lattice the server accepts
  x.nring = ring_depth(x.seg_cap);
  E->max_queries = nq;
  pc_status rc = PC_OK;
  do {
    if ((e = cudaMemsetAsync(E->mem, 0, bytes, st)) != cudaSuccess) { rc = cuda_fail(e, "server memset"); break; }
    server_reset_kernel<<<1, 1024, 0, st>>>(x);
    if ((e = cudaGetLastError()) != cudaSuccess) { rc = cuda_fail(e, "server reset"); break; }
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaMallocHost((void**)&E->h_phase[b], sizeof(int) * K);
      if (e == cudaSuccess) e = cudaMallocHost((void**)&E->h_qdone[b], sizeof(unsigned long long) * nq);
    }
    if (e != cudaSuccess) { rc = cuda_fail(e, "pinned"); break; }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if ((e = cudaFuncSetAttribute(sweep_fn(x), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  sweep_smem_bytes(x.seg_cap, x.nring, x.K))) != cudaSuccess) {
      rc = cuda_fail(e, "sweep smem"); break;
    }
    cudaGraph_t g;
    if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) { rc = cuda_fail(e, "graph"); break; }
    void* args[] = {&x};
    cudaGraphNode_t prev = nullptr;
    for (int t = 0; t < std::max(1, ticks_per_chunk) && rc == PC_OK; ++t) {
      cudaKernelNodeParams sp = {};
      sp.func = const_cast<void*>(sweep_fn(x)); sp.gridDim = dim3(sweep_grid(x)); sp.blockDim = dim3(kCols);
      sp.kernelParams = args;
      sp.sharedMemBytes = (unsigned)sweep_smem_bytes(x.seg_cap, x.nring, x.K);
      cudaGraphNode_t ns, nc;
      if ((e = cudaGraphAddKernelNode(&ns, g, prev ? &prev : nullptr, prev ? 1 : 0, &sp)) != cudaSuccess) { rc = cuda_fail(e, "node"); break; }
      cudaKernelNodeParams cp = {};
      cp.func = (void*)control_kernel; cp.gridDim = dim3(K); cp.blockDim = dim3(kCols);
      cp.kernelParams = args;
      if ((e = cudaGraphAddKernelNode(&nc, g, &ns, 1, &cp)) != cudaSuccess) { rc = cuda_fail(e, "node"); break; }
      prev = nc;
    }
    if (rc == PC_OK && (e = cudaGraphInstantiate(&E->chunk, g, 0)) != cudaSuccess) rc = cuda_fail(e, "instantiate");
    cudaGraphDestroy(g);
    if (rc == PC_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) rc = cuda_fail(e, "server init sync");
  } while (0);
  if (rc) { server_engine_destroy(E); return rc; }
  *out = E;
  return PC_OK;
}

void server_engine_destroy(ServerEngine* E) {
  if (!E) return;
  if (E->chunk) cudaGraphExecDestroy(E->chunk);
  for (int b = 0; b < 2; ++b) {
    if (E->h_phase[b]) cudaFreeHost(E->h_phase[b]);
    if (E->h_qdone[b]) cudaFreeHost(E->h_qdone[b]);
  }
  if (E->mem) cudaFree(E->mem);
  delete E;
}

int server_engine_slots(const ServerEngine* E) { return E->x.K; }

pc_status server_engine_set_query(ServerEngine* E, int qi, const StreamQuery& sq, cudaStream_t st) {
  if (qi < 0 || qi >= E->max_queries) { set_error("server: query index out of range"); return PC_ERR_ARG; }
  QChunk ch;
  ch.base = qi; ch.n = 1;
  QDev& d = ch.q[0];
  d.lat = stream_view(sq.lat); d.occ = sq.occ; d.occ_bits = sq.occ_bits; d.words_per_cfg = sq.words_per_cfg;
  d.n_cfg = sq.n_cfg; d.cfg0 = sq.cfg0; d.out = sq.out; d.item0 = 0; d.bits_only = sq.bits_only; d.sel = nullptr;
  upload_queries_kernel<<<1, kQChunk, 0, st>>>((QDev*)E->x.qs, ch);
  PC_CUDA(cudaGetLastError());
  PC_CUDA(cudaMemsetAsync(E->x.qnext + qi, 0, sizeof(unsigned long long), st));
  PC_CUDA(cudaMemsetAsync(E->x.qdone + qi, 0, sizeof(unsigned long long), st));
  return PC_OK;
}

pc_status server_engine_bind(ServerEngine* E, const int* slots, const int* queries, char* const* bases,
                             int n, cudaStream_t st) {
  for (int b = 0; b < n; b += kBindChunk) {
    BindList bl;
    bl.n = std::min(kBindChunk, n - b);
    for (int i = 0; i < bl.n; ++i) { bl.slot[i] = slots[b + i]; bl.query[i] = queries[b + i]; bl.base[i] = bases[b + i]; }
    server_bind_kernel<<<1, 1024, 0, st>>>(E->x, bl);
    PC_CUDA(cudaGetLastError());
  }
  return PC_OK;
}

pc_status server_engine_run_chunk(ServerEngine* E, cudaStream_t st) {
  PC_CUDA(cudaGraphLaunch(E->chunk, st));
  return PC_OK;
}

// Enqueue the copy of slot phases and per-query completion counts to pinned
// host memory; valid after st reaches this point.
const int* server_engine_phase_buffer(const ServerEngine* E, int buf) { return E->h_phase[buf]; }
const unsigned long long* server_engine_qdone_buffer(const ServerEngine* E, int buf) { return E->h_qdone[buf]; }

pc_status server_engine_status(ServerEngine* E, cudaStream_t st, int buf, const int** phases,
                               const unsigned long long** qdone) {
  server_status_kernel<<<1, 1024, 0, st>>>(E->x, E->d_phase);
  PC_CUDA(cudaGetLastError());
  PC_CUDA(cudaMemcpyAsync(E->h_phase[buf], E->d_phase, sizeof(int) * E->x.K, cudaMemcpyDeviceToHost, st));
  PC_CUDA(cudaMemcpyAsync(E->h_qdone[buf], E->x.qdone, sizeof(unsigned long long) * E->max_queries,
                          cudaMemcpyDeviceToHost, st));
  *phases = E->h_phase[buf];
  *qdone = E->h_qdone[buf];
  return PC_OK;
}

// Single-query convenience used by pc_inspect: build, run, release (stream
// ordered; no host synchronisation).
namespace {
// configurations whose verdict is 1, in any order (each configuration's
// solve does not depend on its slot)
__global__ void select_percolating_kernel(const uint8_t* verdict, int64_t n, int64_t* sel,
                                          unsigned long long* count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (verdict[i]) sel[atomicAdd(count, 1ull)] = i;
}
}  // namespace

pc_status run_stream_verdict_first(const StreamJob& job, cudaStream_t st) {
  if (job.n_cfg <= 0) return PC_OK;
  // 1. the exact reached set decides every configuration (mass written 0)
  StreamJob b = job;
  b.bits_only = 1;
  pc_status rc = run_stream(b, st);
  if (rc) return rc;
  // 2. the FP32 recursion on the percolating configurations only: the same
  // steps as the single pass, so every output equals it to the bit
  char* mem = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&mem, 256 + sizeof(int64_t) * (size_t)job.n_cfg, st);
  if (e != cudaSuccess) return cuda_fail(e, "verdict-first selection");
  unsigned long long* cnt = (unsigned long long*)mem;
  int64_t* sel = (int64_t*)(mem + 256);
  unsigned long long n_sel = 0;
  e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) {
    const int grid = (int)std::min<int64_t>((job.n_cfg + 255) / 256, 1024);
    select_percolating_kernel<<<grid, 256, 0, st>>>(job.out.verdict, job.n_cfg, sel, cnt);
    e = cudaGetLastError();
  }
  int err1 = 0;  // the verdict pass's error flag: the FP32 pass rewrites error_out
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n_sel, cnt, sizeof(n_sel), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && job.error_out)
    e = cudaMemcpyAsync(&err1, job.error_out, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) rc = cuda_fail(e, "verdict-first selection");
  else if (err1) { set_error("verdict pass: a device bound was reached"); rc = (err1 & 2) ? PC_ERR_TIMEOUT : PC_ERR_INTERNAL; }
  if (rc == PC_OK && n_sel > 0) {
    StreamJob f = job;
    f.bits_only = 0;
    f.sel = sel;
    f.n_cfg = (int64_t)n_sel;
    f.out.n_perc = nullptr;  // counted by the first pass
    rc = run_stream(f, st);
  }
  cudaFreeAsync(mem, st);
  return rc;
}

pc_status run_stream(const StreamJob& job, cudaStream_t st) {
  if (job.n_cfg <= 0) return PC_OK;
  if (job.bits_only) {  // verdict only: 32 steps per visit of a slab where a cluster holds the lattice
    bool handled = false;
    const pc_status rb = run_blocked(job, st, &handled);
    if (handled || rb != PC_OK) return rb;
  }
  StreamQuery q;
  q.lat = job.lat; q.occ = job.occ; q.occ_bits = job.occ_bits; q.words_per_cfg = job.words_per_cfg;
  q.n_cfg = job.n_cfg; q.cfg0 = job.cfg0; q.out = job.out; q.bits_only = job.bits_only; q.sel = job.sel;
  StreamPlan* P = nullptr;
  pc_status rc = stream_plan_create(&q, 1, st, &P);
  if (rc) return rc;
  if (std::getenv("PC_STREAM_HOST_LOOP")) {
    // profiling aid: the same ticks launched from a host loop (profilers do
    // not look inside graphs with conditional nodes)
    Ctx& x = P->x;
    stream_init_kernel<<<1, 1024, 0, st>>>(x);
    unsigned long long done = 0;
    for (int chunk = 0; rc == PC_OK && done < (unsigned long long)x.n_items; ++chunk) {
      for (int i = 0; i < 32; ++i) {
        if (x.fp) sweep_kernel<true><<<P->grid, kCols, sweep_smem_bytes(x.seg_cap, x.nring, x.K), st>>>(x);
        else sweep_kernel<false><<<P->grid, kCols, sweep_smem_bytes(x.seg_cap, x.nring, x.K), st>>>(x);
        control_kernel<<<x.K, kCols, 0, st>>>(x);
      }
      int err = 0;
      cudaError_t e = cudaMemcpyAsync(&done, x.n_done, 8, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&err, x.error, sizeof(int), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = cuda_fail(e, "host loop");
      else if (err) { set_error("streamed solver: device error flag set"); rc = (err & 2) ? PC_ERR_TIMEOUT : PC_ERR_INTERNAL; }
      if ((unsigned long long)chunk * 32 > x.max_ticks) { set_error("streamed solver did not converge"); rc = PC_ERR_INTERNAL; }
    }
    stream_plan_release(P, st);
    return rc;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  do {
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) { rc = cuda_fail(e, "graph create"); break; }
    cudaGraphNode_t last;
    if ((rc = stream_plan_add(P, g, nullptr, 0, &last))) break;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) { rc = cuda_fail(e, "graph instantiate"); break; }
    e = cudaGraphLaunch(ex, st);
    if (e != cudaSuccess) { rc = cuda_fail(e, "graph launch"); break; }
    if (job.error_out) {
      e = cudaMemcpyAsync(job.error_out, P->error_dev, sizeof(int), cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) { rc = cuda_fail(e, "error copy"); break; }
    }
  } while (0);
  if (ex) cudaGraphExecDestroy(ex);  // an in-flight executable is freed on completion
  if (g) cudaGraphDestroy(g);
  stream_plan_release(P, st);
  return rc;
}

}  // namespace pc

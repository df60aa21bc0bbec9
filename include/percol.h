/*
 * percol.h -- C ABI of libpercol, a GB300 (sm_103a) implementation of the
 * Markov-chain percolation inspection of F. Xu, Z. Xu and B. I. Yakobson,
 * "Site-Percolation Threshold of Carbon Nanotube Fibers -- Fast Inspection of
 * Percolation with Markov Stochastic Theory" (arXiv:1401.2130).
 *
 * The method (Sec. II.B, Eqs. (1)-(4), Appendix Eq. (A.3)): for one random
 * configuration of the modified-FCC fibre lattice (Sec. II.A), a random walk
 * over metallic sites with P_ij = 1/deg(i) (Eq. (2)) is started from the
 * metallic sites of one fibre end; repeated sparse matrix-vector products
 * propagate its probability mass until the first step m at which mass reaches
 * the detector site joined to every metallic site of the other end (the
 * configuration percolates; m - 1 is the length of the shortest spanning
 * path), or until the set of reached sites stops growing (it does not).
 * Pi(p) is the fraction of percolating configurations (Sec. III).
 *
 * Geometry (Sec. II.A): columns (q, r) of a hexagon of radius W in axial
 * coordinates, max(|q|, |r|, |q + r|) <= W, A = 3W(W+1)+1 columns, L tubes
 * per column, N = A*L sites.  Site id i = t*A + a, a = column rank in
 * row-major order (r = -W..W, q ascending), t = 0..L-1 along the fibre.
 * Each site has 12 side contacts (the FCC nearest neighbours) and 2 end
 * contacts (same column, t +- 1).  Mass starts uniformly on the metallic
 * sites of t = 0; the detector is joined to the metallic sites of t = L-1.
 *
 * Occupancy (Sec. II.A, Bernoulli(p) per site) comes from Philox4x32-10
 * (Salmon et al., SC'11) with key = (seed & 0xffffffff, seed >> 32),
 * counter = (i >> 2, config_index, W | (L << 8), 0); site i is metallic iff
 * output word (i & 3) < floor(p * 2^32).  Bit-packed occupancy stores site i
 * in bit (i & 31) of 32-bit word (i >> 5) of its configuration.
 *
 * Conventions for every call:
 *  - Returns PC_OK (0) or a negative pc_status; pc_last_error() then holds a
 *    thread-local message.  No call aborts the process.
 *  - The caller owns every buffer it passes.  The library owns only its own
 *    device scratch (stream-ordered, released before the call returns for
 *    host outputs, or in stream order for device outputs) and a per-device
 *    cache of lattice tables released by pc_shutdown().
 *  - cuda_stream is a cudaStream_t or NULL (legacy default stream).  Work is
 *    enqueued on it; with host outputs the call synchronises that stream
 *    before returning, with PC_OUT_DEVICE it returns without synchronising.
 *  - Results do not depend on batching, stream or placement: the generator
 *    is counter based and all reductions that decide results are integer.
 *  - Argument rules: 0 <= W <= 255, 1 <= L < 2^24, 0 <= p <= 1 (not NaN),
 *    n_configs >= 0, 0 <= config_begin, config_begin + n_configs <= 2^32.
 */
#ifndef PERCOL_H
#define PERCOL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pc_status;

#define PC_OK 0
#define PC_ERR_ARG (-1)        /* invalid argument */
#define PC_ERR_OOM (-2)        /* device memory or footprint budget exceeded */
#define PC_ERR_CUDA (-3)       /* a CUDA runtime call failed */
#define PC_ERR_TIMEOUT (-4)    /* a bounded wait expired */
#define PC_ERR_BUSY (-5)       /* result not ready yet (server poll) */
#define PC_ERR_CANCELLED (-6)  /* query cancelled or server shut down */
#define PC_ERR_INTERNAL (-7)   /* an internal consistency check failed */

/* flags */
#define PC_OUT_DEVICE 0x1      /* per-configuration outputs and n_percolating
                                  are device pointers; Pi must be NULL */
#define PC_MODE_RESIDENT 0x10  /* force the shared-memory resident solver */
#define PC_MODE_STREAM 0x20    /* force the streamed (global memory) solver */
#define PC_BITS_ONLY 0x40      /* verdicts only: propagate the exact reached set
                                  alone and skip the FP32 recursion.  The
                                  method needs only whether the detector
                                  probability is zero (Sec. II.B), which the
                                  reached set decides exactly; verdicts,
                                  first_hit, m_stop and n_percolating equal the
                                  full inspection's, mass is written 0 */
#define PC_VERDICT_FIRST 0x80  /* the same outputs as the full inspection, to
                                  the bit, with less work: only configurations
                                  that percolate have a non-zero mass (the
                                  detector probability is exactly 0 otherwise,
                                  Sec. II.B), so the reached set decides every
                                  configuration first and the FP32 recursion
                                  then runs, for exactly first_hit - 1 steps,
                                  on the percolating ones only.  In pc_inspect
                                  and pc_inspect_occupancy both solvers apply
                                  it; on the streamed path the call waits for
                                  the verdicts before it starts the FP32
                                  solves (it synchronises cuda_stream even with
                                  PC_OUT_DEVICE).  pc_batch_run's streamed
                                  queries run their single pass.  Ignored with
                                  PC_BITS_ONLY */

/*
 * Lattice size (Sec. II.A): n_columns = A = 3W(W+1)+1, n_sites = A*L.
 * Either pointer may be NULL.  Errors: PC_ERR_ARG.
 */
pc_status pc_lattice_info(int32_t W, int32_t L, int64_t* n_columns, int64_t* n_sites);

/*
 * Draw the occupancy of configurations config_begin .. +n_configs-1
 * (Sec. II.A) into occ_bits, a DEVICE buffer of n_configs * ceil(N/32)
 * uint32 words, configuration-major, bit-packed in site order.  Asynchronous
 * on cuda_stream.  Errors: PC_ERR_ARG, PC_ERR_CUDA.
 */
pc_status pc_occupancy(int32_t W, int32_t L, double p, uint64_t seed,
                       int64_t config_begin, int64_t n_configs,
                       uint32_t* occ_bits, void* cuda_stream);

/*
 * Fixed-count occupancy (Sec. II.A: a random permutation of the N sites puts
 * exactly n_metallic = Np of them metallic), in the layout of pc_occupancy.
 * Site i carries the key (u_i << 32) | i, u_i its 32-bit word of the
 * Bernoulli stream above; the Np sites with the smallest keys are metallic (a
 * uniformly random Np-subset; it equals the Bernoulli configuration at p
 * whenever Np is that configuration's metallic count).  Inspect the result
 * with pc_inspect_occupancy.  Synchronises cuda_stream (a convergence check).
 * Errors: PC_ERR_ARG (n_metallic outside [0, N]), PC_ERR_CUDA,
 * PC_ERR_INTERNAL.
 */
pc_status pc_occupancy_fixed(int32_t W, int32_t L, int64_t n_metallic, uint64_t seed,
                             int64_t config_begin, int64_t n_configs,
                             uint32_t* occ_bits, void* cuda_stream);

/*
 * Inspect configurations config_begin .. +n_configs-1 at probability p
 * (Sec. II.B; Pi(p) of Sec. III).  Per-configuration outputs, each
 * [n_configs] and each optional except verdicts:
 *   verdicts  : 1 if the configuration percolates, else 0
 *   first_hit : first step m with non-zero detector probability (Eq. (3));
 *               first_hit - 1 = shortest spanning path length; -1 if none
 *   mass      : FP32 detector probability at first_hit (the first-passage
 *               probability averaged over the start sites); 0 if none
 *   m_stop    : steps taken: first_hit if percolating, else the first step
 *               whose reached set did not grow; 0 if no start site is metallic
 * n_percolating (int64) and Pi (= n_percolating / n_configs) are optional.
 * Outputs are host pointers unless flags has PC_OUT_DEVICE.  flags may also
 * hold one of PC_MODE_RESIDENT / PC_MODE_STREAM, PC_BITS_ONLY and
 * PC_VERDICT_FIRST; any other bit is PC_ERR_ARG.
 * Errors: PC_ERR_ARG, PC_ERR_OOM, PC_ERR_CUDA, PC_ERR_INTERNAL, and
 * PC_ERR_TIMEOUT if a bounded device wait of the streamed solver expires
 * (host outputs only: with PC_OUT_DEVICE the call returns before the device
 * work ends, except with PC_VERDICT_FIRST on the streamed path).
 * Solvers: the resident one where a configuration's state fits one CTA's
 * shared memory, else the streamed one; with PC_BITS_ONLY the streamed path
 * runs 32 steps per visit of a slab where one thread-block cluster holds the
 * cross-section (pc_bits_blocked_shape).
 */
pc_status pc_inspect(int32_t W, int32_t L, double p, uint64_t seed,
                     int64_t config_begin, int64_t n_configs,
                     uint8_t* verdicts, int32_t* first_hit, float* mass,
                     int32_t* m_stop, int64_t* n_percolating, double* Pi,
                     int32_t flags, void* cuda_stream);

/*
 * As pc_inspect, for caller-given occupancies: occ_bits is a DEVICE buffer of
 * n_configs * ceil(N/32) uint32 words in the layout pc_occupancy writes.
 */
pc_status pc_inspect_occupancy(int32_t W, int32_t L, const uint32_t* occ_bits,
                               int64_t n_configs, uint8_t* verdicts,
                               int32_t* first_hit, float* mass, int32_t* m_stop,
                               int64_t* n_percolating, double* Pi,
                               int32_t flags, void* cuda_stream);

/*
 * One query of a batch: configurations config_begin .. +n_configs-1 of the
 * lattice (W, L) at probability p with the stream of seed.  The output
 * pointers are optional; they are device pointers if the batch flags have
 * PC_OUT_DEVICE, else host pointers.  n_percolating receives the count.
 */
typedef struct pc_query {
  int32_t W, L;
  double p;
  uint64_t seed;
  int64_t config_begin, n_configs;
  uint8_t* verdicts;        /* [n_configs] */
  int32_t* first_hit;       /* [n_configs] */
  float* mass;              /* [n_configs] */
  int32_t* m_stop;          /* [n_configs] */
  int64_t* n_percolating;   /* [1] */
} pc_query;

/* Host-side summary of one query of a batch. */
typedef struct pc_result {
  int64_t n_percolating;
  double Pi;
  int32_t solver;           /* 0 = shared-memory resident, 1 = streamed,
                               2 = verdict-only with temporal blocking */
  int32_t threads;          /* CTA size the resident solver ran with */
} pc_result;

/*
 * Inspect many queries of mixed lattice sizes in one GPU submission (the
 * batching of a finite-size-scaling sweep, Sec. III): the queries whose
 * configuration state fits one CTA's shared memory run the resident solver
 * in at most three persistent launches, one per shared-memory class (up to
 * a quarter, a half, or all of an SM's shared memory), each taking the
 * configurations of its queries from one list ordered by decreasing lattice
 * size; every other query shares one pool of streamed-solver slots that
 * refill as configurations finish, largest lattices first.  The whole batch
 * is one CUDA graph, built on the first call and replayed when the same
 * batch (same queries and output pointers) is submitted again.  The
 * resident CTA size of each (W, L, p bin of width 0.025) is picked by timing
 * candidates on first use (autotuner; choices kept in memory and in the JSON
 * file named by the environment variable PC_TUNE_FILE, if set); a launch
 * runs with the size tuned for its heaviest query (sites x configurations),
 * reported in pc_result.threads.
 * out: [n_queries] host summaries, or NULL.  Unless flags has PC_ASYNC the
 * call synchronises cuda_stream and fills out; with PC_ASYNC (requires
 * PC_OUT_DEVICE and out == NULL) it returns after enqueueing.  PC_BITS_ONLY
 * and PC_VERDICT_FIRST apply to every query of the batch; any other flag bit
 * is PC_ERR_ARG.  With PC_BITS_ONLY and without PC_ASYNC, a streamed query
 * whose cross-section one thread-block cluster holds (pc_bits_blocked_shape)
 * runs on the verdict-only solver with temporal blocking, on cuda_stream
 * after the batch's graph (solver 2 in out).
 * Results equal those of pc_inspect on each query.
 * Threads: calls from several host threads are safe.  A cached batch is
 * reference counted, so evicting it (or pc_shutdown) never frees one that a
 * running call uses.  Replays of the same batch are serialised: each waits,
 * on its own stream, for the previous replay (of any stream, PC_ASYNC
 * included) to finish, because they share counters and the output buffers
 * named in the queries.  A PC_ASYNC batch's outputs are therefore rewritten
 * by the next submission of the same batch once that one runs.
 * Errors: PC_ERR_ARG, PC_ERR_OOM, PC_ERR_CUDA, PC_ERR_INTERNAL.
 */
#define PC_ASYNC 0x2
pc_status pc_batch_run(const pc_query* queries, int64_t n_queries, pc_result* out,
                       int32_t flags, void* cuda_stream);

/*
 * Serving: a continuous-batching request loop on one device (the current
 * device at pc_server_create).  Queries are admitted in arrival order as soon
 * as their HBM footprint -- output buffers, plus the streamed solver's state
 * for max(1, min(slots free, max_slots_per_query)) configurations when the
 * lattice exceeds shared memory -- fits the server's device arena of
 * hbm_budget_bytes.  Admitted queries run concurrently on the device:
 * resident-size queries as persistent kernels on side streams, the others in
 * the streamed solver's slots, which refill on the device while the query
 * has configurations left.  New arrivals are admitted between chunks of
 * ticks_per_poll device ticks.  Lattice state and occupancy counters stay on
 * the device.  Each query's results equal pc_inspect's on the same query.
 */
typedef struct pc_server pc_server;

typedef struct pc_server_opts {
  uint64_t hbm_budget_bytes;   /* device arena (default 8 GiB) */
  int32_t max_slots;           /* streamed-solver slots, 1..4096 (default 256) */
  int32_t max_slots_per_query; /* cap per query (default 64) */
  int32_t ticks_per_poll;      /* device ticks between admissions (default 8) */
  int64_t max_pending;         /* queue bound; submit returns PC_ERR_BUSY beyond */
  int32_t max_W;               /* widest lattice solved in HBM slots, 0..255 (0 = 255):
                                  sizes the sweep's shared-memory staging; a
                                  narrower bound lets more planes be in flight */
} pc_server_opts;

typedef struct pc_server_stats {
  int64_t submitted, completed, configs_completed;
  double p50_ms, p99_ms, mean_ms;  /* submit-to-completion latency */
  double configs_per_s;            /* completed configurations / (last completion - first submission) */
} pc_server_stats;

/* opts may be NULL (defaults).  Errors: PC_ERR_ARG, PC_ERR_OOM, PC_ERR_CUDA. */
pc_status pc_server_create(const pc_server_opts* opts, pc_server** out);

/*
 * Enqueue a query (n_configs >= 1).  Its output pointers are HOST pointers
 * (optional), filled when the query completes.  Returns a ticket at once.
 * Errors: PC_ERR_ARG (also: a lattice that needs HBM slots and is wider
 * than the server's max_W), PC_ERR_OOM (footprint larger than the whole budget),
 * PC_ERR_BUSY (queue full), PC_ERR_CANCELLED (server shutting down).
 */
pc_status pc_server_submit(pc_server* s, const pc_query* q, uint64_t* ticket);

/*
 * Wait up to timeout_ns (0: do not wait) for a ticket.  PC_OK fills out and
 * retires the ticket; PC_ERR_BUSY if it is not finished yet (poll again);
 * PC_ERR_CANCELLED if it was cancelled; PC_ERR_ARG for an unknown ticket.
 * A query whose work failed returns that failure (e.g. PC_ERR_CUDA,
 * PC_ERR_TIMEOUT, PC_ERR_INTERNAL) and retires the ticket.  If the device
 * loop itself fails, every queued and running query fails with its status
 * and later submits return PC_ERR_CANCELLED.
 */
pc_status pc_server_poll(pc_server* s, uint64_t ticket, pc_result* out, int64_t timeout_ns);

/* Cancel a ticket that has not been admitted yet (PC_ERR_BUSY if running). */
pc_status pc_server_cancel(pc_server* s, uint64_t ticket);

/* Latency percentiles and throughput of the completed queries so far. */
pc_status pc_server_get_stats(pc_server* s, pc_server_stats* out);

/* Stop the loop; pending tickets are cancelled; running work is drained. */
pc_status pc_server_destroy(pc_server* s);

/*
 * pc_inspect_static -- pc_inspect for callers that must not allocate device
 * memory.  The paper has no counterpart: this is a deployment variant of the
 * resident (shared-memory) solver.
 *
 * Who needs it: processes whose framework has reserved the whole device for
 * its own pool allocator, where a cudaMalloc fails or fragments that pool,
 * and latency-critical loops that cannot afford cudaMalloc / cudaFree, which
 * may synchronise the whole device.  This call performs no device allocation
 * of any kind: its scratch (counters, lattice tables, device staging of the
 * outputs) is one static device array of about 3.9 MB that every GPU loading
 * the library holds until the process exits.
 *
 * Arguments and outputs as pc_inspect with host outputs (all output pointers
 * are HOST pointers; verdicts required, the others optional); the call
 * synchronises cuda_stream before returning.
 * Limits: n_configs <= 262144; W <= 51 (at most 8192 columns, the size of
 * the static tables); the lattice must fit the resident solver's shared
 * memory, which on GB300 (227 KB per CTA) bounds it further: W <= 26 (at
 * L = 1), W = 20 up to L = 8, W = 8 up to L = 74.  Anything larger returns
 * PC_ERR_ARG with a message, before any work is enqueued.
 * Sharing: every call on a device uses the same static array, which keeps
 * the previous call's contents; counters are cleared and tables rewritten on
 * each call, but calls whose GPU work overlaps (e.g. on two streams) race on
 * the array and must be serialised by the caller.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make it before any
 * stream capture starts.  After cudaDeviceReset call pc_shutdown() before
 * the next call: it forgets the cached address (and every other cached
 * device object of the library).
 * Errors: PC_ERR_ARG, PC_ERR_CUDA.
 */
pc_status pc_inspect_static(int32_t W, int32_t L, double p, uint64_t seed,
                            int64_t config_begin, int64_t n_configs,
                            uint8_t* verdicts, int32_t* first_hit, float* mass,
                            int32_t* m_stop, int64_t* n_percolating, double* Pi,
                            void* cuda_stream);

/*
 * Plane layout used by the solvers for per-layer FP arrays (diagnostics and
 * tests; host only).  Rows of the hexagon are stored in order with 2-4 zero
 * entries before each, so that plane position mod 3 equals the column's
 * sublattice, followed by a zero zone that stands for the rows outside the
 * hexagon.  Outputs: P (entries per plane), the strips [s_begin, s_begin +
 * n_strips) (strip s = positions 3s..3s+2), strip_row [n_strips] (row index
 * 0..2W of each strip), row_off [(2W+1) x 4] (offset from a column of row r
 * to the same q in rows r-2, r-1, r+1, r+2), ppos [A] (position of each
 * column), pcol [P] (column at each position, -1 for zeros).  Query P and
 * n_strips first with NULL arrays.  Errors: PC_ERR_ARG.
 */
pc_status pc_lattice_layout(int32_t W, int32_t* P, int32_t* s_begin, int32_t* n_strips,
                            int16_t* strip_row, int32_t* row_off, int32_t* ppos, int32_t* pcol);

/*
 * The paired plane layout of the streamed solver (diagnostics and tests;
 * host only), with the outputs of pc_lattice_layout.  In addition to that
 * layout's properties, every row offset is even, so a strip pair (plane
 * positions 6h .. 6h+5) reads its runs with aligned 64-bit loads, and no
 * strip pair holds columns of two rows; the zero zones before and after the
 * rows are W + 20 entries long.  Errors: PC_ERR_ARG.
 */
pc_status pc_stream_layout(int32_t W, int32_t* P, int32_t* s_begin, int32_t* n_strips,
                           int16_t* strip_row, int32_t* row_off, int32_t* ppos, int32_t* pcol);

/*
 * Shape of the verdict-only solver with temporal blocking on the current
 * device (diagnostics and tests).  PC_BITS_ONLY inspections on the streamed
 * path run 32 steps per visit of a slab of word rows when one thread-block
 * cluster can hold every column of the lattice's cross-section in shared
 * memory (Sec. II.B: the reached set alone decides the verdict, first_hit
 * and m_stop).  Outputs (each may be NULL): cluster_size (CTAs per cluster,
 * 1..16), columns_per_cta (cross-section columns each CTA owns, one per
 * thread, at most 800), slab_rows (32-tube word rows per slab in shared
 * memory, the valid rows plus one halo row above and one below: a multiple
 * of 4 from 12 to 36), clusters (clusters the device runs at once).
 * Errors: PC_ERR_ARG (W outside [0, 255], or no cluster of this device holds
 * the cross-section -- the step-synchronous solver then runs such
 * inspections), PC_ERR_CUDA (no device).
 */
pc_status pc_bits_blocked_shape(int32_t W, int32_t* cluster_size, int32_t* columns_per_cta,
                                int32_t* slab_rows, int32_t* clusters);

/*
 * The lazy walk of the self-loop remark in Sec. II.B: at every step the
 * electron stays on its site with probability hold, otherwise it moves as
 * Eq. (2) says (the chain hold * I + (1 - hold) * P).  Percolation, first_hit
 * and m_stop do not change, and the probability of arriving at the first
 * hit is the plain one times (1 - hold)^first_hit (each of the first_hit
 * moves of a shortest spanning walk now happens with probability 1 - hold).
 * This writes that mass from pc_inspect's first_hit and mass outputs:
 * mass_lazy[i] = mass[i] * (1 - hold)^first_hit[i] (computed in FP64,
 * stored as FP32), 0 where first_hit[i] <= 0.  All three arrays have
 * n_configs entries and are host buffers (the call then synchronises
 * cuda_stream), or device buffers with flags = PC_OUT_DEVICE (asynchronous).
 * mass_lazy may alias mass.  Errors: PC_ERR_ARG (hold outside [0, 1),
 * n_configs < 0, a NULL buffer, other flag bits), PC_ERR_CUDA.
 */
pc_status pc_lazy_mass(const int32_t* first_hit, const float* mass, int64_t n_configs,
                       double hold, float* mass_lazy, int32_t flags, void* cuda_stream);

/* Release cached lattice tables, batch graphs and scratch of every device,
 * and forget the static array's cached device addresses (pc_inspect_static).
 * Call it after cudaDeviceReset, before any further call of the library. */
pc_status pc_shutdown(void);

/* Thread-local message of the last failing call ("" if none). */
const char* pc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PERCOL_H */

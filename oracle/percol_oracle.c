/*
 * percol_oracle.c -- plain, slow CPU oracle for the percolation-inspection
 * method of F. Xu, Z. Xu and B. I. Yakobson, "Site-Percolation Threshold of
 * Carbon Nanotube Fibers -- Fast Inspection of Percolation with Markov
 * Stochastic Theory" (arXiv:1401.2130).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check of the package
 * entry module and the CPU-baseline leg of the benchmark may load or call
 * this code.  The GPU library never links it, includes it or reads anything
 * it writes, and it shares no code with the GPU library: the lattice, the
 * random stream and the Markov iteration below are written independently.
 *
 * What it computes, and the passage each part follows:
 *   - Philox4x32-10 counter-based generator: J. K. Salmon, M. A. Moraes,
 *     R. O. Dror, D. E. Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3",
 *     SC'11 (round function, multipliers and Weyl key schedule from there).
 *   - Lattice (Sec. II.A, Fig. 1): FCC sites with tubes along <111>;
 *     hexagonal cross-section of radius W (unit = nearest axis-to-axis
 *     spacing of the projected columns); L tubes per column.  Neighbours are
 *     derived GEOMETRICALLY: the 12 FCC nearest neighbours are the sites at
 *     Euclidean distance sqrt(3) (side contacts) and the 2 end contacts are
 *     the sites of the same column one FCC period up or down (Sec. II.A:
 *     coordination 14 = 12 side + 2 end).
 *   - Occupancy (Sec. II.A): each site metallic with probability p
 *     (Bernoulli), drawn from the counter layout documented below.
 *   - Transition matrix (Eqs. (1)-(2)) over metallic sites, plus the detector
 *     site j1 connected to every metallic site of the far end surface
 *     (Sec. II.B).  Built explicitly in CSR, FP64.
 *   - First-passage recursion (Eqs. (3)-(4), Appendix Eqs. (A.1)-(A.3)):
 *     forward propagation of the start distribution with the detector column
 *     removed, and the backward f^(m) recursion, both FP64.
 *   - Stop rule (Sec. II.B): stop when the detector probability becomes
 *     non-zero (decided on the exact support, so FP underflow cannot decide
 *     it), or when the reached set stops growing; N_max = min(N_b, Np) + 1
 *     bounds the step count.
 *   - Independent verdict routes: breadth-first search (the shortest spanning
 *     path of Sec. II.B is the BFS distance) and union-find.
 *   - The lazy walk of the self-loop remark (Sec. II.B): forward first
 *     passage under hold * I + (1 - hold) * P.
 *   - Critical word per configuration: union-find over the sites in
 *     increasing order of their random word; it gives the verdict at every p
 *     at once (used by the finite-size-scaling pin of the lattice, Sec. III).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   * mu_0 is uniform over the metallic sites of the start layer t = 0.
 *   * deg(i) counts the detector for end-layer sites (Sec. II.B detector).
 *   * a metallic site with deg 0 has an all-zero row: its mass is dropped.
 *   * L = 1: start layer = end layer; the first hit is at m = 1.
 *
 * Counter layout of the occupancy stream (not in the paper; fixed here):
 *   key = (seed & 0xffffffff, seed >> 32)
 *   ctr = (site >> 2, config_index, W | (L << 8), 0)
 *   site i takes output word (i & 3); metallic <=> (uint64)word < T,
 *   T = floor(p * 2^32) computed in double (exact power-of-two scaling).
 * Site order: i = t * A + a, a = column rank in row-major order over
 * r = -W..W and, within a row, q ascending; (q, r) axial hexagon coordinates
 * with max(|q|, |r|, |q + r|) <= W.  Sublattice sigma = (q - r) mod 3 and
 * FCC layer height h = 3 t + sigma.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_OOM (-2)
#define OR_ERR_NMAX (-7) /* N_max bound violated: an internal inconsistency */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11)                                      */
/* ------------------------------------------------------------------------ */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]) {
  /* Multipliers of the two 32x32->64 products and the Weyl increments of the
   * key schedule, as published for Philox-4x32. */
  const uint32_t M_A = 0xD2511F53u, M_B = 0xCD9E8D57u;
  const uint32_t WEYL_0 = 0x9E3779B9u, WEYL_1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t pa = (uint64_t)M_A * (uint64_t)x0;
    uint64_t pb = (uint64_t)M_B * (uint64_t)x2;
    uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
    uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
    uint32_t y0 = pb_hi ^ x1 ^ k0;
    uint32_t y1 = pb_lo;
    uint32_t y2 = pa_hi ^ x3 ^ k1;
    uint32_t y3 = pa_lo;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += WEYL_0; /* key for the next round */
    k1 += WEYL_1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

uint64_t oracle_threshold(double p) {
  /* T = floor(p * 2^32); p in [0, 1]; p = 1 gives 2^32 (every site). */
  return (uint64_t)floor(p * 4294967296.0);
}

/* ------------------------------------------------------------------------ */
/* Lattice (Sec. II.A, Fig. 1)                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
  int W, L;
  int64_t A, N;
  int *q, *r, *sigma;   /* per column */
  /* Column-level neighbour list: for column a, entries k in
   * [cptr[a], cptr[a+1]) give a neighbouring column cnb[k] and the tube-index
   * offset cdt[k] (site (a, t) touches (cnb[k], t + cdt[k])). */
  int64_t *cptr;
  int *cnb, *cdt;
} lattice_t;

static int hex_inside(int W, int q, int r) {
  int s = q + r;
  return abs(q) <= W && abs(r) <= W && abs(s) <= W;
}

static int mod3(int v) { int m = v % 3; return m < 0 ? m + 3 : m; }

int64_t oracle_n_columns(int W) {
  int64_t n = 0;
  for (int r = -W; r <= W; ++r)
    for (int q = -W; q <= W; ++q)
      if (hex_inside(W, q, r)) ++n;
  return n;
}

static void lattice_free(lattice_t *lat) {
  free(lat->q); free(lat->r); free(lat->sigma);
  free(lat->cptr); free(lat->cnb); free(lat->cdt);
  memset(lat, 0, sizeof(*lat));
}

/*
 * Geometry: projected column (q, r) sits at x = q + r/2, y = r*sqrt(3)/2
 * (unit = nearest projected axis spacing).  Layer h = 3t + sigma sits at
 * z = h*sqrt(2): one FCC (111) layer spacing for nearest-neighbour distance
 * sqrt(3).  Squared distance times 4:
 *   4 d^2 = (2 dq + dr)^2 + 3 dr^2 + 8 dh^2.
 * Side contact  <=> 4 d^2 = 12 (FCC nearest neighbour, d = sqrt(3)).
 * End contact   <=> same column and |dh| = 3 (one FCC period along <111>).
 */
static int geometric_contact(int dq, int dr, int dh) {
  int ex = 2 * dq + dr;
  int d4 = ex * ex + 3 * dr * dr + 8 * dh * dh;
  if (d4 == 12) return 1;
  if (dq == 0 && dr == 0 && (dh == 3 || dh == -3)) return 1;
  return 0;
}

static int lattice_build(lattice_t *lat, int W, int L) {
  memset(lat, 0, sizeof(*lat));
  lat->W = W; lat->L = L;
  int64_t A = oracle_n_columns(W);
  lat->A = A; lat->N = A * (int64_t)L;
  lat->q = malloc(sizeof(int) * A);
  lat->r = malloc(sizeof(int) * A);
  lat->sigma = malloc(sizeof(int) * A);
  lat->cptr = malloc(sizeof(int64_t) * (A + 1));
  if (!lat->q || !lat->r || !lat->sigma || !lat->cptr) { lattice_free(lat); return OR_ERR_OOM; }
  int64_t a = 0;
  for (int r = -W; r <= W; ++r)
    for (int q = -W; q <= W; ++q)
      if (hex_inside(W, q, r)) {
        lat->q[a] = q; lat->r[a] = r; lat->sigma[a] = mod3(q - r); ++a;
      }
  /* Count (pass 0), then fill (pass 1).  Candidate partners: every column,
   * tube offsets -1..+1 (a contact changes h by at most 3, hence t by at
   * most 1).  The |dq|, |dr| <= 2 prefilter only skips pairs whose projected
   * distance alone already exceeds sqrt(3). */
  int64_t total = 0;
  for (int pass = 0; pass < 2; ++pass) {
    total = 0;
    for (int64_t i = 0; i < A; ++i) {
      lat->cptr[i] = total;
      for (int64_t j = 0; j < A; ++j) {
        int dq = lat->q[j] - lat->q[i], dr = lat->r[j] - lat->r[i];
        if (dq > 2 || dq < -2 || dr > 2 || dr < -2) continue;
        for (int dt = -1; dt <= 1; ++dt) {
          int dh = 3 * dt + lat->sigma[j] - lat->sigma[i];
          if (geometric_contact(dq, dr, dh)) {
            if (pass == 1) { lat->cnb[total] = (int)j; lat->cdt[total] = dt; }
            ++total;
          }
        }
      }
    }
    lat->cptr[A] = total;
    if (pass == 0) {
      lat->cnb = malloc(sizeof(int) * (total ? total : 1));
      lat->cdt = malloc(sizeof(int) * (total ? total : 1));
      if (!lat->cnb || !lat->cdt) { lattice_free(lat); return OR_ERR_OOM; }
    }
  }
  return OR_OK;
}

/* Lattice neighbours of site i (ignoring occupancy).  Returns the count. */
static int site_neighbours(const lattice_t *lat, int64_t i, int64_t *out) {
  int64_t a = i % lat->A, t = i / lat->A;
  int n = 0;
  for (int64_t k = lat->cptr[a]; k < lat->cptr[a + 1]; ++k) {
    int64_t tt = t + lat->cdt[k];
    if (tt < 0 || tt >= lat->L) continue;
    out[n++] = tt * lat->A + lat->cnb[k];
  }
  return n;
}

/* ------------------------------------------------------------------------ */
/* Occupancy (Sec. II.A)                                                     */
/* ------------------------------------------------------------------------ */

static void draw_occupancy(int W, int L, int64_t N, double p, uint64_t seed,
                           uint64_t config, uint8_t *occ) {
  uint64_t T = oracle_threshold(p);
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  uint32_t word[4] = {0, 0, 0, 0};
  for (int64_t i = 0; i < N; ++i) {
    if ((i & 3) == 0) {
      uint32_t ctr[4] = {(uint32_t)(i >> 2), (uint32_t)config,
                         (uint32_t)W | ((uint32_t)L << 8), 0u};
      oracle_philox4x32_10(ctr, key, word);
    }
    occ[i] = ((uint64_t)word[i & 3] < T) ? 1 : 0;
  }
}

/* ------------------------------------------------------------------------ */
/* Explicit transition matrix with detector (Eqs. (1)-(2), Sec. II.B)        */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t Np;          /* metallic sites */
  int64_t Nb;          /* bonds between metallic sites (lattice bonds) */
  int64_t *site;       /* compact index -> site id */
  int64_t *ptr;        /* CSR over compact rows, size Np + 1 */
  int64_t *col;        /* compact column, or DET (= Np) for the detector j1 */
  double *val;         /* P_ij = 1 / deg(i) */
  int *deg;            /* per compact row */
  uint8_t *is_start, *is_end;
} markov_t;

static void markov_free(markov_t *M) {
  free(M->site); free(M->ptr); free(M->col); free(M->val); free(M->deg);
  free(M->is_start); free(M->is_end);
  memset(M, 0, sizeof(*M));
}

static int markov_build(const lattice_t *lat, const uint8_t *occ, markov_t *M) {
  memset(M, 0, sizeof(*M));
  int64_t N = lat->N, A = lat->A;
  int64_t *cidx = malloc(sizeof(int64_t) * N);
  if (!cidx) return OR_ERR_OOM;
  int64_t Np = 0;
  for (int64_t i = 0; i < N; ++i) cidx[i] = occ[i] ? Np++ : -1;
  M->Np = Np;
  M->site = malloc(sizeof(int64_t) * (Np ? Np : 1));
  M->ptr = malloc(sizeof(int64_t) * (Np + 1));
  M->deg = malloc(sizeof(int) * (Np ? Np : 1));
  M->is_start = calloc(Np ? Np : 1, 1);
  M->is_end = calloc(Np ? Np : 1, 1);
  if (!M->site || !M->ptr || !M->deg || !M->is_start || !M->is_end) { free(cidx); markov_free(M); return OR_ERR_OOM; }
  int64_t nb[32];
  int64_t nnz = 0, bonds2 = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (!occ[i]) continue;
    int64_t k = cidx[i];
    M->site[k] = i;
    int64_t t = i / A;
    M->is_start[k] = (t == 0);
    M->is_end[k] = (t == lat->L - 1);
    int n = site_neighbours(lat, i, nb), d = 0;
    for (int e = 0; e < n; ++e) if (occ[nb[e]]) ++d;
    bonds2 += d;
    if (M->is_end[k]) ++d; /* detector edge (Sec. II.B) */
    M->deg[k] = d;
    nnz += d;
  }
  M->Nb = bonds2 / 2;
  M->col = malloc(sizeof(int64_t) * (nnz ? nnz : 1));
  M->val = malloc(sizeof(double) * (nnz ? nnz : 1));
  if (!M->col || !M->val) { free(cidx); markov_free(M); return OR_ERR_OOM; }
  int64_t pos = 0;
  for (int64_t k = 0; k < Np; ++k) {
    M->ptr[k] = pos;
    int64_t i = M->site[k];
    int d = M->deg[k];
    if (d == 0) continue; /* isolated metallic site: zero row */
    double w = 1.0 / (double)d; /* Eq. (2) */
    int n = site_neighbours(lat, i, nb);
    for (int e = 0; e < n; ++e)
      if (occ[nb[e]]) { M->col[pos] = cidx[nb[e]]; M->val[pos] = w; ++pos; }
    if (M->is_end[k]) { M->col[pos] = Np; M->val[pos] = w; ++pos; }
  }
  M->ptr[Np] = pos;
  free(cidx);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Markov inspection of one configuration (Eqs. (3)-(4), Sec. II.B)          */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t verdict, first_hit, m_stop;
  double mass;          /* a_{first_hit}; 0 if no hit */
  int64_t n0, Np, Nb;
  double dropped;       /* mass lost at deg-0 sites up to m_stop */
  double residual;      /* sum of mu_{m_stop - 1} left on the lattice */
  double absorbed;      /* sum of a_m, m <= m_stop */
  int32_t fp_first_nonzero; /* first m with a_m > 0 in FP64, or -1 */
  int32_t nmax_ok;      /* m_stop <= N_max */
} markov_out_t;

/*
 * Forward form: mu_m(j) = sum_i mu_{m-1}(i) P_ij for j != j1, and the mass
 * hitting j1 at step m, a_m = sum_i mu_{m-1}(i) P_{i j1}.  By Appendix
 * Eq. (A.3), a_m = mu_0^T f^(m): the first-passage probability of Eq. (3)
 * averaged over the start distribution.
 * Exact support S_m = supp(mu_m) is propagated with the same sparsity
 * pattern; R_m = R_{m-1} u S_m.  a_m != 0 exactly <=> S_{m-1} meets the end
 * surface.  Stop at the first such m, or once R stops growing.  With
 * run_to_nmax the iteration continues to N_max after R stops growing, to
 * confirm that no later hit exists (used by tests on tiny lattices).
 */
static int markov_inspect(const lattice_t *lat, const uint8_t *occ,
                          int run_to_nmax, markov_out_t *o) {
  memset(o, 0, sizeof(*o));
  o->first_hit = -1; o->fp_first_nonzero = -1; o->nmax_ok = 1;
  markov_t M;
  int st = markov_build(lat, occ, &M);
  if (st) return st;
  int64_t Np = M.Np;
  o->Np = Np; o->Nb = M.Nb;
  int64_t nmax = (M.Nb < Np ? M.Nb : Np) + 1;
  double *mu = calloc(Np ? Np : 1, sizeof(double));
  double *mu2 = calloc(Np ? Np : 1, sizeof(double));
  uint8_t *S = calloc(Np ? Np : 1, 1), *S2 = calloc(Np ? Np : 1, 1);
  uint8_t *R = calloc(Np ? Np : 1, 1);
  if (!mu || !mu2 || !S || !S2 || !R) { st = OR_ERR_OOM; goto done; }
  int64_t n0 = 0;
  for (int64_t k = 0; k < Np; ++k) n0 += M.is_start[k];
  o->n0 = n0;
  if (n0 == 0) { o->m_stop = 0; goto done; }
  for (int64_t k = 0; k < Np; ++k)
    if (M.is_start[k]) { mu[k] = 1.0 / (double)n0; S[k] = 1; R[k] = 1; }
  int decided = 0;
  for (int64_t m = 1;; ++m) {
    /* a_m from mu_{m-1}; exact test: S_{m-1} meets the end surface */
    double a = 0.0;
    int hit_exact = 0;
    for (int64_t k = 0; k < Np; ++k) {
      if (M.is_end[k] && S[k]) hit_exact = 1;
      for (int64_t e = M.ptr[k]; e < M.ptr[k + 1]; ++e)
        if (M.col[e] == Np) a += mu[k] * M.val[e];
    }
    if (a > 0.0 && o->fp_first_nonzero < 0) o->fp_first_nonzero = (int32_t)m;
    if (decided) {
      /* run_to_nmax: after the reached set stopped growing no hit may follow */
      if (hit_exact || a > 0.0) { o->nmax_ok = 0; break; }
      if (m > nmax) break;
    } else if (hit_exact) {
      o->verdict = 1; o->first_hit = (int32_t)m; o->mass = a; o->m_stop = (int32_t)m;
      if (m > nmax) o->nmax_ok = 0;
      double res = 0.0;
      for (int64_t k = 0; k < Np; ++k) res += mu[k];
      o->residual = res; /* mass of mu_{m-1}, before this step's absorption */
      break;
    }
    /* mu_m = mu_{m-1} ^(j1)P (Eq. (4): column j1 removed) and S_m */
    memset(mu2, 0, sizeof(double) * Np);
    memset(S2, 0, Np);
    double drop = 0.0;
    for (int64_t k = 0; k < Np; ++k) {
      if (M.deg[k] == 0) drop += mu[k];
      for (int64_t e = M.ptr[k]; e < M.ptr[k + 1]; ++e) {
        int64_t j = M.col[e];
        if (j == Np) continue;
        mu2[j] += mu[k] * M.val[e];
        if (S[k]) S2[j] = 1;
      }
    }
    if (!decided) { o->absorbed += a; o->dropped += drop; }
    int grew = 0;
    for (int64_t k = 0; k < Np; ++k)
      if (S2[k] && !R[k]) { R[k] = 1; grew = 1; }
    { double *t = mu; mu = mu2; mu2 = t; }
    { uint8_t *t = S; S = S2; S2 = t; }
    if (decided && grew) { o->nmax_ok = 0; break; } /* cannot happen */
    if (!grew && !decided) {
      o->verdict = 0; o->first_hit = -1; o->mass = 0.0; o->m_stop = (int32_t)m;
      if (m > nmax) o->nmax_ok = 0;
      double res = 0.0;
      for (int64_t k = 0; k < Np; ++k) res += mu[k];
      o->residual = res; /* mass of mu_m */
      decided = 1;
      if (!run_to_nmax) break;
    }
  }
done:
  free(mu); free(mu2); free(S); free(S2); free(R);
  markov_free(&M);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Breadth-first search (shortest spanning path, Sec. II.B)                  */
/* ------------------------------------------------------------------------ */

static int bfs_inspect(const lattice_t *lat, const uint8_t *occ, int32_t *verdict,
                       int32_t *first_hit, int32_t *m_stop) {
  int64_t N = lat->N, A = lat->A;
  int32_t *dist = malloc(sizeof(int32_t) * N);
  int64_t *queue = malloc(sizeof(int64_t) * N);
  if (!dist || !queue) { free(dist); free(queue); return OR_ERR_OOM; }
  for (int64_t i = 0; i < N; ++i) dist[i] = -1;
  int64_t head = 0, tail = 0;
  for (int64_t a = 0; a < A; ++a)
    if (occ[a]) { dist[a] = 0; queue[tail++] = a; }
  *verdict = 0; *first_hit = -1; *m_stop = 0;
  if (tail == 0) { free(dist); free(queue); return OR_OK; }
  int32_t ecc = 0;
  int64_t nb[32];
  while (head < tail) {
    int64_t i = queue[head++];
    if (dist[i] > ecc) ecc = dist[i];
    int n = site_neighbours(lat, i, nb);
    for (int e = 0; e < n; ++e) {
      int64_t j = nb[e];
      if (occ[j] && dist[j] < 0) { dist[j] = dist[i] + 1; queue[tail++] = j; }
    }
  }
  int32_t best = -1;
  for (int64_t a = 0; a < A; ++a) {
    int64_t i = (int64_t)(lat->L - 1) * A + a;
    if (dist[i] >= 0 && (best < 0 || dist[i] < best)) best = dist[i];
  }
  if (best >= 0) { *verdict = 1; *first_hit = best + 1; *m_stop = best + 1; }
  else { *verdict = 0; *first_hit = -1; *m_stop = ecc + 1; }
  free(dist); free(queue);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Union-find spanning test (verdict only)                                   */
/* ------------------------------------------------------------------------ */

static int64_t uf_find(int64_t *parent, int64_t x) {
  while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; }
  return x;
}

static int uf_inspect(const lattice_t *lat, const uint8_t *occ, int32_t *verdict) {
  int64_t N = lat->N, A = lat->A;
  int64_t TOP = N, BOT = N + 1;
  int64_t *parent = malloc(sizeof(int64_t) * (N + 2));
  if (!parent) return OR_ERR_OOM;
  for (int64_t i = 0; i < N + 2; ++i) parent[i] = i;
  int64_t nb[32];
  for (int64_t i = 0; i < N; ++i) {
    if (!occ[i]) continue;
    int64_t t = i / A;
    if (t == 0) { int64_t x = uf_find(parent, i), y = uf_find(parent, TOP); if (x != y) parent[x] = y; }
    if (t == lat->L - 1) { int64_t x = uf_find(parent, i), y = uf_find(parent, BOT); if (x != y) parent[x] = y; }
    int n = site_neighbours(lat, i, nb);
    for (int e = 0; e < n; ++e)
      if (occ[nb[e]]) { int64_t x = uf_find(parent, i), y = uf_find(parent, nb[e]); if (x != y) parent[x] = y; }
  }
  *verdict = uf_find(parent, TOP) == uf_find(parent, BOT);
  free(parent);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Exported API                                                              */
/* ------------------------------------------------------------------------ */

static int check_args(int W, int L) {
  if (W < 0 || W > 255 || L < 1 || L >= (1 << 24)) return OR_ERR_ARG;
  return OR_OK;
}

int oracle_lattice_info(int W, int L, int64_t *n_columns, int64_t *n_sites) {
  if (check_args(W, L)) return OR_ERR_ARG;
  int64_t A = oracle_n_columns(W);
  if (n_columns) *n_columns = A;
  if (n_sites) *n_sites = A * (int64_t)L;
  return OR_OK;
}

/* Column coordinates in canonical order. */
int oracle_columns(int W, int32_t *q, int32_t *r, int32_t *sigma) {
  if (W < 0 || W > 255) return OR_ERR_ARG;
  int64_t a = 0;
  for (int rr = -W; rr <= W; ++rr)
    for (int qq = -W; qq <= W; ++qq)
      if (hex_inside(W, qq, rr)) { q[a] = qq; r[a] = rr; sigma[a] = mod3(qq - rr); ++a; }
  return OR_OK;
}

/* Full lattice adjacency: nbr[i*14 + k] (k < count[i]) lists the neighbours
 * of site i; unused slots are -1.  Returns OR_ERR_ARG if some site had more
 * than 14 neighbours (the geometry forbids it). */
int oracle_adjacency(int W, int L, int64_t *nbr, int32_t *count) {
  if (check_args(W, L)) return OR_ERR_ARG;
  lattice_t lat;
  int st = lattice_build(&lat, W, L);
  if (st) return st;
  int64_t tmp[32];
  for (int64_t i = 0; i < lat.N; ++i) {
    int n = site_neighbours(&lat, i, tmp);
    if (n > 14) { lattice_free(&lat); return OR_ERR_ARG; }
    count[i] = n;
    for (int k = 0; k < 14; ++k) nbr[i * 14 + k] = k < n ? tmp[k] : -1;
  }
  lattice_free(&lat);
  return OR_OK;
}

/* Occupancy of configs [cfg0, cfg0 + n) as bytes, [n][N]. */
int oracle_occupancy(int W, int L, double p, uint64_t seed, int64_t cfg0,
                     int64_t n, uint8_t *occ) {
  if (check_args(W, L) || !(p >= 0.0 && p <= 1.0) || cfg0 < 0 || n < 0 ||
      cfg0 + n > 4294967296LL) return OR_ERR_ARG;
  int64_t N = oracle_n_columns(W) * (int64_t)L;
  for (int64_t c = 0; c < n; ++c)
    draw_occupancy(W, L, N, p, seed, (uint64_t)(cfg0 + c), occ + c * N);
  return OR_OK;
}

/*
 * The 32-bit random word of every site (words: [n][N]) of configurations
 * cfg0..cfg0+n-1: the same counter stream as the Bernoulli draw above.  The
 * fixed-count sample space of Sec. II.A (a random permutation of the sites
 * puts exactly Np of them metallic) is built from these words by the Python
 * wrapper: the metallic sites are the Np smallest keys (word, site index).
 */
int oracle_site_words(int W, int L, uint64_t seed, int64_t cfg0, int64_t n, uint32_t *words) {
  if (check_args(W, L) || cfg0 < 0 || n < 0 || cfg0 + n > 4294967296LL) return OR_ERR_ARG;
  int64_t N = oracle_n_columns(W) * (int64_t)L;
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (int64_t c = 0; c < n; ++c) {
    uint32_t word[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < N; ++i) {
      if ((i & 3) == 0) {
        uint32_t ctr[4] = {(uint32_t)(i >> 2), (uint32_t)(cfg0 + c),
                           (uint32_t)W | ((uint32_t)L << 8), 0u};
        oracle_philox4x32_10(ctr, key, word);
      }
      words[c * N + i] = word[i & 3];
    }
  }
  return OR_OK;
}

static int cmp_u64(const void *x, const void *y) {
  uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
  return a < b ? -1 : a > b;
}

/*
 * Critical word of each configuration cfg0..cfg0+n-1 (out: [n]).  With the
 * coupled draws above, site i is metallic at p exactly when its word is below
 * T(p), so a configuration percolates at p exactly when T(p) exceeds its
 * critical word w*: the word of the site whose addition, in increasing order
 * of (word, site index), first joins the start face t = 0 to the end face
 * t = L-1 through metallic sites (Sec. II.B: percolation is the existence of
 * such a path).  One pass gives the verdict at every p, so Pi(p) of Eq. (5)
 * is the empirical distribution of w* / 2^32.
 * nbr/count: the adjacency to use, laid out as oracle_adjacency writes it
 * ([N][14], -1 padded, and the count per site); NULL = the lattice's own.
 * w* is 2^32 only if no spanning path exists with every site metallic, which
 * the axial contacts of each column rule out.
 */
int oracle_critical_words(int W, int L, const int64_t *nbr, const int32_t *count, uint64_t seed,
                          int64_t cfg0, int64_t n, int threads, uint64_t *out) {
  if (check_args(W, L) || cfg0 < 0 || n < 0 || cfg0 + n > 4294967296LL) return OR_ERR_ARG;
  lattice_t lat;
  int st = lattice_build(&lat, W, L);
  if (st) return st;
  const int64_t N = lat.N, A = lat.A;
  if (N >= (1LL << 32)) { lattice_free(&lat); return OR_ERR_ARG; }
  int err = OR_OK;
#ifdef _OPENMP
  int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int64_t c = 0; c < n; ++c) {
    uint32_t *w = malloc(sizeof(uint32_t) * N);
    uint64_t *key = malloc(sizeof(uint64_t) * N);
    int64_t *parent = malloc(sizeof(int64_t) * (N + 2));
    uint8_t *on = calloc(N, 1);
    if (!w || !key || !parent || !on) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      err = OR_ERR_OOM;
      free(w); free(key); free(parent); free(on);
      continue;
    }
    oracle_site_words(W, L, seed, cfg0 + c, 1, w);
    for (int64_t i = 0; i < N; ++i) key[i] = ((uint64_t)w[i] << 32) | (uint64_t)i;
    qsort(key, (size_t)N, sizeof(uint64_t), cmp_u64);
    const int64_t TOP = N, BOT = N + 1;
    for (int64_t i = 0; i < N + 2; ++i) parent[i] = i;
    uint64_t crit = 1ULL << 32;
    int64_t nb[32];
    for (int64_t j = 0; j < N; ++j) {
      const int64_t i = (int64_t)(key[j] & 0xffffffffu), t = i / A;
      on[i] = 1;
      if (t == 0) { int64_t x = uf_find(parent, i), y = uf_find(parent, TOP); if (x != y) parent[x] = y; }
      if (t == L - 1) { int64_t x = uf_find(parent, i), y = uf_find(parent, BOT); if (x != y) parent[x] = y; }
      int m;
      if (nbr) {
        m = count[i];
        for (int k = 0; k < m; ++k) nb[k] = nbr[i * 14 + k];
      } else {
        m = site_neighbours(&lat, i, nb);
      }
      for (int k = 0; k < m; ++k)
        if (on[nb[k]]) { int64_t x = uf_find(parent, i), y = uf_find(parent, nb[k]); if (x != y) parent[x] = y; }
      if (uf_find(parent, TOP) == uf_find(parent, BOT)) { crit = key[j] >> 32; break; }
    }
    out[c] = crit;
    free(w); free(key); free(parent); free(on);
  }
  lattice_free(&lat);
  return err;
}

enum { MODE_MARKOV = 0, MODE_BFS = 1, MODE_UNIONFIND = 2, MODE_MARKOV_FULL = 3 };

/*
 * Inspect configurations given explicitly (occ: [n][N] bytes) or drawn from
 * the stream (occ == NULL: configs cfg0..cfg0+n-1 at probability p).
 * Outputs (each may be NULL): verdict, first_hit, m_stop, mass (a_{first_hit}),
 * and stats[n][8] = {n0, Np, Nb, dropped, residual, absorbed,
 * fp_first_nonzero, nmax_ok} (Markov modes only).
 * threads <= 0 uses the OpenMP default.  Parallel over configurations.
 */
int oracle_inspect(int W, int L, const uint8_t *occ_in, double p, uint64_t seed,
                   int64_t cfg0, int64_t n, int mode, int threads,
                   int32_t *verdict, int32_t *first_hit, int32_t *m_stop,
                   double *mass, double *stats) {
  if (check_args(W, L) || n < 0 || mode < 0 || mode > 3) return OR_ERR_ARG;
  if (!occ_in && (!(p >= 0.0 && p <= 1.0) || cfg0 < 0 || cfg0 + n > 4294967296LL)) return OR_ERR_ARG;
  lattice_t lat;
  int st = lattice_build(&lat, W, L);
  if (st) return st;
  int err = OR_OK;
#ifdef _OPENMP
  int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
#endif
  for (int64_t c = 0; c < n; ++c) {
    uint8_t *own = NULL;
    const uint8_t *occ;
    if (occ_in) occ = occ_in + c * lat.N;
    else {
      own = malloc(lat.N ? lat.N : 1);
      if (!own) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
        err = OR_ERR_OOM;
        continue;
      }
      draw_occupancy(W, L, lat.N, p, seed, (uint64_t)(cfg0 + c), own);
      occ = own;
    }
    int32_t v = 0, fh = -1, ms = 0;
    double ma = 0.0;
    int s2 = OR_OK;
    if (mode == MODE_MARKOV || mode == MODE_MARKOV_FULL) {
      markov_out_t o;
      s2 = markov_inspect(&lat, occ, mode == MODE_MARKOV_FULL, &o);
      v = o.verdict; fh = o.first_hit; ms = o.m_stop; ma = o.mass;
      if (stats) {
        double *s = stats + c * 8;
        s[0] = (double)o.n0; s[1] = (double)o.Np; s[2] = (double)o.Nb;
        s[3] = o.dropped; s[4] = o.residual; s[5] = o.absorbed;
        s[6] = (double)o.fp_first_nonzero; s[7] = (double)o.nmax_ok;
      }
    } else if (mode == MODE_BFS) {
      s2 = bfs_inspect(&lat, occ, &v, &fh, &ms);
    } else {
      s2 = uf_inspect(&lat, occ, &v);
    }
    if (s2) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      err = s2;
    }
    if (verdict) verdict[c] = v;
    if (first_hit) first_hit[c] = fh;
    if (m_stop) m_stop[c] = ms;
    if (mass) mass[c] = ma;
    free(own);
  }
  lattice_free(&lat);
  return err;
}

/*
 * First-passage probabilities a_m, m = 1..mmax, for one explicit
 * configuration, by two routes (Appendix Eq. (A.3)):
 *   forward : a_m = sum_i mu_{m-1}(i) P_{i j1}, mu_m = mu_{m-1} ^(j1)P
 *   backward: f^(1) = P[:, j1], f^(m) = ^(j1)P f^(m-1), a_m = mu_0^T f^(m)
 * mu_0 uniform over metallic start-layer sites (zero vector if none).
 */
int oracle_first_passage(int W, int L, const uint8_t *occ, int32_t mmax,
                         double *a_forward, double *a_backward) {
  if (check_args(W, L) || mmax < 0) return OR_ERR_ARG;
  lattice_t lat;
  int st = lattice_build(&lat, W, L);
  if (st) return st;
  markov_t M;
  st = markov_build(&lat, occ, &M);
  if (st) { lattice_free(&lat); return st; }
  int64_t Np = M.Np;
  double *mu = calloc(Np + 1, sizeof(double)), *mu2 = calloc(Np + 1, sizeof(double));
  double *f = calloc(Np + 1, sizeof(double)), *f2 = calloc(Np + 1, sizeof(double));
  double *mu0 = calloc(Np + 1, sizeof(double));
  if (!mu || !mu2 || !f || !f2 || !mu0) { st = OR_ERR_OOM; goto out; }
  int64_t n0 = 0;
  for (int64_t k = 0; k < Np; ++k) n0 += M.is_start[k];
  for (int64_t k = 0; k < Np; ++k) mu0[k] = (n0 && M.is_start[k]) ? 1.0 / (double)n0 : 0.0;
  memcpy(mu, mu0, sizeof(double) * Np);
  /* f^(1) = column j1 of P */
  for (int64_t k = 0; k < Np; ++k)
    for (int64_t e = M.ptr[k]; e < M.ptr[k + 1]; ++e)
      if (M.col[e] == Np) f[k] = M.val[e];
  for (int32_t m = 1; m <= mmax; ++m) {
    double a = 0.0;
    for (int64_t k = 0; k < Np; ++k)
      for (int64_t e = M.ptr[k]; e < M.ptr[k + 1]; ++e)
        if (M.col[e] == Np) a += mu[k] * M.val[e];
    a_forward[m - 1] = a;
    double b = 0.0;
    for (int64_t k = 0; k < Np; ++k) b += mu0[k] * f[k];
    a_backward[m - 1] = b;
    /* advance both */
    memset(mu2, 0, sizeof(double) * Np);
    for (int64_t k = 0; k < Np; ++k)
      for (int64_t e = M.ptr[k]; e < M.ptr[k + 1]; ++e)
        if (M.col[e] != Np) mu2[M.col[e]] += mu[k] * M.val[e];
    for (int64_t k = 0; k < Np; ++k) {
      double s = 0.0;
      for (int64_t e = M.ptr[k]; e < M.ptr[k + 1]; ++e)
        if (M.col[e] != Np) s += M.val[e] * f[M.col[e]];
      f2[k] = s;
    }
    { double *t = mu; mu = mu2; mu2 = t; }
    { double *t = f; f = f2; f2 = t; }
  }
out:
  free(mu); free(mu2); free(f); free(f2); free(mu0);
  markov_free(&M);
  lattice_free(&lat);
  return st;
}

/*
 * The lazy walk of the self-loop remark in Sec. II.B: at every step the
 * electron stays on its site with probability hold and otherwise moves as
 * Eq. (2) says, i.e. the chain hold * I + (1 - hold) * P over the metallic
 * sites (the detector stays absorbing).  Forward first-passage probabilities
 * a_m, m = 1..mmax, as oracle_first_passage computes them for P:
 *   a_m = (1 - hold) sum_i mu_{m-1}(i) P_{i j1},
 *   mu_m = hold mu_{m-1} + (1 - hold) mu_{m-1} ^(j1)P.
 * hold in [0, 1).
 */
int oracle_first_passage_lazy(int W, int L, const uint8_t *occ, int32_t mmax, double hold,
                              double *a_forward) {
  if (check_args(W, L) || mmax < 0 || !(hold >= 0.0 && hold < 1.0)) return OR_ERR_ARG;
  lattice_t lat;
  int st = lattice_build(&lat, W, L);
  if (st) return st;
  markov_t M;
  st = markov_build(&lat, occ, &M);
  if (st) { lattice_free(&lat); return st; }
  int64_t Np = M.Np;
  double *mu = calloc(Np + 1, sizeof(double)), *mu2 = calloc(Np + 1, sizeof(double));
  if (!mu || !mu2) { st = OR_ERR_OOM; goto out; }
  int64_t n0 = 0;
  for (int64_t k = 0; k < Np; ++k) n0 += M.is_start[k];
  for (int64_t k = 0; k < Np; ++k) mu[k] = (n0 && M.is_start[k]) ? 1.0 / (double)n0 : 0.0;
  for (int32_t m = 1; m <= mmax; ++m) {
    double a = 0.0;
    for (int64_t k = 0; k < Np; ++k)
      for (int64_t e = M.ptr[k]; e < M.ptr[k + 1]; ++e)
        if (M.col[e] == Np) a += mu[k] * M.val[e];
    a_forward[m - 1] = (1.0 - hold) * a;
    for (int64_t k = 0; k < Np; ++k) mu2[k] = hold * mu[k];
    for (int64_t k = 0; k < Np; ++k)
      for (int64_t e = M.ptr[k]; e < M.ptr[k + 1]; ++e)
        if (M.col[e] != Np) mu2[M.col[e]] += (1.0 - hold) * mu[k] * M.val[e];
    { double *t = mu; mu = mu2; mu2 = t; }
  }
out:
  free(mu); free(mu2);
  markov_free(&M);
  lattice_free(&lat);
  return st;
}

/*
 * Eq. (3) on an explicit dense n x n transition matrix P (row-major):
 * returns f^(m)_{i0} = P_{i0}[tau_{j0} = m] for m = 1..mmax.
 */
int oracle_first_passage_dense(int n, const double *P, int j0, int i0,
                               int mmax, double *out) {
  if (n <= 0 || j0 < 0 || j0 >= n || i0 < 0 || i0 >= n || mmax < 0) return OR_ERR_ARG;
  double *f = malloc(sizeof(double) * n), *g = malloc(sizeof(double) * n);
  if (!f || !g) { free(f); free(g); return OR_ERR_OOM; }
  for (int i = 0; i < n; ++i) f[i] = P[i * n + j0];
  for (int m = 1; m <= mmax; ++m) {
    out[m - 1] = f[i0];
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int k = 0; k < n; ++k)
        if (k != j0) s += P[i * n + k] * f[k]; /* ^(j0)P: column j0 zeroed */
      g[i] = s;
    }
    double *t = f; f = g; g = t;
  }
  free(f); free(g);
  return OR_OK;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

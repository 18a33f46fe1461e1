/*
 * qhap_oracle.c -- FP64 CPU oracle for the QHap phasing hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or constant generator with the CUDA library; it is deliberately plain
 * and slow: literal loops in the order and notation of the paper (QHap,
 * "Quantum-Inspired Haplotype Phasing", Methods), FP64 throughout.
 *
 * Citations are to the paper's Methods subsections and equations:
 *   Read-based: Matrix construction (Eq. M), Max-Cut graph construction
 *   (Eqs. delta, w_ab), SB algorithm solution (J = -A, Ising energy, Max-Cut
 *   identity), Consistency processing (vote counts c_l^(+/-)).
 *   SNP-based: Matrix construction (q~ = 1 - 10^(-Q/10), W = M o q~),
 *   Max-Cut graph construction (P_cis, P_trans, l_uv, Eq. edge_weight_SNP),
 *   SB algorithm solution (w' sign inversion, flip counter C, parity swap).
 *   Pore-C data support (alpha scaling).  SNP linkage depth analysis (k/10).
 * The bSB update itself is not printed in the paper (it cites the ballistic
 * simulated bifurcation literature); the oracle uses the standard bSB
 * equations of Goto et al. (Sci. Adv. 2021):
 *   y <- y + dt * ( -(a0 - a(t)) x + c0 J x ),  x <- x + dt * a0 * y,
 *   |x| > 1  =>  x <- sgn(x), y <- 0,  a(t) = a0 * t / steps.
 *
 * Parity pins (tests, without a GPU): hand-worked example graphs, closed-form
 * Max-Cut values, brute-force Max-Cut, an independent ODE integration of the
 * bSB dynamics, the closed-form LLR identity, planted truth partitions and the
 * paper's own switch/Hamming error example.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define QO_OK 0
#define QO_EINVAL 1
#define QO_ENOMEM 2

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the n-th output of a stream
 * with initial state `key` is mix(key + (n + 1) * gamma).                    */
static const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ULL;

static uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static uint64_t sm_out(uint64_t key, uint64_t n) { return sm_mix(key + (n + 1) * SM_GAMMA); }

/* Initial bSB state draw, uniform on [-0.1, 0.1] in 2^-24 steps.
 * Stream key  = output #((block << 16) | iter) of the stream seeded by `seed`;
 * draw index  = ((replica << 24) | node) * 2 + which   (which: 0 = x, 1 = y). */
double qo_init_value(uint64_t seed, int64_t block, int32_t iter, int32_t replica, int64_t node,
                     int which) {
  uint64_t key = sm_out(seed, ((uint64_t)block << 16) | (uint64_t)(uint32_t)iter);
  uint64_t v = sm_out(key, ((((uint64_t)replica) << 24) | (uint64_t)node) * 2u + (uint64_t)which);
  double u = (double)(v >> 40) * (1.0 / 16777216.0);
  return u * 0.2 - 0.1;
}

uint64_t qo_splitmix64(uint64_t key, uint64_t n) { return sm_out(key, n); }

/* ------------------------------------------------------------------------ */
/* Input validation shared by both graph builders (fragments are CSR).       */
static int check_fragments(int32_t m, int32_t n, const int64_t* fp, const int32_t* snp,
                           const int8_t* allele) {
  if (m < 0 || n < 0) return QO_EINVAL;
  if (fp[0] != 0) return QO_EINVAL;
  for (int32_t i = 0; i < m; ++i) {
    if (fp[i + 1] < fp[i]) return QO_EINVAL;
    for (int64_t e = fp[i]; e < fp[i + 1]; ++e) {
      if (snp[e] < 0 || snp[e] >= n) return QO_EINVAL;
      if (e > fp[i] && snp[e] <= snp[e - 1]) return QO_EINVAL;
      if (allele[e] != 1 && allele[e] != -1) return QO_EINVAL;
    }
  }
  return QO_OK;
}

/* ------------------------------------------------------------------------ */
/* Read graph (read-based Max-Cut graph construction).
 * mode 0 = CONFLICT: w_ab = sum_j 1[M_aj * M_bj = -1]            (Eqs. delta, w_ab)
 * mode 1 = SIGNED:   w_ab = sum_j -M_aj * M_bj  (= conflicts - agreements), i.e.
 *                    W = -M M^T with zero diagonal.
 * Literal pair loop over a < b, each pair walking the shared SNPs.
 * Output: dense symmetric m x m int64 matrix (row-major), zero diagonal.      */
int qo_read_graph_dense(int32_t m, int32_t n, const int64_t* fp, const int32_t* snp,
                        const int8_t* allele, int mode, int64_t* W) {
  int rc = check_fragments(m, n, fp, snp, allele);
  if (rc) return rc;
  if (mode != 0 && mode != 1) return QO_EINVAL;
  memset(W, 0, sizeof(int64_t) * (size_t)m * (size_t)m);
  for (int32_t a = 0; a < m; ++a) {
    for (int32_t b = a + 1; b < m; ++b) {
      int64_t ea = fp[a], eb = fp[b], w = 0;
      while (ea < fp[a + 1] && eb < fp[b + 1]) {
        if (snp[ea] < snp[eb]) {
          ++ea;
        } else if (snp[ea] > snp[eb]) {
          ++eb;
        } else {
          int prod = (int)allele[ea] * (int)allele[eb];
          if (mode == 0)
            w += (prod == -1) ? 1 : 0;
          else
            w += -prod;
          ++ea;
          ++eb;
        }
      }
      W[(size_t)a * m + b] = w;
      W[(size_t)b * m + a] = w;
    }
  }
  return QO_OK;
}

/* Same graph as CSR (both directions, only w != 0 entries, columns ascending).
 * Pairs whose SNP ranges cannot intersect are skipped before the walk (their
 * weight is zero by definition).  Arrays are malloc'ed; free with qo_free.    */
int64_t qo_read_graph_csr(int32_t m, int32_t n, const int64_t* fp, const int32_t* snp,
                          const int8_t* allele, int mode, int64_t** row_ptr, int32_t** col,
                          double** w) {
  if (check_fragments(m, n, fp, snp, allele)) return -QO_EINVAL;
  if (mode != 0 && mode != 1) return -QO_EINVAL;
  int64_t cap = 1024, nnz = 0;
  int32_t* ea_row = (int32_t*)malloc(sizeof(int32_t) * cap);
  int32_t* eb_col = (int32_t*)malloc(sizeof(int32_t) * cap);
  double* ew = (double*)malloc(sizeof(double) * cap);
  for (int32_t a = 0; a < m; ++a) {
    for (int32_t b = 0; b < m; ++b) {
      if (a == b || fp[a] == fp[a + 1] || fp[b] == fp[b + 1]) continue;
      if (snp[fp[a + 1] - 1] < snp[fp[b]] || snp[fp[b + 1] - 1] < snp[fp[a]]) continue;
      int64_t ea = fp[a], eb = fp[b], acc = 0;
      while (ea < fp[a + 1] && eb < fp[b + 1]) {
        if (snp[ea] < snp[eb]) {
          ++ea;
        } else if (snp[ea] > snp[eb]) {
          ++eb;
        } else {
          int prod = (int)allele[ea] * (int)allele[eb];
          acc += (mode == 0) ? (prod == -1 ? 1 : 0) : -prod;
          ++ea;
          ++eb;
        }
      }
      if (acc == 0) continue;
      if (nnz == cap) {
        cap *= 2;
        ea_row = (int32_t*)realloc(ea_row, sizeof(int32_t) * cap);
        eb_col = (int32_t*)realloc(eb_col, sizeof(int32_t) * cap);
        ew = (double*)realloc(ew, sizeof(double) * cap);
      }
      ea_row[nnz] = a;
      eb_col[nnz] = b;
      ew[nnz] = (double)acc;
      ++nnz;
    }
  }
  int64_t* rp = (int64_t*)calloc((size_t)m + 1, sizeof(int64_t));
  for (int64_t e = 0; e < nnz; ++e) rp[ea_row[e] + 1]++;
  for (int32_t a = 0; a < m; ++a) rp[a + 1] += rp[a];
  free(ea_row);
  *row_ptr = rp;
  *col = eb_col;
  *w = ew;
  return nnz;
}

/* ------------------------------------------------------------------------ */
/* SNP graph (SNP-based matrix and Max-Cut graph construction).
 *   q~ = 1 - 10^(-Q/10),  q_u = |W_iu|, q_v = |W_iv|
 *   P_cis   = q_u q_v + (1 - q_u)(1 - q_v)
 *   P_trans = q_u (1 - q_v) + (1 - q_u) q_v
 *   l_uv^(i) = sgn(W_iu W_iv) * log10(P_cis / P_trans)
 *   w_uv = - sum_{i in F_uv} alpha_i * l_uv^(i) / (|S_i| - 1)
 * alpha_i = porec_alpha for Pore-C fragments, 1 otherwise (Pore-C data support).
 * Linkage depth k/10: SNP at fragment position p links to the next
 * floor(k (|S_i| - 1) / 10) SNPs of the same fragment (linkage depth analysis).
 * Terms are accumulated per edge in fragment order.  The aggregation keeps a
 * list of (u, v, fragment, position) terms, orders it with qsort on that key
 * and sums each edge's run in order -- the same sequence of additions as a
 * dense accumulator updated fragment by fragment.
 * Output: CSR, both directions, columns ascending, every edge with at least
 * one contributing term (its weight may be exactly 0.0 only by cancellation). */
typedef struct {
  int32_t u, v;
  int32_t frag;
  int32_t pos;
  double term;
} qo_term;

static int term_cmp(const void* pa, const void* pb) {
  const qo_term* a = (const qo_term*)pa;
  const qo_term* b = (const qo_term*)pb;
  if (a->u != b->u) return a->u < b->u ? -1 : 1;
  if (a->v != b->v) return a->v < b->v ? -1 : 1;
  if (a->frag != b->frag) return a->frag < b->frag ? -1 : 1;
  if (a->pos != b->pos) return a->pos < b->pos ? -1 : 1;
  return 0;
}

int64_t qo_snp_graph_csr(int32_t m, int32_t n, const int64_t* fp, const int32_t* snp,
                         const int8_t* allele, const uint8_t* qual, const uint8_t* is_porec,
                         double porec_alpha, int linkage_k, int64_t** row_ptr, int32_t** col,
                         double** w) {
  if (check_fragments(m, n, fp, snp, allele)) return -QO_EINVAL;
  if (linkage_k < 1 || linkage_k > 10) return -QO_EINVAL;
  for (int64_t e = 0; e < fp[m]; ++e)
    if (qual[e] < 4 || qual[e] > 93) return -QO_EINVAL;
  int64_t cap = 0;
  for (int32_t i = 0; i < m; ++i) {
    int64_t s = fp[i + 1] - fp[i];
    cap += s * (s - 1); /* both directions */
  }
  qo_term* t = (qo_term*)malloc(sizeof(qo_term) * (size_t)(cap > 0 ? cap : 1));
  if (!t) return -QO_ENOMEM;
  int64_t nt = 0;
  for (int32_t i = 0; i < m; ++i) {
    int64_t S = fp[i + 1] - fp[i];
    if (S < 2) continue;
    double alpha = (is_porec && is_porec[i]) ? porec_alpha : 1.0;
    int64_t depth = ((int64_t)linkage_k * (S - 1)) / 10;
    for (int64_t p = 0; p < S; ++p) {
      for (int64_t pp = p + 1; pp < S && pp <= p + depth; ++pp) {
        int64_t eu = fp[i] + p, ev = fp[i] + pp;
        double qu = 1.0 - pow(10.0, -(double)qual[eu] / 10.0);
        double qv = 1.0 - pow(10.0, -(double)qual[ev] / 10.0);
        double Wiu = (double)allele[eu] * qu, Wiv = (double)allele[ev] * qv;
        double au = fabs(Wiu), av = fabs(Wiv);
        double pcis = au * av + (1.0 - au) * (1.0 - av);
        double ptrans = au * (1.0 - av) + (1.0 - au) * av;
        double sgn = (Wiu * Wiv > 0) ? 1.0 : -1.0;
        double l = sgn * log10(pcis / ptrans);
        double term = -(alpha * l) / (double)(S - 1);
        int32_t u = snp[eu], v = snp[ev];
        t[nt++] = (qo_term){u, v, i, (int32_t)p, term};
        t[nt++] = (qo_term){v, u, i, (int32_t)p, term};
      }
    }
  }
  qsort(t, (size_t)nt, sizeof(qo_term), term_cmp);
  int64_t* rp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* c = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nt > 0 ? nt : 1));
  double* ww = (double*)malloc(sizeof(double) * (size_t)(nt > 0 ? nt : 1));
  int64_t ne = 0;
  for (int64_t k = 0; k < nt;) {
    int64_t k2 = k;
    double acc = 0.0;
    while (k2 < nt && t[k2].u == t[k].u && t[k2].v == t[k].v) {
      acc += t[k2].term;
      ++k2;
    }
    rp[t[k].u + 1]++;
    c[ne] = t[k].v;
    ww[ne] = acc;
    ++ne;
    k = k2;
  }
  for (int32_t a = 0; a < n; ++a) rp[a + 1] += rp[a];
  free(t);
  *row_ptr = rp;
  *col = c;
  *w = ww;
  return ne;
}

void qo_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Connected components by breadth-first search over edges with w != 0
 * (both graph constructions, read graph and SNP graph: components are independent
 * subproblems; single-node components are excluded).
 * label[v] = component index, components numbered in order of their smallest
 * vertex.  Returns the number of components (singletons included).          */
int32_t qo_components(int32_t n, const int64_t* rp, const int32_t* col, const double* w,
                      int32_t* label) {
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t v = 0; v < n; ++v) label[v] = -1;
  int32_t nc = 0;
  for (int32_t s = 0; s < n; ++s) {
    if (label[s] >= 0) continue;
    int32_t head = 0, tail = 0;
    queue[tail++] = s;
    label[s] = nc;
    while (head < tail) {
      int32_t u = queue[head++];
      for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        if (w[e] == 0.0) continue;
        int32_t v = col[e];
        if (label[v] < 0) {
          label[v] = nc;
          queue[tail++] = v;
        }
      }
    }
    ++nc;
  }
  free(queue);
  return nc;
}

/* ------------------------------------------------------------------------ */
/* Simulated bifurcation on one component given as CSR of the coupling J (J = -A,
 * SB algorithm solution).  x, y: [R][n] row-major, updated in place from step t0
 * to t1-1 of a schedule of `steps` steps; each replica evolves independently.
 * Symplectic Euler as for bSB: y from x_t, then x from y_{t+1}; a(t) = a0 t / steps.
 * The paper compares three SB variants and cites their standard formulations:
 *   variant 0, ballistic (bSB):  y += dt (-(a0 - a(t)) x + c0 J x); x += dt a0 y;
 *                                |x| > 1 => x = sgn(x), y = 0
 *   variant 1, discrete (dSB):   as bSB with J sgn(x) in place of J x
 *                                (sgn(0) = +1, as for the spins)
 *   variant 2, adiabatic (aSB):  y += dt (-(x^2 + a0 - a(t)) x + c0 J x);
 *                                x += dt a0 y; no walls                        */
void qo_sb_run_h(int32_t n, const int64_t* rp, const int32_t* col, const double* J, int32_t R,
                 double* x, double* y, int32_t t0, int32_t t1, int32_t steps, double dt, double a0,
                 double c0, int32_t variant, double h, const double* hdir);

void qo_sb_run(int32_t n, const int64_t* rp, const int32_t* col, const double* J, int32_t R,
               double* x, double* y, int32_t t0, int32_t t1, int32_t steps, double dt, double a0,
               double c0, int32_t variant) {
  qo_sb_run_h(n, rp, col, J, R, x, y, t0, t1, steps, dt, a0, c0, variant, 0.0, NULL);
}

/* The same with the deformation term of the SNP refinement's adaptive strategy (SB
 * algorithm solution, SNP-based method: a term h added to escape local minima when
 * the cut stays negative; the paper gives no formula).  Reading used here: a field
 * along a direction d (d_i in {-1, +1}; NULL = all +1) whose strength falls linearly
 * to zero over the schedule, added to the force on y:
 *     y_i += dt (... + h (1 - t / steps) d_i)
 * so the landscape is tilted toward d early and is the undeformed one at the end. */
void qo_sb_run_h(int32_t n, const int64_t* rp, const int32_t* col, const double* J, int32_t R,
                 double* x, double* y, int32_t t0, int32_t t1, int32_t steps, double dt, double a0,
                 double c0, int32_t variant, double h, const double* hdir) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t r = 0; r < R; ++r) {
    double* xr = x + (size_t)r * n;
    double* yr = y + (size_t)r * n;
    double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int32_t t = t0; t < t1; ++t) {
      double at = a0 * (double)t / (double)steps;
      for (int32_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
          double xj = xr[col[e]];
          if (variant == 1) xj = xj >= 0.0 ? 1.0 : -1.0;
          acc += J[e] * xj;
        }
        z[i] = acc;
      }
      double ht = h * (1.0 - (double)t / (double)steps);
      for (int32_t i = 0; i < n; ++i) {
        double detune = a0 - at;
        if (variant == 2) detune += xr[i] * xr[i];
        double field = ht * (hdir ? hdir[i] : 1.0);
        yr[i] += dt * (-detune * xr[i] + c0 * z[i] + field);
      }
      for (int32_t i = 0; i < n; ++i) xr[i] += dt * a0 * yr[i];
      if (variant != 2)
        for (int32_t i = 0; i < n; ++i) {
          if (fabs(xr[i]) > 1.0) {
            xr[i] = xr[i] > 0 ? 1.0 : -1.0;
            yr[i] = 0.0;
          }
        }
    }
    free(z);
  }
}

void qo_bsb_run(int32_t n, const int64_t* rp, const int32_t* col, const double* J, int32_t R,
                double* x, double* y, int32_t t0, int32_t t1, int32_t steps, double dt, double a0,
                double c0) {
  qo_sb_run(n, rp, col, J, R, x, y, t0, t1, steps, dt, a0, c0, 0);
}

/* Initial state for replicas replica_ids[0..R-1] of component `block`.       */
void qo_bsb_init(int32_t n, int32_t R, const int32_t* replica_ids, uint64_t seed, int64_t block,
                 int32_t iter, double* x, double* y) {
  for (int32_t r = 0; r < R; ++r)
    for (int32_t i = 0; i < n; ++i) {
      x[(size_t)r * n + i] = qo_init_value(seed, block, iter, replica_ids[r], i, 0);
      y[(size_t)r * n + i] = qo_init_value(seed, block, iter, replica_ids[r], i, 1);
    }
}

/* Default c0 = 0.5 / (sigma * sqrt(N)), sigma^2 = sum_{a != b} J_ab^2 / (N (N - 1)). */
double qo_default_c0(int32_t n, const int64_t* rp, const double* J) {
  double s2 = 0.0;
  for (int32_t i = 0; i < n; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s2 += J[e] * J[e];
  if (n < 2 || s2 == 0.0) return 0.0;
  double sigma = sqrt(s2 / ((double)n * (double)(n - 1)));
  return 0.5 / (sigma * sqrt((double)n));
}

/* Cut value sum_{a<b} w_ab 1[s_a != s_b] of spins s in {-1,+1} (Max-Cut objective). */
double qo_cut(int32_t n, const int64_t* rp, const int32_t* col, const double* w,
              const int8_t* s) {
  double cut = 0.0;
  for (int32_t a = 0; a < n; ++a)
    for (int64_t e = rp[a]; e < rp[a + 1]; ++e) {
      int32_t b = col[e];
      if (b > a && s[a] != s[b]) cut += w[e];
    }
  return cut;
}

/* Ising energy E(s) = -1/2 s^T J s. */
double qo_ising_energy(int32_t n, const int64_t* rp, const int32_t* col, const double* J,
                       const int8_t* s) {
  double e = 0.0;
  for (int32_t a = 0; a < n; ++a)
    for (int64_t k = rp[a]; k < rp[a + 1]; ++k) e += (double)s[a] * J[k] * (double)s[col[k]];
  return -0.5 * e;
}

/* Full multi-replica bSB on one component with weights w (J = -w): returns the
 * best replica's spins (s = sgn(x), sgn(0) = +1), its cut, and every replica's
 * cut.  Ties between replicas go to the lowest replica index.               */
double qo_sb_solve_h(int32_t n, const int64_t* rp, const int32_t* col, const double* w, int32_t R,
                     const int32_t* replica_ids, int32_t steps, double dt, double a0, double c0,
                     uint64_t seed, int64_t block, int32_t iter, int8_t* best_s, double* cuts,
                     int32_t* best_r, int32_t variant, double h);

double qo_sb_solve(int32_t n, const int64_t* rp, const int32_t* col, const double* w, int32_t R,
                   const int32_t* replica_ids, int32_t steps, double dt, double a0, double c0,
                   uint64_t seed, int64_t block, int32_t iter, int8_t* best_s, double* cuts,
                   int32_t* best_r, int32_t variant) {
  return qo_sb_solve_h(n, rp, col, w, R, replica_ids, steps, dt, a0, c0, seed, block, iter,
                       best_s, cuts, best_r, variant, 0.0);
}

/* qo_sb_solve with the deformation field of strength h along +1 on every vertex (the
 * incumbent partition in the refinement's gauged frame). */
double qo_sb_solve_h(int32_t n, const int64_t* rp, const int32_t* col, const double* w, int32_t R,
                     const int32_t* replica_ids, int32_t steps, double dt, double a0, double c0,
                     uint64_t seed, int64_t block, int32_t iter, int8_t* best_s, double* cuts,
                     int32_t* best_r, int32_t variant, double h) {
  int64_t nnz = rp[n];
  double* J = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  for (int64_t e = 0; e < nnz; ++e) J[e] = -w[e];
  if (c0 <= 0.0) c0 = qo_default_c0(n, rp, J);
  double* x = (double*)malloc(sizeof(double) * (size_t)R * (size_t)(n > 0 ? n : 1));
  double* y = (double*)malloc(sizeof(double) * (size_t)R * (size_t)(n > 0 ? n : 1));
  int8_t* s = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
  qo_bsb_init(n, R, replica_ids, seed, block, iter, x, y);
  qo_sb_run_h(n, rp, col, J, R, x, y, 0, steps, steps, dt, a0, c0, variant, h, NULL);
  double best = -INFINITY;
  *best_r = -1;
  for (int32_t r = 0; r < R; ++r) {
    for (int32_t i = 0; i < n; ++i) s[i] = (x[(size_t)r * n + i] >= 0.0) ? 1 : -1;
    double c = qo_cut(n, rp, col, w, s);
    cuts[r] = c;
    if (c > best) {
      best = c;
      *best_r = r;
      memcpy(best_s, s, (size_t)n);
    }
  }
  free(J);
  free(x);
  free(y);
  free(s);
  return best;
}

double qo_bsb_solve(int32_t n, const int64_t* rp, const int32_t* col, const double* w, int32_t R,
                    const int32_t* replica_ids, int32_t steps, double dt, double a0, double c0,
                    uint64_t seed, int64_t block, int32_t iter, int8_t* best_s, double* cuts,
                    int32_t* best_r) {
  return qo_sb_solve(n, rp, col, w, R, replica_ids, steps, dt, a0, c0, seed, block, iter, best_s,
                     cuts, best_r, 0);
}

/* Multi-replica SB with early stop on energy stagnation.  The paper caps its runs by
 * a "maximum convergence count"; the reading used here is a patience on the best
 * energy over replicas:
 *   every check_every steps, while the schedule still has steps left (t < steps),
 *   each replica's spins s = sgn(x) are cut-evaluated and the best cut over the
 *   replicas is compared with the best of all earlier checks of this solve;
 *   a strictly larger value resets the stall count, any other adds one;
 *   when the stall count reaches `patience` the solve stops after t steps.
 * The replicas' state is then the state after t steps of the `steps`-step schedule
 * (a(t) keeps its full-schedule definition), and the result is evaluated from it as in
 * qo_sb_solve.  check_every = 0 or patience = 0: no early stop.  *steps_run receives
 * the number of steps made.
 * track_best != 0 (the best value reached during the run, Results): the result is the
 * best cut over the replicas at any check or at the end, with its replica and spins;
 * ties keep the earliest check (the end counts as the last) and the lowest replica.
 * cuts[] stays the final state's.  Checks then run every check_every steps even when
 * patience = 0 (no early stop).                                                      */
double qo_sb_solve_es(int32_t n, const int64_t* rp, const int32_t* col, const double* w,
                      int32_t R, const int32_t* replica_ids, int32_t steps, double dt, double a0,
                      double c0, uint64_t seed, int64_t block, int32_t iter, int32_t check_every,
                      int32_t patience, int8_t* best_s, double* cuts, int32_t* best_r,
                      int32_t* steps_run, int32_t variant, int32_t track_best) {
  int64_t nnz = rp[n];
  double* J = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  for (int64_t e = 0; e < nnz; ++e) J[e] = -w[e];
  if (c0 <= 0.0) c0 = qo_default_c0(n, rp, J);
  double* x = (double*)malloc(sizeof(double) * (size_t)R * (size_t)(n > 0 ? n : 1));
  double* y = (double*)malloc(sizeof(double) * (size_t)R * (size_t)(n > 0 ? n : 1));
  int8_t* s = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
  /* best during the run (track_best): its cut, replica and spins, over the checks */
  int8_t* kept_s = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
  double kept = -INFINITY;
  int32_t kept_r = -1;
  qo_bsb_init(n, R, replica_ids, seed, block, iter, x, y);
  int32_t t = 0;
  if (check_every > 0 && (patience > 0 || track_best)) {
    double seen = -INFINITY;
    int32_t stall = 0;
    while (t < steps) {
      int32_t t1 = t + check_every < steps ? t + check_every : steps;
      qo_sb_run(n, rp, col, J, R, x, y, t, t1, steps, dt, a0, c0, variant);
      t = t1;
      if (t >= steps) break; /* no check once the schedule is complete */
      double best_now = -INFINITY;
      for (int32_t r = 0; r < R; ++r) {
        for (int32_t i = 0; i < n; ++i) s[i] = (x[(size_t)r * n + i] >= 0.0) ? 1 : -1;
        double c = qo_cut(n, rp, col, w, s);
        if (c > best_now) best_now = c;
        if (track_best && c > kept) { /* strictly better: ties keep the earlier */
          kept = c;
          kept_r = r;
          memcpy(kept_s, s, (size_t)n);
        }
      }
      if (patience <= 0) continue; /* checks for track_best only */
      if (best_now > seen) {
        seen = best_now;
        stall = 0;
      } else if (++stall >= patience) {
        break;
      }
    }
  } else {
    qo_sb_run(n, rp, col, J, R, x, y, 0, steps, steps, dt, a0, c0, variant);
    t = steps;
  }
  *steps_run = t;
  double best = -INFINITY;
  *best_r = -1;
  for (int32_t r = 0; r < R; ++r) {
    for (int32_t i = 0; i < n; ++i) s[i] = (x[(size_t)r * n + i] >= 0.0) ? 1 : -1;
    double c = qo_cut(n, rp, col, w, s);
    cuts[r] = c;
    if (c > best) {
      best = c;
      *best_r = r;
      memcpy(best_s, s, (size_t)n);
    }
  }
  /* the final state is the last check: an earlier check keeps the result unless the
     final best is strictly better */
  if (track_best && kept_r >= 0 && kept >= best) {
    best = kept;
    *best_r = kept_r;
    memcpy(best_s, kept_s, (size_t)n);
  }
  free(J);
  free(x);
  free(y);
  free(s);
  free(kept_s);
  return best;
}

/* ------------------------------------------------------------------------ */
/* SNP-based iterative refinement (SB algorithm solution, SNP-based method).
 * Repeat up to refine_max times: solve with bSB; stop if the cut is <= 0 or
 * every vertex lies in one subset; otherwise C(p) += 1 for p in the smaller
 * subset (tie: the subset without the lowest-index vertex) and invert the
 * sign of every edge crossing the partition (w' = -w if s_u != s_v).
 * w is modified in place (the final gauged weights).  Returns iterations done. */
int32_t qo_refine_v(int32_t n, const int64_t* rp, const int32_t* col, double* w, int32_t R,
                    const int32_t* replica_ids, int32_t steps, double dt, double a0, double c0,
                    uint64_t seed, int64_t block, int32_t refine_max, int32_t* C,
                    double* first_cut, double deform_h, int32_t deform_tries, int32_t* solves,
                    int32_t variant);

int32_t qo_refine_h(int32_t n, const int64_t* rp, const int32_t* col, double* w, int32_t R,
                    const int32_t* replica_ids, int32_t steps, double dt, double a0, double c0,
                    uint64_t seed, int64_t block, int32_t refine_max, int32_t* C,
                    double* first_cut, double deform_h, int32_t deform_tries, int32_t* solves) {
  return qo_refine_v(n, rp, col, w, R, replica_ids, steps, dt, a0, c0, seed, block, refine_max,
                     C, first_cut, deform_h, deform_tries, solves, 0);
}

int32_t qo_refine(int32_t n, const int64_t* rp, const int32_t* col, double* w, int32_t R,
                  const int32_t* replica_ids, int32_t steps, double dt, double a0, double c0,
                  uint64_t seed, int64_t block, int32_t refine_max, int32_t* C,
                  double* first_cut) {
  return qo_refine_h(n, rp, col, w, R, replica_ids, steps, dt, a0, c0, seed, block, refine_max,
                     C, first_cut, 0.0, 0, NULL);
}

/* The refinement with the adaptive deformation (reading of the SNP-based method's
 * adaptive parameter strategy): when a solve ends with a cut <= 0 or with every
 * vertex in one subset, and fewer than deform_tries re-solves have been made since the
 * last accepted partition, the component is solved again with the deformation field
 * along the incumbent (all +1 in the gauged frame), of strength deform_h 2^(k-1) on
 * the k-th re-solve; a positive cut is then accepted as usual.  Every solve, plain or
 * deformed, counts toward refine_max and draws its initial state with its own
 * iteration index.  Returns the number of accepted partitions; *solves (if not NULL)
 * receives the number of solves.  variant: the SB variant of every solve (0 = bSB,
 * the paper's solver; 1 = dSB, 2 = aSB as in qo_sb_run).                           */
int32_t qo_refine_v(int32_t n, const int64_t* rp, const int32_t* col, double* w, int32_t R,
                    const int32_t* replica_ids, int32_t steps, double dt, double a0, double c0,
                    uint64_t seed, int64_t block, int32_t refine_max, int32_t* C,
                    double* first_cut, double deform_h, int32_t deform_tries, int32_t* solves,
                    int32_t variant) {
  int8_t* s = (int8_t*)malloc((size_t)(n > 0 ? n : 1));
  double* cuts = (double*)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1));
  int32_t it = 0, accepted = 0, tries = 0;
  for (int32_t v = 0; v < n; ++v) C[v] = 0;
  for (it = 0; it < refine_max; ++it) {
    int32_t br;
    double h = tries == 0 ? 0.0 : deform_h * ldexp(1.0, tries - 1);
    double cut = qo_sb_solve_h(n, rp, col, w, R, replica_ids, steps, dt, a0, c0, seed, block, it,
                               s, cuts, &br, variant, h);
    if (it == 0 && first_cut) *first_cut = cut;
    int32_t n_pos = 0;
    for (int32_t v = 0; v < n; ++v) n_pos += (s[v] > 0);
    if (cut <= 0.0 || n_pos == 0 || n_pos == n) {
      if (deform_h > 0.0 && tries < deform_tries) {
        ++tries;
        continue;
      }
      ++it;
      break;
    }
    tries = 0;
    ++accepted;
    int8_t small;
    if (n_pos * 2 < n)
      small = 1;
    else if (n_pos * 2 > n)
      small = -1;
    else
      small = (int8_t)(-s[0]);
    for (int32_t v = 0; v < n; ++v)
      if (s[v] == small) C[v] += 1;
    for (int32_t a = 0; a < n; ++a)
      for (int64_t e = rp[a]; e < rp[a + 1]; ++e)
        if (s[a] != s[col[e]]) w[e] = -w[e];
  }
  if (solves) *solves = it;
  free(s);
  free(cuts);
  return accepted;
}

/* ------------------------------------------------------------------------ */
/* Read-based consistency processing (voting).
 * read_spin[i]  : +1 (S_1), -1 (S_2) or 0 (read not in a phased block)
 * read_block[i] : component index of read i, -1 if none
 * Each SNP is voted on by the block holding the most reads that cover it
 * (ties: lowest block index).  With d_l = c_l^(+) - c_l^(-):
 *   unphased if no coverage or d_1 = d_2 = 0;
 *   opposing majorities: S_1 takes sign(d_1);
 *   otherwise the subset with the larger |d_l| keeps its majority allele
 *   (tie: S_1) and the other takes the complement.
 * hap1[j] = haplotype of S_1 at SNP j: +1 (initial-H1 allele), -1 (initial-H2
 * allele), 0 unphased; snp_block[j] = voting block or -1.                    */
void qo_vote(int32_t m, int32_t n, const int64_t* fp, const int32_t* snp, const int8_t* allele,
             const int8_t* read_spin, const int32_t* read_block, int32_t n_blocks, int8_t* hap1,
             int32_t* snp_block) {
  int32_t* cover = (int32_t*)calloc((size_t)(n_blocks > 0 ? n_blocks : 1), sizeof(int32_t));
  /* SNP -> covering reads, in read order (transpose of the fragment CSR). */
  int64_t* cp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  for (int64_t e = 0; e < fp[m]; ++e) cp[snp[e] + 1]++;
  for (int32_t j = 0; j < n; ++j) cp[j + 1] += cp[j];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  memcpy(fill, cp, sizeof(int64_t) * ((size_t)n + 1));
  int32_t* crd = (int32_t*)malloc(sizeof(int32_t) * (size_t)(fp[m] > 0 ? fp[m] : 1));
  int8_t* cal = (int8_t*)malloc((size_t)(fp[m] > 0 ? fp[m] : 1));
  for (int32_t i = 0; i < m; ++i)
    for (int64_t e = fp[i]; e < fp[i + 1]; ++e) {
      crd[fill[snp[e]]] = i;
      cal[fill[snp[e]]] = allele[e];
      fill[snp[e]]++;
    }
  for (int32_t j = 0; j < n; ++j) {
    hap1[j] = 0;
    snp_block[j] = -1;
    int32_t best = -1, bestc = 0;
    for (int64_t k = cp[j]; k < cp[j + 1]; ++k)
      if (read_block[crd[k]] >= 0) cover[read_block[crd[k]]]++;
    for (int64_t k = cp[j]; k < cp[j + 1]; ++k) {
      int32_t b = read_block[crd[k]];
      if (b < 0) continue;
      if (cover[b] > bestc || (cover[b] == bestc && b < best)) {
        bestc = cover[b];
        best = b;
      }
    }
    for (int64_t k = cp[j]; k < cp[j + 1]; ++k)
      if (read_block[crd[k]] >= 0) cover[read_block[crd[k]]] = 0;
    if (best < 0) continue;
    int32_t c1p = 0, c1m = 0, c2p = 0, c2m = 0;
    for (int64_t k = cp[j]; k < cp[j + 1]; ++k) {
      int32_t i = crd[k];
      if (read_block[i] != best) continue;
      if (read_spin[i] > 0) {
        if (cal[k] > 0) c1p++; else c1m++;
      } else if (read_spin[i] < 0) {
        if (cal[k] > 0) c2p++; else c2m++;
      }
    }
    int32_t d1 = c1p - c1m, d2 = c2p - c2m;
    if (c1p + c1m + c2p + c2m == 0 || (d1 == 0 && d2 == 0)) continue;
    int8_t h;
    if ((d1 > 0 && d2 < 0) || (d1 < 0 && d2 > 0)) {
      h = d1 > 0 ? 1 : -1;
    } else {
      int32_t a1 = d1 < 0 ? -d1 : d1, a2 = d2 < 0 ? -d2 : d2;
      if (a1 >= a2)
        h = d1 > 0 ? 1 : -1;
      else
        h = d2 > 0 ? -1 : 1;
    }
    hap1[j] = h;
    snp_block[j] = best;
  }
  free(cover);
  free(cp);
  free(fill);
  free(crd);
  free(cal);
}

/* SNP-based reconstruction: (H1'[u], H2'[u]) swapped where C(p_u) is odd.
 * hap1[u] = +1 keeps the initial-H1 allele on H1', -1 swaps; 0 where the SNP is
 * in no phased block (in_block[u] == 0).                                      */
void qo_parity(int32_t n, const int32_t* C, const uint8_t* in_block, int8_t* hap1) {
  for (int32_t u = 0; u < n; ++u) hap1[u] = in_block[u] ? ((C[u] % 2 == 0) ? 1 : -1) : 0;
}

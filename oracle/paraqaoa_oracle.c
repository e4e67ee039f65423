/*
 * ParaQAOA CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision restatement of what the method computes,
 * used to check the CUDA path. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code with the CUDA
 * library and includes none of its headers.
 *
 * Every function follows one passage of the paper (arXiv 2603.26232):
 *   Sec. 2.1        Max-Cut objective CutVal
 *   Sec. 2.2        QAOA ansatz |psi> = prod_l U_M(beta_l) U_C(gamma_l) |+>^n,
 *                   U_C = exp(-i gamma H_C), U_M = exp(-i beta H_M),
 *                   H_M = sum_j X_j (transverse field), H_C = C(z) (cut value)
 *   Sec. 3.2, Alg. 1  Connectivity-Preserving Partitioning and GetSubgraph
 *   Sec. 3.3.2      Selective Distribution Exploration (top-K)
 *   Sec. 3.4, Alg. 2  Level-Aware Parallel Merge (exhaustive DFS), plus a
 *                   beam reading of it for product spaces too large to walk
 *
 * Conventions: bit j of a bitstring z is local vertex j of the subgraph (the
 * j-th smallest global index in V_i); z_j = 1 puts the vertex in S.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -4
#define OR_ESEARCH -5

/* ------------------------------------------------------------------ */
/* Sec. 2.1: CutVal(S, S-bar) = sum of w_ij over edges with i in S, j not. */

/* Cut value of a subgraph assignment z over an explicit edge list. */
static int64_t cut_of(uint64_t z, int64_t m, const int32_t *eu, const int32_t *ev,
                      const int32_t *ew) {
  int64_t c = 0;
  for (int64_t e = 0; e < m; e++) {
    int bu = (int)((z >> eu[e]) & 1u);
    int bv = (int)((z >> ev[e]) & 1u);
    if (bu != bv) c += ew[e];
  }
  return c;
}

/* Cut value of a full-graph assignment (side[v] in {0,1}) over a symmetric CSR;
 * each undirected edge is stored twice, so count it from its smaller end. */
int64_t or_cutval(int32_t nv, const int64_t *row_ptr, const int32_t *col,
                  const int32_t *w, const uint8_t *side) {
  int64_t c = 0;
  for (int32_t u = 0; u < nv; u++)
    for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++) {
      int32_t v = col[k];
      if (u < v && side[u] != side[v]) c += w[k];
    }
  return c;
}

/* Cut table C(z) for every z in [0, 2^n), straight from the definition. */
void or_cut_table(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                  const int32_t *ew, int64_t *out) {
  uint64_t dim = 1ull << n;
  for (uint64_t z = 0; z < dim; z++) out[z] = cut_of(z, m, eu, ev, ew);
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2, Alg. 1: partitioning. Three readings (see the design notes):
 *   mode 0 BALANCED: the |V|-1 steps between consecutive parts' first
 *     vertices are split as evenly as possible, larger steps first; part i
 *     covers [o_i, o_i + t_i], so neighbours share exactly one vertex.
 *   mode 1 ALG1_LITERAL: s = floor(|V|/M) - 1, part i (1-based) covers
 *     [(i-1)s, (i-1)s + s + 1), the last part runs to |V|.
 *   mode 2 SIZES: explicit sizes, sum(sizes) - (M-1) = |V|.
 * Output: first vertex and size of each part. */
int or_partition(int32_t nv, int32_t M, int32_t mode, const int32_t *sizes,
                 int32_t *out_first, int32_t *out_size) {
  if (nv < 1 || M < 1) return OR_EINVAL;
  if (mode == 0) {
    if (M > 1 && nv - 1 < M) return OR_EINVAL;
    if (M == 1) {
      out_first[0] = 0;
      out_size[0] = nv;
      return OR_OK;
    }
    int32_t q = (nv - 1) / M, r = (nv - 1) % M, o = 0;
    for (int32_t i = 0; i < M; i++) {
      int32_t t = q + (i < r ? 1 : 0);
      out_first[i] = o;
      out_size[i] = t + 1;
      o += t;
    }
    return OR_OK;
  }
  if (mode == 1) {
    int32_t s = nv / M - 1;
    if (s < 1 && M > 1) return OR_EINVAL;
    for (int32_t i = 1; i <= M; i++) {
      int32_t start = (i - 1) * s;
      int32_t end = (i == M) ? nv : start + s + 1;
      out_first[i - 1] = start;
      out_size[i - 1] = end - start;
    }
    return OR_OK;
  }
  if (mode == 2) {
    int64_t tot = 0;
    for (int32_t i = 0; i < M; i++) {
      if (sizes[i] < 1 || (M > 1 && sizes[i] < 2)) return OR_EINVAL;
      tot += sizes[i];
    }
    if (tot - (M - 1) != nv) return OR_EINVAL;
    int32_t o = 0;
    for (int32_t i = 0; i < M; i++) {
      out_first[i] = o;
      out_size[i] = sizes[i];
      o += sizes[i] - 1;
    }
    return OR_OK;
  }
  return OR_EINVAL;
}

/* GetSubgraph (Alg. 1): every edge (u, v) of E with both ends in
 * V_i = [first, first + size) becomes a local edge (u - first, v - first).
 * Edges are visited in CSR order from their smaller end, so the output is
 * sorted by (u, v). Returns the number of edges written (or, when out_u is
 * NULL, only counts them). */
int64_t or_get_subgraph(int32_t nv, const int64_t *row_ptr, const int32_t *col,
                        const int32_t *w, int32_t first, int32_t size, int32_t *out_u,
                        int32_t *out_v, int32_t *out_w) {
  int64_t cnt = 0;
  for (int32_t u = 0; u < nv; u++)
    for (int64_t k = row_ptr[u]; k < row_ptr[u + 1]; k++) {
      int32_t v = col[k];
      if (u < v && u >= first && u < first + size && v >= first && v < first + size) {
        if (out_u) {
          out_u[cnt] = u - first;
          out_v[cnt] = v - first;
          out_w[cnt] = w[k];
        }
        cnt++;
      }
    }
  return cnt;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2: state-vector simulation in complex128, literal gate order.
 * Layer l: the diagonal cost unitary psi_z <- exp(-i gamma_l C(z)) psi_z,
 * then exp(-i beta_l X_j) on every qubit j = 0..n-1, which maps the pair
 * (a, b) = (psi_{z with bit j = 0}, psi_{z with bit j = 1}) to
 * (cos(beta) a - i sin(beta) b, cos(beta) b - i sin(beta) a). */
static void simulate_one(int32_t n, const int64_t *cut, int32_t p, const double *gamma,
                         const double *beta, double complex *psi) {
  uint64_t dim = 1ull << n;
  double amp0 = 1.0 / sqrt((double)dim);
  for (uint64_t z = 0; z < dim; z++) psi[z] = amp0;
  for (int32_t l = 0; l < p; l++) {
    for (uint64_t z = 0; z < dim; z++) psi[z] *= cexp(-I * gamma[l] * (double)cut[z]);
    double c = cos(beta[l]), s = sin(beta[l]);
    for (int32_t j = 0; j < n; j++) {
      uint64_t bit = 1ull << j;
      for (uint64_t z = 0; z < dim; z++) {
        if (z & bit) continue;
        double complex a = psi[z], b = psi[z | bit];
        psi[z] = c * a - I * s * b;
        psi[z | bit] = c * b - I * s * a;
      }
    }
  }
}

/* <C> = sum_z |psi_z|^2 C(z), Kahan-compensated. */
static double expect_one(int32_t n, const double complex *psi, const int64_t *cut) {
  uint64_t dim = 1ull << n;
  double s = 0.0, comp = 0.0;
  for (uint64_t z = 0; z < dim; z++) {
    double pz = creal(psi[z]) * creal(psi[z]) + cimag(psi[z]) * cimag(psi[z]);
    double y = pz * (double)cut[z] - comp;
    double t = s + y;
    comp = (t - s) - y;
    s = t;
  }
  return s;
}

/* Simulate one subgraph; the state is written interleaved (re, im). */
int or_simulate(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                const int32_t *ew, int32_t p, const double *gamma, const double *beta,
                double *out_state) {
  if (n < 1 || n > 30 || p < 0) return OR_EINVAL;
  uint64_t dim = 1ull << n;
  int64_t *cut = (int64_t *)malloc(sizeof(int64_t) * dim);
  if (!cut) return OR_ENOMEM;
  or_cut_table(n, m, eu, ev, ew, cut);
  simulate_one(n, cut, p, gamma, beta, (double complex *)out_state);
  free(cut);
  return OR_OK;
}

double or_expect_state(int32_t n, const double *state, const int64_t *cut) {
  return expect_one(n, (const double complex *)state, cut);
}

/* <C> for a batch of (subgraph, angle) instances. Instance i uses subgraph
 * sub[i] (edge list slice [edge_off[sub[i]], edge_off[sub[i]+1]) with n =
 * nq[sub[i]]) and angles gamma[i*p .. i*p+p), beta[i*p ..]. Instances are
 * independent; OpenMP only spreads them over cores. */
int or_expect_batch(int32_t num_sub, const int32_t *nq, const int64_t *edge_off,
                    const int32_t *eu, const int32_t *ev, const int32_t *ew,
                    int32_t count, const int32_t *sub, int32_t p, const double *gamma,
                    const double *beta, double *out) {
  int err = OR_OK;
  for (int32_t i = 0; i < count; i++)
    if (sub[i] < 0 || sub[i] >= num_sub || nq[sub[i]] < 1 || nq[sub[i]] > 30) return OR_EINVAL;
#pragma omp parallel for schedule(dynamic, 1)
  for (int32_t i = 0; i < count; i++) {
    int32_t s = sub[i], n = nq[s];
    uint64_t dim = 1ull << n;
    int64_t *cut = (int64_t *)malloc(sizeof(int64_t) * dim);
    double complex *psi = (double complex *)malloc(sizeof(double complex) * dim);
    if (!cut || !psi) {
      free(cut);
      free(psi);
#pragma omp atomic write
      err = OR_ENOMEM;
      continue;
    }
    int64_t e0 = edge_off[s], m = edge_off[s + 1] - e0;
    or_cut_table(n, m, eu + e0, ev + e0, ew + e0, cut);
    simulate_one(n, cut, p, gamma + (int64_t)i * p, beta + (int64_t)i * p, psi);
    out[i] = expect_one(n, psi, cut);
    free(cut);
    free(psi);
  }
  return err;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3.2: the K most probable bitstrings. Canonical mode keeps only z
 * with bit n-1 = 0 (the state satisfies P(z) = P(not z), so the other half
 * repeats it); raw mode ranks all z. Key: probability descending, then z
 * ascending. Probabilities are compared in double precision here. */
typedef struct {
  double p;
  uint32_t z;
} pz_t;

static int cmp_pz(const void *a, const void *b) {
  const pz_t *x = (const pz_t *)a, *y = (const pz_t *)b;
  if (x->p > y->p) return -1;
  if (x->p < y->p) return 1;
  return (x->z < y->z) ? -1 : (x->z > y->z);
}

int or_topk(int32_t n, const double *state, int32_t K, int32_t canonical,
            uint32_t *out_z, double *out_p) {
  if (n < 1 || n > 30 || K < 1) return OR_EINVAL;
  uint64_t dim = 1ull << n;
  uint64_t cnt = canonical ? (dim >> 1) : dim;
  if (n == 1 && canonical) cnt = 1;
  if ((uint64_t)K > cnt) return OR_EINVAL;
  pz_t *arr = (pz_t *)malloc(sizeof(pz_t) * cnt);
  if (!arr) return OR_ENOMEM;
  for (uint64_t z = 0; z < cnt; z++) {
    double re = state[2 * z], im = state[2 * z + 1];
    arr[z].p = re * re + im * im;
    arr[z].z = (uint32_t)z;
  }
  qsort(arr, cnt, sizeof(pz_t), cmp_pz);
  for (int32_t k = 0; k < K; k++) {
    out_z[k] = arr[k].z;
    out_p[k] = arr[k].p;
  }
  free(arr);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Brute-force Max-Cut of a small graph: the best of all 2^(n-1)
 * assignments with vertex n-1 on side 0 (a cut and its complement are the
 * same cut). Returns the optimum; the first optimal z (ascending) goes to
 * *best_z. */
int64_t or_bruteforce_maxcut(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                             const int32_t *ew, uint32_t *best_z) {
  if (n < 1 || n > 32) return -1;
  uint64_t half = (n == 1) ? 1 : (1ull << (n - 1));
  int64_t best = -1;
  uint64_t arg = 0;
  for (uint64_t z = 0; z < half; z++) {
    int64_t c = cut_of(z, m, eu, ev, ew);
    if (c > best) {
      best = c;
      arg = z;
    }
  }
  if (best_z) *best_z = (uint32_t)arg;
  return best;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.4: merge. Parts are contiguous ranges [first_i, first_i + size_i)
 * with first_{i+1} = first_i + size_i - 1 (one shared vertex). A path picks
 * candidate j_i of part i. Part 1's bitstring is used as is; for i > 1 the
 * candidate or its complement is taken so that its bit 0 (the shared vertex)
 * agrees with the side already given to that vertex (the compatibility rule
 * of Sec. 3.4.1 that halves the 2K choices per level to K). */

typedef struct {
  int32_t nv, M, K;
  const int64_t *row_ptr;
  const int32_t *col, *w;
  const int32_t *first, *size;
  const uint32_t *cand;
} merge_in_t;

/* Assign the vertices of part `lvl` from candidate j, oriented to the path. */
static void assign_part(const merge_in_t *in, int32_t lvl, int32_t j, uint8_t *side) {
  int32_t f = in->first[lvl], s = in->size[lvl];
  uint32_t b = in->cand[(int64_t)lvl * in->K + j];
  uint32_t mask = (s >= 32) ? 0xFFFFFFFFu : ((1u << s) - 1u);
  if (lvl > 0 && (int)(b & 1u) != side[f]) b = (~b) & mask;
  for (int32_t v = 0; v < s; v++) side[f + v] = (uint8_t)((b >> v) & 1u);
}

/* Alg. 2, DepthFirstTraversal: at the last level evaluate CutVal on the
 * whole graph and keep the path if it is strictly better. */
static void dfs(const merge_in_t *in, int32_t lvl, uint8_t *side, int64_t *best,
                uint8_t *best_side, int64_t *leaves) {
  if (lvl == in->M) {
    int64_t c = or_cutval(in->nv, in->row_ptr, in->col, in->w, side);
    (*leaves)++;
    if (c > *best) {
      *best = c;
      memcpy(best_side, side, (size_t)in->nv);
    }
    return;
  }
  for (int32_t j = 0; j < in->K; j++) {
    assign_part(in, lvl, j, side);
    dfs(in, lvl + 1, side, best, best_side, leaves);
  }
}

/* Exhaustive level-aware merge (Alg. 2). The starting paths are the K^L
 * prefixes over the first L parts in lexicographic order; each is walked
 * depth-first on its own and keeps its own best; the results are reduced by
 * (cut descending, prefix index ascending), so the answer is the first best
 * leaf in lexicographic order whatever L is. Output normalised so that global
 * vertex 0 is on side 0. */
int or_merge_exhaustive(int32_t nv, const int64_t *row_ptr, const int32_t *col,
                        const int32_t *w, int32_t M, const int32_t *first,
                        const int32_t *size, const uint32_t *cand, int32_t K, int32_t L,
                        uint8_t *out_side, int64_t *out_cut, int64_t *out_leaves) {
  if (M < 1 || K < 1 || L < 1 || L > M) return OR_EINVAL;
  double space = pow((double)K, (double)M);
  if (space > 4294967296.0) return OR_ESEARCH;
  merge_in_t in = {nv, M, K, row_ptr, col, w, first, size, cand};
  uint8_t *side = (uint8_t *)calloc((size_t)nv, 1);
  uint8_t *loc = (uint8_t *)calloc((size_t)nv, 1);
  if (!side || !loc) {
    free(side);
    free(loc);
    return OR_ENOMEM;
  }
  int64_t nprefix = 1;
  for (int32_t i = 0; i < L; i++) nprefix *= K;
  int64_t best = -1, leaves = 0;
  for (int64_t pfx = 0; pfx < nprefix; pfx++) {
    /* starting path: digits of pfx in base K, most significant = part 1 */
    int64_t rest = pfx, div = nprefix / K;
    for (int32_t lvl = 0; lvl < L; lvl++) {
      int32_t j = (int32_t)(rest / div);
      rest %= div;
      div = (div > 1) ? div / K : 1;
      assign_part(&in, lvl, j, side);
    }
    int64_t lbest = -1;
    dfs(&in, L, side, &lbest, loc, &leaves);
    if (lbest > best) {
      best = lbest;
      memcpy(out_side, loc, (size_t)nv);
    }
  }
  if (out_side[0]) {
    for (int32_t v = 0; v < nv; v++) out_side[v] ^= 1u;
  }
  *out_cut = best;
  if (out_leaves) *out_leaves = leaves;
  free(side);
  free(loc);
  return OR_OK;
}

/* Beam reading of the merge for product spaces too large to walk: level by
 * level, every kept path is extended by each of the K candidates of the next
 * part; a path's score is CutVal restricted to the edges whose two ends are
 * both assigned (vertices are assigned in index order, so these are the edges
 * (u, v), u < v < end of the last assigned part). The best `beam` extensions
 * are kept, ranked by score descending, then by the tuple (j_1, ..., j_l) in
 * lexicographic order. With beam >= K^(M-1) nothing is ever dropped before
 * the last level and the result equals the exhaustive merge. */
typedef struct {
  int64_t score;
  int32_t *tuple; /* length = current level */
  uint8_t *side;  /* nv entries */
} path_t;

static int tuple_cmp(const int32_t *a, const int32_t *b, int32_t len) {
  for (int32_t i = 0; i < len; i++) {
    if (a[i] < b[i]) return -1;
    if (a[i] > b[i]) return 1;
  }
  return 0;
}

static int32_t g_cmp_len;
static int cmp_path(const void *pa, const void *pb) {
  const path_t *a = (const path_t *)pa, *b = (const path_t *)pb;
  if (a->score > b->score) return -1;
  if (a->score < b->score) return 1;
  return tuple_cmp(a->tuple, b->tuple, g_cmp_len);
}

int or_merge_beam(int32_t nv, const int64_t *row_ptr, const int32_t *col, const int32_t *w,
                  int32_t M, const int32_t *first, const int32_t *size, const uint32_t *cand,
                  int32_t K, int64_t beam, uint8_t *out_side, int64_t *out_cut) {
  if (M < 1 || K < 1 || beam < 1) return OR_EINVAL;
  merge_in_t in = {nv, M, K, row_ptr, col, w, first, size, cand};
  int64_t cap = beam * K;
  path_t *cur = (path_t *)calloc((size_t)cap, sizeof(path_t));
  path_t *ext = (path_t *)calloc((size_t)cap, sizeof(path_t));
  int rc = OR_OK;
  if (!cur || !ext) {
    rc = OR_ENOMEM;
    goto done;
  }
  for (int64_t i = 0; i < cap; i++) {
    cur[i].tuple = (int32_t *)malloc(sizeof(int32_t) * M);
    cur[i].side = (uint8_t *)calloc((size_t)nv, 1);
    ext[i].tuple = (int32_t *)malloc(sizeof(int32_t) * M);
    ext[i].side = (uint8_t *)calloc((size_t)nv, 1);
    if (!cur[i].tuple || !cur[i].side || !ext[i].tuple || !ext[i].side) {
      rc = OR_ENOMEM;
      goto done;
    }
  }
  int64_t ncur = 1; /* the empty path */
  cur[0].score = 0;
  for (int32_t lvl = 0; lvl < M; lvl++) {
    int32_t f = first[lvl], s = size[lvl];
    int32_t new_lo = (lvl == 0) ? 0 : f + 1; /* vertices assigned at this level */
    int32_t new_hi = f + s;
    int64_t next = 0;
    for (int64_t a = 0; a < ncur; a++)
      for (int32_t j = 0; j < K; j++) {
        path_t *e = &ext[next++];
        memcpy(e->side, cur[a].side, (size_t)nv);
        memcpy(e->tuple, cur[a].tuple, sizeof(int32_t) * lvl);
        e->tuple[lvl] = j;
        assign_part(&in, lvl, j, e->side);
        int64_t add = 0;
        for (int32_t v = new_lo; v < new_hi; v++)
          for (int64_t k = row_ptr[v]; k < row_ptr[v + 1]; k++) {
            int32_t u = col[k];
            if (u < v && e->side[u] != e->side[v]) add += w[k];
          }
        e->score = cur[a].score + add;
      }
    g_cmp_len = lvl + 1;
    qsort(ext, (size_t)next, sizeof(path_t), cmp_path);
    int64_t keep = next < beam ? next : beam;
    /* swap the kept extensions into cur (pointer swap keeps buffers owned) */
    for (int64_t i = 0; i < keep; i++) {
      path_t t = cur[i];
      cur[i] = ext[i];
      ext[i] = t;
    }
    ncur = keep;
  }
  memcpy(out_side, cur[0].side, (size_t)nv);
  if (out_side[0]) {
    for (int32_t v = 0; v < nv; v++) out_side[v] ^= 1u;
  }
  *out_cut = cur[0].score;
done: /* calloc zeroed the path records, so unallocated members are NULL */
  for (int64_t i = 0; i < cap; i++) {
    if (cur) {
      free(cur[i].tuple);
      free(cur[i].side);
    }
    if (ext) {
      free(ext[i].tuple);
      free(ext[i].side);
    }
  }
  free(cur);
  free(ext);
  return rc;
}

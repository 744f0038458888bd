/*
 * qis_oracle.c -- reference oracle for the quantum-inspired (QI) search of
 * Ueda, Otsuka and Yunoki, "Quantum-inspired search method for low-energy states of
 * classical Ising Hamiltonians" (arXiv 2010.00180).
 *
 * TEST INFRASTRUCTURE ONLY. Plain, slow, single-threaded FP64 code that follows the
 * paper's Algorithms 1-4 step by step. Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it; the library's product path never does.
 * It shares no code, header or table with the CUDA path.
 *
 * Conventions (Sec. III, Eq. (4)):
 *   state psi = sum_i 2^i sigma_i, stored as W = ceil(N/64) little-endian uint64 words;
 *   sigma_i = 1  <=>  s_i = -1  (sigma^z|1> = -|1>).
 *   H0 = sum_{i<j} J_ij s_i s_j + sum_i h_i s_i                       (Eq. (1))
 *   J is a dense N x N row-major symmetric array with zero diagonal.
 *
 * Floating-point evaluation order (fixed here, since the paper does not state one;
 * compile with -ffp-contract=off so no multiply-add is fused):
 *   E(psi)  = P + F with P = sum_{i<j} J_ij s_i s_j accumulated i-major, j ascending,
 *             and F = sum_i h_i s_i accumulated i ascending, both starting from +0.0.
 *   f_i     = (sum_{j != i} s_j J_ij, j ascending from +0.0) + h_i.
 *   a_i     = -2 s_i f_i                     (energy change of the single flip i)
 *   dE_i    = a_i
 *   dE_ij   = (a_i + a_j) + 4 s_i s_j J_ij  (energy change of the pair flip i<j)
 *   E'      = E_parent + dE                  (Sec. III: the energy of a flipped state
 *                                             is updated from the couplings of the
 *                                             flipped sites only)
 * Products with s = +-1 and scalings by 2 or 4 are exact, so each E' carries exactly
 * the roundings of the additions listed.
 *
 * Candidate order (Alg. 3 loop over j = 1..J, n = 1..n_j with the flip sets I_1, I_2 of
 * Sec. III): candidate index c = i for the single flip of site i (c < N), then
 * c = N + rank(i, j) for the pair i < j in lexicographic order.
 *
 * Flip sets (`flips`): 0 = the single and pair flips of H1 (Eq. (H1), the paper's study);
 * 1 = single flips only (J = 1, the uniform transverse field of the Sec. V outlook);
 * 2 = spin exchanges only (the XX + YY interaction of the Sec. V outlook: the pair (i, j) is
 * a candidate only when s_i != s_j, flipping both, so the total sigma^z is conserved). The
 * candidate index space and loop order stay those of flips = 0; excluded candidates are
 * skipped. With flips = 2 the reachable states are the initial state's magnetisation
 * sector; if that sector is smaller than K+1, the first unused entry can be a placeholder,
 * which (as for any search whose reachable states are all used) ends the search.
 *
 * Every list entry also records a "stamp": 0 for the initial state, (t << 32) | c for a
 * state inserted as candidate c of iteration t (1-based). Stamps are bookkeeping for the
 * tests; they never influence the algorithm.
 */
#include <float.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_EPLACEHOLDER -3 /* a placeholder slot would become a parent (unreachable for K < 2^N) */

static int nwords(int n) { return (n + 63) / 64; }
static int get_sigma(const uint64_t* b, int i) { return (int)((b[i >> 6] >> (i & 63)) & 1u); }
static double spin(const uint64_t* b, int i) { return get_sigma(b, i) ? -1.0 : 1.0; }

/* Compare two states as the integers psi of Eq. (4): most significant word first. */
static int cmp_state(const uint64_t* a, const uint64_t* b, int W) {
  for (int w = W - 1; w >= 0; --w) {
    if (a[w] < b[w]) return -1;
    if (a[w] > b[w]) return 1;
  }
  return 0;
}

/* ---------------------------------------------------------------- Eq. (1) */
double orc_energy(int n, const double* J, const double* h, const uint64_t* bits) {
  double P = 0.0, F = 0.0;
  for (int i = 0; i < n; ++i) {
    double si = spin(bits, i);
    for (int j = i + 1; j < n; ++j) P += J[(size_t)i * n + j] * si * spin(bits, j);
  }
  for (int i = 0; i < n; ++i) F += h[i] * spin(bits, i);
  return P + F;
}

/* Local fields f_i = sum_j J_ij s_j + h_i of one state. */
void orc_fields(int n, const double* J, const double* h, const uint64_t* bits, double* f) {
  for (int i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      acc += spin(bits, j) * J[(size_t)i * n + j];
    }
    f[i] = acc + h[i];
  }
}

/* Candidate index <-> flipped sites (Sec. III flip sets I_1 then I_2). */
int64_t orc_pair_rank(int n, int i, int j) {
  return (int64_t)i * n - (int64_t)i * (i + 1) / 2 + (j - i - 1);
}

/* Energy change of candidate c of a parent with spins from `bits` and fields f. */
static double cand_dE(int n, const double* J, const double* f, const uint64_t* bits, int i, int j) {
  double ai = -2.0 * spin(bits, i) * f[i];
  if (j < 0) return ai;
  double aj = -2.0 * spin(bits, j) * f[j];
  return (ai + aj) + 4.0 * spin(bits, i) * spin(bits, j) * J[(size_t)i * n + j];
}

/* E' of every candidate of one parent, in candidate order (singles, then pairs i<j):
 * E' = E(parent) + dE with the incremental formulas above. out has n(n+1)/2 entries. */
/* Whether candidate (i, j) (j < 0: single flip) belongs to the flip set (see top). */
static int in_flip_set(int flips, const uint64_t* bits, int i, int j) {
  if (j < 0) return flips != 2;
  if (flips == 1) return 0;
  if (flips == 2) return get_sigma(bits, i) != get_sigma(bits, j);
  return 1;
}

/* As orc_candidates for a flip set; excluded candidates get +infinity. */
void orc_candidates_flips(int n, const double* J, const double* h, const uint64_t* bits, int flips,
                          double* out) {
  double* f = malloc((size_t)n * sizeof(double));
  if (!f) return;
  orc_fields(n, J, h, bits, f);
  const double Ep = orc_energy(n, J, h, bits);
  int64_t c = 0;
  for (int i = 0; i < n; ++i, ++c)
    out[c] = in_flip_set(flips, bits, i, -1) ? Ep + cand_dE(n, J, f, bits, i, -1) : 1.0 / 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j, ++c)
      out[c] = in_flip_set(flips, bits, i, j) ? Ep + cand_dE(n, J, f, bits, i, j) : 1.0 / 0.0;
  free(f);
}

void orc_candidates(int n, const double* J, const double* h, const uint64_t* bits, double* out) {
  orc_candidates_flips(n, J, h, bits, 0, out);
}

/* ------------------------------------------------------------ state lists */
/* The four lists of Alg. 2: psi (energy order), psi' (ascending integer order), E, l.
 * Placeholders (I_M in psi/psi', R_M in E) are flagged `empty`; an empty psi' entry
 * compares above every state, like the maximum integer I_M. */
typedef struct {
  int n, W, K1;
  uint64_t* psi;     /* K1 x W, energy order */
  double* E;         /* K1 */
  uint8_t* l;        /* K1: used as a parent */
  uint8_t* empty;    /* K1 */
  uint64_t* stamp;   /* K1 (bookkeeping) */
  uint64_t* src;     /* K1 (bookkeeping for Alg. 4: (search << 32) | position) */
  uint64_t* psis;    /* K1 x W, psi' in ascending order */
  uint8_t* psis_empty;
} qlist;

static void list_free(qlist* L) {
  free(L->psi); free(L->E); free(L->l); free(L->empty); free(L->stamp); free(L->src);
  free(L->psis); free(L->psis_empty);
}

static int list_init(qlist* L, int n, int K) {
  memset(L, 0, sizeof(*L));
  L->n = n; L->W = nwords(n); L->K1 = K + 1;
  L->psi = calloc((size_t)L->K1 * L->W, 8);
  L->E = calloc(L->K1, sizeof(double));
  L->l = calloc(L->K1, 1);
  L->empty = calloc(L->K1, 1);
  L->stamp = calloc(L->K1, 8);
  L->src = calloc(L->K1, 8);
  L->psis = calloc((size_t)L->K1 * L->W, 8);
  L->psis_empty = calloc(L->K1, 1);
  if (!L->psi || !L->E || !L->l || !L->empty || !L->stamp || !L->src || !L->psis || !L->psis_empty) {
    list_free(L);
    return ORC_ENOMEM;
  }
  for (int k = 0; k < L->K1; ++k) {
    L->E[k] = DBL_MAX;         /* R_M */
    L->empty[k] = 1;           /* I_M */
    L->psis_empty[k] = 1;
    L->stamp[k] = UINT64_MAX;
    L->src[k] = UINT64_MAX;
  }
  return ORC_OK;
}

/* Binary_search of Alg. 2 over psi': returns p (0..K1) with psi'_p <= x < psi'_{p+1}
 * in 1-based terms, i.e. the number of entries <= x, and sets *found when psi'_p == x. */
static int bsearch_state(const qlist* L, const uint64_t* x, int* found) {
  int lo = 0, hi = L->K1; /* count of entries <= x lies in [lo, hi] */
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    int le = L->psis_empty[mid] ? 0 : (cmp_state(L->psis + (size_t)mid * L->W, x, L->W) <= 0);
    if (le) lo = mid + 1; else hi = mid;
  }
  *found = (lo > 0 && !L->psis_empty[lo - 1] && cmp_state(L->psis + (size_t)(lo - 1) * L->W, x, L->W) == 0);
  return lo;
}

/* Binary_search of Alg. 2 over E: number of entries with E_k <= e (insertion after equals). */
static int bsearch_energy(const qlist* L, double e) {
  int lo = 0, hi = L->K1;
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (L->E[mid] <= e) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* update_list_sub of Alg. 2: if E < E_{K+1}, drop slot K+1 and insert (x, E, l) after every
 * entry of energy <= E; keep psi' sorted (remove the dropped state, insert x at p'). */
static void update_list_sub(qlist* L, const uint64_t* x, double e, uint8_t l, int pprime,
                            uint64_t stamp, uint64_t src) {
  const int W = L->W, K1 = L->K1;
  if (!(e < L->E[K1 - 1])) return;
  /* position of the evicted state psi_{K+1} in psi' */
  int pe;
  if (L->empty[K1 - 1]) {
    pe = K1 - 1; /* an I_M entry: the last one of psi' */
  } else {
    int f;
    pe = bsearch_state(L, L->psi + (size_t)(K1 - 1) * W, &f) - 1;
  }
  /* psi': remove index pe, insert x so that it follows the first pprime entries of the old list */
  int ins = pprime; /* 0-based insertion index in the old list */
  if (pe < ins) {
    memmove(L->psis + (size_t)pe * W, L->psis + (size_t)(pe + 1) * W, (size_t)(ins - 1 - pe) * W * 8);
    memmove(L->psis_empty + pe, L->psis_empty + pe + 1, (size_t)(ins - 1 - pe));
    ins -= 1;
  } else {
    memmove(L->psis + (size_t)(ins + 1) * W, L->psis + (size_t)ins * W, (size_t)(pe - ins) * W * 8);
    memmove(L->psis_empty + ins + 1, L->psis_empty + ins, (size_t)(pe - ins));
  }
  memcpy(L->psis + (size_t)ins * W, x, (size_t)W * 8);
  L->psis_empty[ins] = 0;
  /* energy-ordered lists: insert after all entries with E_k <= e, drop the last */
  int p = bsearch_energy(L, e);
  int tail = K1 - 1 - p;
  memmove(L->psi + (size_t)(p + 1) * W, L->psi + (size_t)p * W, (size_t)tail * W * 8);
  memmove(L->E + p + 1, L->E + p, (size_t)tail * sizeof(double));
  memmove(L->l + p + 1, L->l + p, (size_t)tail);
  memmove(L->empty + p + 1, L->empty + p, (size_t)tail);
  memmove(L->stamp + p + 1, L->stamp + p, (size_t)tail * 8);
  memmove(L->src + p + 1, L->src + p, (size_t)tail * 8);
  memcpy(L->psi + (size_t)p * W, x, (size_t)W * 8);
  L->E[p] = e;
  L->l[p] = l;
  L->empty[p] = 0;
  L->stamp[p] = stamp;
  L->src[p] = src;
}

/* ---------------------------------------------------------------- Alg. 3 */
/* One QI single search. The list starts as [psi0, placeholders]; each of I iterations
 * takes the first unused entry (in list order) as the parent and pushes all of its
 * single and pair flips through update_list (Alg. 2).
 * update_list computes E' first and performs the duplicate binary search only when
 * E' < E_{K+1}: both tests are side-effect free and the insertion needs both, so the
 * outcome equals the paper's search-first order. */
static int qi_search(const double* J, const double* h, int n, int K, int I, int flips, const uint64_t* psi0,
                     qlist* L, int* n_productive) {
  const int W = nwords(n);
  int rc = list_init(L, n, K);
  if (rc) return rc;
  double* f = malloc((size_t)n * sizeof(double));
  uint64_t* parent = malloc((size_t)W * 8);
  uint64_t* x = malloc((size_t)W * 8);
  if (!f || !parent || !x) { free(f); free(parent); free(x); list_free(L); return ORC_ENOMEM; }

  memcpy(L->psi, psi0, (size_t)W * 8);
  L->E[0] = orc_energy(n, J, h, psi0);
  L->empty[0] = 0;
  L->stamp[0] = 0;
  memcpy(L->psis, psi0, (size_t)W * 8);
  L->psis_empty[0] = 0;

  int prod = 0;
  for (int it = 1; it <= I; ++it) {
    int k;
    for (k = 0; k < L->K1; ++k)
      if (!L->l[k]) break;
    if (k == L->K1) continue;              /* every entry used: the iteration does nothing */
    if (L->empty[k]) {
      if (flips == 0) { rc = ORC_EPLACEHOLDER; break; }   /* unreachable for K < 2^N */
      continue;                            /* the sector's reachable states are all used */
    }
    L->l[k] = 1;
    ++prod;
    memcpy(parent, L->psi + (size_t)k * W, (size_t)W * 8);
    const double Ep = L->E[k];
    orc_fields(n, J, h, parent, f);

    int64_t c = 0;
    for (int order = 1; order <= 2; ++order) {
      for (int i = 0; i < n; ++i) {
        for (int j = (order == 1 ? -1 : i + 1); j < (order == 1 ? 0 : n); ++j, ++c) {
          if (!in_flip_set(flips, parent, i, j)) continue;
          const double e = Ep + cand_dE(n, J, f, parent, i, j);   /* E' */
          if (!(e < L->E[L->K1 - 1])) continue;
          memcpy(x, parent, (size_t)W * 8);                        /* Alg. 1: XOR with 2^i (+2^j) */
          x[i >> 6] ^= (uint64_t)1 << (i & 63);
          if (j >= 0) x[j >> 6] ^= (uint64_t)1 << (j & 63);
          int found;
          int p = bsearch_state(L, x, &found);
          if (found) continue;
          update_list_sub(L, x, e, 0, p, ((uint64_t)it << 32) | (uint64_t)c, 0);
        }
      }
    }
  }
  if (n_productive) *n_productive = prod;
  free(f); free(parent); free(x);
  if (rc) list_free(L);
  return rc;
}

static int check_args(int n, int K) {
  if (n < 1 || K < 1) return ORC_EINVAL;
  if (n < 63 && (uint64_t)K >= ((uint64_t)1 << n)) return ORC_EINVAL; /* 1 <= K < 2^N (Alg. 2) */
  return ORC_OK;
}

static void export_list(const qlist* L, uint64_t* bits, double* E, uint8_t* used, uint64_t* stamp,
                        uint64_t* src, int* count) {
  int cnt = 0;
  for (int k = 0; k < L->K1; ++k) {
    if (L->empty[k]) break;
    ++cnt;
  }
  if (bits) memcpy(bits, L->psi, (size_t)L->K1 * L->W * 8);
  if (E) memcpy(E, L->E, (size_t)L->K1 * sizeof(double));
  if (used) memcpy(used, L->l, (size_t)L->K1);
  if (stamp) memcpy(stamp, L->stamp, (size_t)L->K1 * 8);
  if (src) memcpy(src, L->src, (size_t)L->K1 * 8);
  if (count) *count = cnt;
}

/* Alg. 3. Outputs hold K+1 slots in energy order; slots past *count are placeholders
 * (bits 0, E = DBL_MAX, stamp = UINT64_MAX). Any output pointer may be NULL. */
int orc_qi_search_flips(int n, const double* J, const double* h, int K, int I, int flips,
                        const uint64_t* psi0, uint64_t* bits_out, double* E_out, uint8_t* used_out,
                        uint64_t* stamp_out, int* count_out, int* productive_out) {
  int rc = check_args(n, K);
  if (rc) return rc;
  if (flips < 0 || flips > 2) return ORC_EINVAL;
  qlist L;
  rc = qi_search(J, h, n, K, I, flips, psi0, &L, productive_out);
  if (rc) return rc;
  export_list(&L, bits_out, E_out, used_out, stamp_out, NULL, count_out);
  list_free(&L);
  return ORC_OK;
}

int orc_qi_search(int n, const double* J, const double* h, int K, int I, const uint64_t* psi0,
                  uint64_t* bits_out, double* E_out, uint8_t* used_out, uint64_t* stamp_out,
                  int* count_out, int* productive_out) {
  return orc_qi_search_flips(n, J, h, K, I, 0, psi0, bits_out, E_out, used_out, stamp_out, count_out,
                             productive_out);
}

/* ---------------------------------------------------------------- Alg. 4 */
/* QI multi search with the L initial states phi (L x W) given by the caller. Search 1's
 * list receives the lists of searches 2..L in turn: each entry, taken in energy order,
 * is binary-searched in psi' and, when absent, offered to update_list_sub with its own
 * energy and used flag. (The paper's listing pairs the spin-ordered psi'_{0,j} with the
 * energy-ordered E_{0,j}; the entries are read here as (psi_{0,j}, E_{0,j}, l_{0,j}).)
 * src of a merged entry = (search index r << 32) | position in search r's final list.
 * Optional per-search outputs (L x (K+1) slots each) may be NULL. */
int orc_qi_multi_search_flips(int n, const double* J, const double* h, int K, int I, int flips, int Lc,
                              const uint64_t* phi, uint64_t* bits_out, double* E_out, uint8_t* used_out,
                              uint64_t* src_out, int* count_out,
                              uint64_t* all_bits, double* all_E, uint8_t* all_used, uint64_t* all_stamp,
                              int* all_count) {
  int rc = check_args(n, K);
  if (rc) return rc;
  if (Lc < 1 || flips < 0 || flips > 2) return ORC_EINVAL;
  const int W = nwords(n), K1 = K + 1;
  qlist M;
  rc = qi_search(J, h, n, K, I, flips, phi, &M, NULL);
  if (rc) return rc;
  for (int k = 0; k < K1; ++k)
    if (!M.empty[k]) M.src[k] = (uint64_t)k;
  if (all_bits || all_E || all_used || all_stamp || all_count)
    export_list(&M, all_bits, all_E, all_used, all_stamp, NULL, all_count);
  for (int r = 1; r < Lc && !rc; ++r) {
    qlist S;
    rc = qi_search(J, h, n, K, I, flips, phi + (size_t)r * W, &S, NULL);
    if (rc) break;
    if (all_bits || all_E || all_used || all_stamp || all_count)
      export_list(&S, all_bits ? all_bits + (size_t)r * K1 * W : NULL, all_E ? all_E + (size_t)r * K1 : NULL,
                  all_used ? all_used + (size_t)r * K1 : NULL, all_stamp ? all_stamp + (size_t)r * K1 : NULL,
                  NULL, all_count ? all_count + r : NULL);
    for (int j = 0; j < K1; ++j) {
      if (S.empty[j]) break;
      int found;
      const uint64_t* x = S.psi + (size_t)j * W;
      int p = bsearch_state(&M, x, &found);
      if (!found) update_list_sub(&M, x, S.E[j], S.l[j], p, S.stamp[j], ((uint64_t)r << 32) | (uint64_t)j);
    }
    list_free(&S);
  }
  if (!rc) export_list(&M, bits_out, E_out, used_out, NULL, src_out, count_out);
  list_free(&M);
  return rc;
}

int orc_qi_multi_search(int n, const double* J, const double* h, int K, int I, int Lc,
                        const uint64_t* phi, uint64_t* bits_out, double* E_out, uint8_t* used_out,
                        uint64_t* src_out, int* count_out,
                        uint64_t* all_bits, double* all_E, uint8_t* all_used, uint64_t* all_stamp,
                        int* all_count) {
  return orc_qi_multi_search_flips(n, J, h, K, I, 0, Lc, phi, bits_out, E_out, used_out, src_out, count_out,
                                   all_bits, all_E, all_used, all_stamp, all_count);
}

/* ------------------------------------------------------------ brute force */
/* Exhaustive search over all 2^N states (the paper's exact reference for N <= 30):
 * E of every psi from Eq. (1) directly, then the k lowest by (E, psi). n <= 24. */
typedef struct { double e; uint64_t psi; } epair;
static int cmp_epair(const void* a, const void* b) {
  const epair* x = a; const epair* y = b;
  if (x->e < y->e) return -1;
  if (x->e > y->e) return 1;
  return (x->psi < y->psi) ? -1 : (x->psi > y->psi);
}

int orc_brute_force(int n, const double* J, const double* h, int k, uint64_t* psi_out, double* E_out) {
  if (n < 1 || n > 24 || k < 1) return ORC_EINVAL;
  const uint64_t total = (uint64_t)1 << n;
  if ((uint64_t)k > total) return ORC_EINVAL;
  epair* all = malloc(total * sizeof(epair));
  if (!all) return ORC_ENOMEM;
  for (uint64_t psi = 0; psi < total; ++psi) {
    all[psi].psi = psi;
    all[psi].e = orc_energy(n, J, h, &psi);
  }
  qsort(all, total, sizeof(epair), cmp_epair);
  for (int t = 0; t < k; ++t) { psi_out[t] = all[t].psi; E_out[t] = all[t].e; }
  free(all);
  return ORC_OK;
}

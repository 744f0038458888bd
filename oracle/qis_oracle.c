/*
 * qis_oracle.c -- reference oracle for the quantum-inspired (QI) search of
 * Ueda, Otsuka and Yunoki, "Quantum-inspired search method for low-energy states of
 * classical Ising Hamiltonians" (arXiv 2010.00180).
 *
 * TEST INFRASTRUCTURE ONLY. Plain, slow, single-threaded FP64 code that restates what the
 * paper's Algorithms 1-4 compute, in their order, from the definitions of Sec. III: the flip
 * sets, the incremental energy, and the kept states of Alg. 2 as an ordered set with its
 * admission rule. Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it; the library's product path never does. It shares no code, header or
 * table with the CUDA path.
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

/* ------------------------------------------------------------ kept states */
/* What Alg. 2 maintains, stated as a data structure: the kept states of a search, at most
 * K+1 of them, in ascending order of the key (E, arrival). Its rules follow from Sec. III:
 *   - a state is kept at most once (a generated state already kept is skipped);
 *   - a new state arrives after every state already kept, so among equal energies it ranks
 *     last: it is placed after every kept state with E <= E';
 *   - only the K+1 lowest keys are kept: when all K+1 places are taken, a new state enters
 *     only if its key precedes the last one, i.e. E' < E_{K+1} strictly (its arrival is later),
 *     and the last state leaves.
 * Unfilled places are the listing's placeholders (I_M, R_M): they are simply absent here.
 * Membership is a hash set of the kept states (open addressing with linear probing, FNV-1a 64
 * over the state's words); a removed state is taken out by shifting later members of its
 * probe run back, so no tombstones accumulate. */
typedef struct {
  int n, W, K1, count;
  uint64_t* psi;     /* K1 x W, key order; entries 0 .. count-1 are kept states */
  double* E;         /* K1 */
  uint8_t* l;        /* K1: used as a parent */
  uint64_t* stamp;   /* K1 (bookkeeping) */
  uint64_t* src;     /* K1 (bookkeeping for Alg. 4: (search << 32) | position) */
  uint64_t* hkey;    /* hcap x W: the member states of the hash set */
  uint8_t* hused;    /* hcap: slot occupied */
  int hcap;          /* power of two >= 4 K1 */
} kept_set;

static uint64_t state_hash(const uint64_t* x, int W) {
  uint64_t h = 0xcbf29ce484222325ull;   /* FNV-1a, 64 bits, over the bytes of the words */
  for (int w = 0; w < W; ++w)
    for (int b = 0; b < 8; ++b) {
      h ^= (x[w] >> (8 * b)) & 0xffu;
      h *= 0x100000001b3ull;
    }
  return h;
}

/* Slot of x in the hash set, or the empty slot where its probe run ends. */
static int hs_find(const kept_set* S, const uint64_t* x, int* present) {
  int pos = (int)(state_hash(x, S->W) & (uint64_t)(S->hcap - 1));
  while (S->hused[pos]) {
    if (memcmp(S->hkey + (size_t)pos * S->W, x, (size_t)S->W * 8) == 0) {
      *present = 1;
      return pos;
    }
    pos = (pos + 1) & (S->hcap - 1);
  }
  *present = 0;
  return pos;
}

static int hs_contains(const kept_set* S, const uint64_t* x) {
  int present;
  hs_find(S, x, &present);
  return present;
}

static void hs_insert(kept_set* S, const uint64_t* x) {
  int present;
  const int pos = hs_find(S, x, &present);
  if (present) return;
  memcpy(S->hkey + (size_t)pos * S->W, x, (size_t)S->W * 8);
  S->hused[pos] = 1;
}

/* Remove x; later members of the probe run move back into the gap when their home slot does
 * not lie cyclically in (gap, their slot]. */
static void hs_remove(kept_set* S, const uint64_t* x) {
  int present;
  int gap = hs_find(S, x, &present);
  if (!present) return;
  const int m = S->hcap - 1;
  S->hused[gap] = 0;
  for (int j = (gap + 1) & m; S->hused[j]; j = (j + 1) & m) {
    const int home = (int)(state_hash(S->hkey + (size_t)j * S->W, S->W) & (uint64_t)m);
    const int stays = (gap <= j) ? (gap < home && home <= j) : (gap < home || home <= j);
    if (stays) continue;
    memcpy(S->hkey + (size_t)gap * S->W, S->hkey + (size_t)j * S->W, (size_t)S->W * 8);
    S->hused[gap] = 1;
    S->hused[j] = 0;
    gap = j;
  }
}

static void kept_free(kept_set* S) {
  free(S->psi); free(S->E); free(S->l); free(S->stamp); free(S->src); free(S->hkey); free(S->hused);
}

static int kept_init(kept_set* S, int n, int K) {
  memset(S, 0, sizeof(*S));
  S->n = n; S->W = nwords(n); S->K1 = K + 1; S->count = 0;
  S->hcap = 4;
  while (S->hcap < 4 * S->K1) S->hcap <<= 1;
  S->psi = calloc((size_t)S->K1 * S->W, 8);
  S->E = calloc(S->K1, sizeof(double));
  S->l = calloc(S->K1, 1);
  S->stamp = calloc(S->K1, 8);
  S->src = calloc(S->K1, 8);
  S->hkey = calloc((size_t)S->hcap * S->W, 8);
  S->hused = calloc(S->hcap, 1);
  if (!S->psi || !S->E || !S->l || !S->stamp || !S->src || !S->hkey || !S->hused) {
    kept_free(S);
    return ORC_ENOMEM;
  }
  return ORC_OK;
}

/* Whether a new state of energy e would be kept (the K+1 rule above). */
static int admissible(const kept_set* S, double e) {
  return S->count < S->K1 || e < S->E[S->K1 - 1];
}

/* Offer state x (not a member) with energy e and flag l: kept if admissible, after every kept
 * state with E <= e; the last state leaves when all K+1 places were taken. */
static void offer(kept_set* S, const uint64_t* x, double e, uint8_t l, uint64_t stamp, uint64_t src) {
  if (!admissible(S, e)) return;
  const int W = S->W;
  if (S->count == S->K1) {
    hs_remove(S, S->psi + (size_t)(S->K1 - 1) * W);
    S->count -= 1;
  }
  int p = 0;   /* first place whose energy exceeds e (binary search over the kept energies) */
  int hi = S->count;
  while (p < hi) {
    const int mid = (p + hi) / 2;
    if (S->E[mid] <= e) p = mid + 1; else hi = mid;
  }
  const int tail = S->count - p;
  memmove(S->psi + (size_t)(p + 1) * W, S->psi + (size_t)p * W, (size_t)tail * W * 8);
  memmove(S->E + p + 1, S->E + p, (size_t)tail * sizeof(double));
  memmove(S->l + p + 1, S->l + p, (size_t)tail);
  memmove(S->stamp + p + 1, S->stamp + p, (size_t)tail * 8);
  memmove(S->src + p + 1, S->src + p, (size_t)tail * 8);
  memcpy(S->psi + (size_t)p * W, x, (size_t)W * 8);
  S->E[p] = e;
  S->l[p] = l;
  S->stamp[p] = stamp;
  S->src[p] = src;
  S->count += 1;
  hs_insert(S, x);
}

/* ---------------------------------------------------------------- Alg. 3 */
/* One QI single search. The kept states start as {psi0} (the other K places unfilled); each of
 * I iterations takes as the parent the first kept state, in key order, not yet used, marks it
 * used, and offers every candidate of its flip set, in the candidate order of Sec. III, to the
 * kept states. A candidate's energy and the K+1 rule are tested before the membership test:
 * both are free of side effects, so the outcome is that of testing membership first. */
static int qi_search(const double* J, const double* h, int n, int K, int I, int flips, const uint64_t* psi0,
                     kept_set* S, int* n_productive) {
  const int W = nwords(n);
  int rc = kept_init(S, n, K);
  if (rc) return rc;
  double* f = malloc((size_t)n * sizeof(double));
  uint64_t* parent = malloc((size_t)W * 8);
  uint64_t* x = malloc((size_t)W * 8);
  if (!f || !parent || !x) { free(f); free(parent); free(x); kept_free(S); return ORC_ENOMEM; }

  offer(S, psi0, orc_energy(n, J, h, psi0), 0, 0, 0);

  int prod = 0;
  for (int it = 1; it <= I; ++it) {
    int k = 0;
    while (k < S->count && S->l[k]) ++k;
    if (k == S->K1) continue;              /* every kept state used: the iteration does nothing */
    if (k == S->count) {
      /* every kept state used with places still unfilled: the listing would pick a placeholder.
       * For single and pair flips that cannot happen when K < 2^N (the kept states would be
       * closed under single flips, i.e. all 2^N states); for exchanges it means the
       * magnetisation sector holds no further state, and the search has ended. */
      if (flips == 0) { rc = ORC_EPLACEHOLDER; break; }
      continue;
    }
    S->l[k] = 1;
    ++prod;
    memcpy(parent, S->psi + (size_t)k * W, (size_t)W * 8);
    const double Ep = S->E[k];
    orc_fields(n, J, h, parent, f);

    int64_t c = 0;   /* candidate index: singles i, then pairs (i, j) in lexicographic order */
    for (int order = 1; order <= 2; ++order) {
      for (int i = 0; i < n; ++i) {
        for (int j = (order == 1 ? -1 : i + 1); j < (order == 1 ? 0 : n); ++j, ++c) {
          if (!in_flip_set(flips, parent, i, j)) continue;
          const double e = Ep + cand_dE(n, J, f, parent, i, j);   /* E' */
          if (!admissible(S, e)) continue;
          memcpy(x, parent, (size_t)W * 8);                        /* Alg. 1: XOR with 2^i (+2^j) */
          x[i >> 6] ^= (uint64_t)1 << (i & 63);
          if (j >= 0) x[j >> 6] ^= (uint64_t)1 << (j & 63);
          if (hs_contains(S, x)) continue;
          offer(S, x, e, 0, ((uint64_t)it << 32) | (uint64_t)c, 0);
        }
      }
    }
  }
  if (n_productive) *n_productive = prod;
  free(f); free(parent); free(x);
  if (rc) kept_free(S);
  return rc;
}

static int check_args(int n, int K) {
  if (n < 1 || K < 1) return ORC_EINVAL;
  if (n < 63 && (uint64_t)K >= ((uint64_t)1 << n)) return ORC_EINVAL; /* 1 <= K < 2^N (Alg. 2) */
  return ORC_OK;
}

/* The K+1 places in key order; places past the kept states are the listing's placeholders:
 * bits 0, E = DBL_MAX (R_M), not used, stamp and src UINT64_MAX. */
static void export_list(const kept_set* S, uint64_t* bits, double* E, uint8_t* used, uint64_t* stamp,
                        uint64_t* src, int* count) {
  const int W = S->W, K1 = S->K1, c = S->count;
  if (bits) {
    memcpy(bits, S->psi, (size_t)c * W * 8);
    memset(bits + (size_t)c * W, 0, (size_t)(K1 - c) * W * 8);
  }
  for (int k = 0; k < K1; ++k) {
    if (E) E[k] = k < c ? S->E[k] : DBL_MAX;
    if (used) used[k] = k < c ? S->l[k] : 0;
    if (stamp) stamp[k] = k < c ? S->stamp[k] : UINT64_MAX;
    if (src) src[k] = k < c ? S->src[k] : UINT64_MAX;
  }
  if (count) *count = c;
}

/* Alg. 3. Outputs hold K+1 slots in energy order; slots past *count are placeholders
 * (bits 0, E = DBL_MAX, stamp = UINT64_MAX). Any output pointer may be NULL. */
int orc_qi_search_flips(int n, const double* J, const double* h, int K, int I, int flips,
                        const uint64_t* psi0, uint64_t* bits_out, double* E_out, uint8_t* used_out,
                        uint64_t* stamp_out, int* count_out, int* productive_out) {
  int rc = check_args(n, K);
  if (rc) return rc;
  if (flips < 0 || flips > 2) return ORC_EINVAL;
  kept_set S;
  rc = qi_search(J, h, n, K, I, flips, psi0, &S, productive_out);
  if (rc) return rc;
  export_list(&S, bits_out, E_out, used_out, stamp_out, NULL, count_out);
  kept_free(&S);
  return ORC_OK;
}

int orc_qi_search(int n, const double* J, const double* h, int K, int I, const uint64_t* psi0,
                  uint64_t* bits_out, double* E_out, uint8_t* used_out, uint64_t* stamp_out,
                  int* count_out, int* productive_out) {
  return orc_qi_search_flips(n, J, h, K, I, 0, psi0, bits_out, E_out, used_out, stamp_out, count_out,
                             productive_out);
}

/* ---------------------------------------------------------------- Alg. 4 */
/* QI multi search with the L initial states phi (L x W) given by the caller: L independent
 * searches; the kept states of search 1 then receive those of searches 2..L in turn, each
 * list read in key order, every state not already kept offered with its own energy, used
 * flag and stamp under the rules of Alg. 2 above. (The paper's listing pairs the spin-ordered
 * psi'_{0,j} with the energy-ordered E_{0,j}; the entries are read here as (psi_{0,j},
 * E_{0,j}, l_{0,j}) of one state.)
 * src of a merged entry = (search index r << 32) | position in search r's final list.
 * Optional per-search outputs (L x (K+1) places each) may be NULL. */
int orc_qi_multi_search_flips(int n, const double* J, const double* h, int K, int I, int flips, int Lc,
                              const uint64_t* phi, uint64_t* bits_out, double* E_out, uint8_t* used_out,
                              uint64_t* src_out, int* count_out,
                              uint64_t* all_bits, double* all_E, uint8_t* all_used, uint64_t* all_stamp,
                              int* all_count) {
  int rc = check_args(n, K);
  if (rc) return rc;
  if (Lc < 1 || flips < 0 || flips > 2) return ORC_EINVAL;
  const int W = nwords(n), K1 = K + 1;
  const int want_all = all_bits || all_E || all_used || all_stamp || all_count;
  kept_set M;
  rc = qi_search(J, h, n, K, I, flips, phi, &M, NULL);
  if (rc) return rc;
  for (int k = 0; k < M.count; ++k) M.src[k] = (uint64_t)k;
  if (want_all) export_list(&M, all_bits, all_E, all_used, all_stamp, NULL, all_count);
  for (int r = 1; r < Lc && !rc; ++r) {
    kept_set S;
    rc = qi_search(J, h, n, K, I, flips, phi + (size_t)r * W, &S, NULL);
    if (rc) break;
    if (want_all)
      export_list(&S, all_bits ? all_bits + (size_t)r * K1 * W : NULL, all_E ? all_E + (size_t)r * K1 : NULL,
                  all_used ? all_used + (size_t)r * K1 : NULL, all_stamp ? all_stamp + (size_t)r * K1 : NULL,
                  NULL, all_count ? all_count + r : NULL);
    for (int j = 0; j < S.count; ++j) {
      const uint64_t* x = S.psi + (size_t)j * W;
      if (!hs_contains(&M, x)) offer(&M, x, S.E[j], S.l[j], S.stamp[j], ((uint64_t)r << 32) | (uint64_t)j);
    }
    kept_free(&S);
  }
  if (!rc) export_list(&M, bits_out, E_out, used_out, NULL, src_out, count_out);
  kept_free(&M);
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

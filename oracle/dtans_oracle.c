/*
 * CSR-dtANS oracle: a plain, slow, deliberately simple CPU reference for the
 * method of "Fast Entropy Decoding for Sparse MVM on GPUs" (Schaetzle,
 * Pegolotti, Pueschel, arXiv 2603.01915).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py may load this library.  The
 * product path (paper_2603_01915_gb300/) never links, imports or calls it,
 * and the two share no code, headers, tables or constant generators.
 *
 * Everything is parametric in (K, W, M, l, o, f) so that the paper's worked
 * dtANS example (Sec. IV-D: K = 8, W = 4, M = 4, l = 2, o = 3, f = 2) runs
 * through the same code as CSR-dtANS (K = 2^12, W = 2^32, M = 2^8, l = 8,
 * o = 3, f = 2).  Arithmetic on the decoder state uses unsigned __int128.
 *
 * Readings of passages where the paper is silent or ambiguous are listed with
 * each function; they are the same readings the library implements.
 *
 * Pins: tests/test_oracle_*.py check this file against the paper's worked
 * examples (Sec. III-D, Sec. IV-D, Fig. "CSR example"), closed forms, size
 * bounds, brute force, round trips and hand-worked multi-lane slices (the
 * interleave order, the escape raw-word order and the placement of the
 * optional slot permutation).  Parity is pinned for every exported function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Parameters                                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t logK;         /* K = 2^logK slots per coding table (Sec. IV-D)    */
  int32_t logW;         /* W = 2^logW, radix of a stored word (Sec. IV-D)   */
  int32_t M;            /* cap on a symbol's multiplicity (Sec. IV-C)       */
  int32_t l;            /* slots per segment (Sec. IV-B)                    */
  int32_t o;            /* words unpacked into one segment's slots          */
  int32_t f;            /* conditional checks per segment                   */
  int32_t spi;          /* symbols per item: 2 = (delta, value), 1 = plain  */
  int32_t raw_words[2]; /* stored words per escaped symbol of each domain   */
  int32_t raw_bits[2];  /* bits charged per escaped symbol (table choice)   */
  int32_t slice;        /* units interleaved per slice (32 = warp width)    */
} or_params;

/* One coding table (Sec. III-D "Constructing the coding table", Sec. IV-C).
 * All arrays are caller-allocated with K entries. */
typedef struct {
  int64_t nkept;        /* T: kept symbols, in rank order                   */
  int32_t has_esc;      /* escape symbol present                            */
  int32_t pad_esc;      /* the tail pad symbol is the escape symbol         */
  uint64_t pad_key;     /* key of the pad symbol when it is a kept symbol   */
  uint32_t esc_first, esc_mult;
  double cost_bits;     /* coded bits + escaped raw bits of the chosen T    */
  uint64_t *kept_key;   /* [K] */
  uint32_t *kept_first; /* [K] first slot of each kept symbol               */
  uint32_t *kept_mult;  /* [K] multiplicity (= base) of each kept symbol    */
  uint64_t *slot_key;   /* [K] symbol key of each slot (0 if unused / esc)  */
  uint32_t *slot_digit; /* [K] digit of each slot                           */
  uint32_t *slot_base;  /* [K] base (multiplicity) of each slot's symbol    */
  uint8_t *slot_kind;   /* [K] 0 unused, 1 kept symbol, 2 escape symbol     */
} or_table;

/* ------------------------------------------------------------------------ */
/* Entropy, Eq. (1) and Eq. (2)                                              */
/* ------------------------------------------------------------------------ */

/* H(P) = sum_w -P(w) log2 P(w), with P the empirical distribution of counts. */
double or_entropy(int64_t ns, const uint64_t *counts) {
  double total = 0.0, h = 0.0;
  for (int64_t i = 0; i < ns; ++i) total += (double)counts[i];
  if (total == 0.0) return 0.0;
  for (int64_t i = 0; i < ns; ++i) {
    if (counts[i] == 0) continue;
    double p = (double)counts[i] / total;
    h -= p * log2(p);
  }
  return h;
}

/* H(P, P') = sum_w -P(w) log2 P'(w). */
double or_cross_entropy(int64_t ns, const uint64_t *counts, const double *q) {
  double total = 0.0, h = 0.0;
  for (int64_t i = 0; i < ns; ++i) total += (double)counts[i];
  if (total == 0.0) return 0.0;
  for (int64_t i = 0; i < ns; ++i) {
    if (counts[i] == 0) continue;
    double p = (double)counts[i] / total;
    h -= p * log2(q[i]);
  }
  return h;
}

/* ------------------------------------------------------------------------ */
/* Coding-table construction (Sec. III-D, Sec. IV-C, Sec. IV-F "Escaping")   */
/* ------------------------------------------------------------------------ */
/*
 * The paper fixes what a table holds (symbol, digit, base per slot; each
 * symbol on consecutive slots with digits 0..m-1 and base m; m <= M), that
 * P' should minimise the cross entropy, and that rare symbols are escaped so
 * that the expected total size is minimal.  It does not print the search.
 * Reading used here:
 *   1. rank the distinct symbols by (count descending, key ascending);
 *   2. for every T in [0, Tmax] keep ranks < T and escape the rest (the escape
 *      symbol exists iff their total count E > 0); Tmax = S if the S distinct
 *      symbols fit in K slots, else K - 1;
 *   3. give every table symbol one slot, then hand out the remaining slots one
 *      at a time to the symbol with the largest gain c*(log2(m+1) - log2(m))
 *      among those with m < M (ties: lower rank, escape ranked last); this
 *      maximises sum c*log2(m) because the objective is separable and concave;
 *   4. cost(T) = sum over table symbols in rank order of c*(logK - log2(m)),
 *      then + E*raw_bits; pick the minimum, ties to the larger T;
 *   5. lay the kept symbols out in rank order on consecutive slots, then the
 *      escape symbol; unused slots stay zero.
 * The pad symbol of a tail segment (Sec. IV-F "end of row") is the rank-0
 * kept symbol, or the escape symbol when nothing is kept.
 */

typedef struct {
  uint64_t key, count;
} or_kc;

static int cmp_rank(const void *a, const void *b) {
  const or_kc *x = (const or_kc *)a, *y = (const or_kc *)b;
  if (x->count != y->count) return x->count > y->count ? -1 : 1;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return 0;
}

typedef struct {
  double g;
  int64_t i;
} or_hent;

static int h_better(or_hent a, or_hent b) { return a.g > b.g || (a.g == b.g && a.i < b.i); }

static void h_push(or_hent *h, int64_t *hn, or_hent e) {
  int64_t i = (*hn)++;
  h[i] = e;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!h_better(h[i], h[p])) break;
    or_hent t = h[i];
    h[i] = h[p];
    h[p] = t;
    i = p;
  }
}

static or_hent h_pop(or_hent *h, int64_t *hn) {
  or_hent top = h[0];
  h[0] = h[--(*hn)];
  int64_t i = 0;
  for (;;) {
    int64_t a = 2 * i + 1, b = a + 1, best = i;
    if (a < *hn && h_better(h[a], h[best])) best = a;
    if (b < *hn && h_better(h[b], h[best])) best = b;
    if (best == i) break;
    or_hent t = h[i];
    h[i] = h[best];
    h[best] = t;
    i = best;
  }
  return top;
}

/* Step 3: greedy marginal-gain allocation of K slots among ns table symbols
 * with counts c[0..ns-1] (rank order, escape last), each between 1 and M. */
static void allocate(int64_t ns, const uint64_t *c, int64_t K, int64_t M, const double *L, uint32_t *m,
                     or_hent *heap) {
  int64_t hn = 0;
  for (int64_t s = 0; s < ns; ++s) {
    m[s] = 1;
    if (M > 1) h_push(heap, &hn, (or_hent){(double)c[s] * (L[2] - L[1]), s});
  }
  int64_t extra = K - ns;
  while (extra > 0 && hn > 0) {
    or_hent t = h_pop(heap, &hn);
    int64_t s = t.i;
    m[s] += 1;
    extra -= 1;
    if ((int64_t)m[s] < M) h_push(heap, &hn, (or_hent){(double)c[s] * (L[m[s] + 1] - L[m[s]]), s});
  }
}

/* Builds one domain's table from its distinct symbols and counts.
 * Returns 0 on success, -1 on bad arguments or allocation failure. */
int or_build_table(const or_params *P, int32_t dom, int64_t S, const uint64_t *keys, const uint64_t *counts,
                   or_table *t) {
  const int64_t K = (int64_t)1 << P->logK, M = P->M;
  if (M < 1 || M > K || dom < 0 || dom > 1) return -1;
  or_kc *r = (or_kc *)malloc(sizeof(or_kc) * (size_t)(S > 0 ? S : 1));
  uint64_t *c = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(K + 1));
  uint32_t *m = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(K + 1));
  uint32_t *mbest = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(K + 1));
  or_hent *heap = (or_hent *)malloc(sizeof(or_hent) * (size_t)(K + 1));
  double *L = (double *)malloc(sizeof(double) * (size_t)(M + 2));
  if (!r || !c || !m || !mbest || !heap || !L) {
    free(r), free(c), free(m), free(mbest), free(heap), free(L);
    return -1;
  }
  for (int64_t i = 0; i < S; ++i) r[i] = (or_kc){keys[i], counts[i]};
  qsort(r, (size_t)S, sizeof(or_kc), cmp_rank); /* step 1 */
  for (int64_t v = 1; v <= M + 1; ++v) L[v] = log2((double)v);
  L[0] = 0.0;
  uint64_t total = 0;
  for (int64_t i = 0; i < S; ++i) total += r[i].count;

  memset(t->kept_key, 0, sizeof(uint64_t) * (size_t)K);
  memset(t->kept_first, 0, sizeof(uint32_t) * (size_t)K);
  memset(t->kept_mult, 0, sizeof(uint32_t) * (size_t)K);
  memset(t->slot_key, 0, sizeof(uint64_t) * (size_t)K);
  memset(t->slot_digit, 0, sizeof(uint32_t) * (size_t)K);
  memset(t->slot_base, 0, sizeof(uint32_t) * (size_t)K);
  memset(t->slot_kind, 0, (size_t)K);
  t->nkept = 0;
  t->has_esc = 0;
  t->pad_esc = 0;
  t->pad_key = 0;
  t->esc_first = 0;
  t->esc_mult = 0;
  t->cost_bits = 0.0;
  if (S == 0) {
    free(r), free(c), free(m), free(mbest), free(heap), free(L);
    return 0;
  }

  const int64_t Tmax = S <= K ? S : K - 1; /* step 2 */
  double best_cost = 0.0;
  int64_t best_T = -1;
  uint64_t kept_total = 0; /* count of ranks < T */
  for (int64_t T = 0; T <= Tmax; ++T) {
    if (T > 0) kept_total += r[T - 1].count;
    const uint64_t E = total - kept_total;
    const int64_t ns = T + (E > 0 ? 1 : 0);
    for (int64_t s = 0; s < T; ++s) c[s] = r[s].count;
    if (E > 0) c[T] = E;
    allocate(ns, c, K, M, L, m, heap); /* step 3 */
    double cost = 0.0;                 /* step 4 */
    for (int64_t s = 0; s < ns; ++s) cost += (double)c[s] * ((double)P->logK - L[m[s]]);
    cost += (double)E * (double)P->raw_bits[dom];
    if (best_T < 0 || cost <= best_cost) {
      best_cost = cost;
      best_T = T;
      memcpy(mbest, m, sizeof(uint32_t) * (size_t)ns);
    }
  }

  /* step 5: slot layout */
  const int64_t T = best_T;
  uint64_t kept_best = 0;
  for (int64_t s = 0; s < T; ++s) kept_best += r[s].count;
  const uint64_t E = total - kept_best;
  uint32_t slot = 0;
  for (int64_t s = 0; s < T; ++s) {
    t->kept_key[s] = r[s].key;
    t->kept_first[s] = slot;
    t->kept_mult[s] = mbest[s];
    for (uint32_t dg = 0; dg < mbest[s]; ++dg, ++slot) {
      t->slot_key[slot] = r[s].key;
      t->slot_digit[slot] = dg;
      t->slot_base[slot] = mbest[s];
      t->slot_kind[slot] = 1;
    }
  }
  if (E > 0) {
    t->has_esc = 1;
    t->esc_first = slot;
    t->esc_mult = mbest[T];
    for (uint32_t dg = 0; dg < mbest[T]; ++dg, ++slot) {
      t->slot_key[slot] = 0;
      t->slot_digit[slot] = dg;
      t->slot_base[slot] = mbest[T];
      t->slot_kind[slot] = 2;
    }
  }
  t->nkept = T;
  t->cost_bits = best_cost;
  if (T > 0) {
    t->pad_key = r[0].key;
    t->pad_esc = 0;
  } else {
    t->pad_esc = 1;
  }
  free(r), free(c), free(m), free(mbest), free(heap), free(L);
  return 0;
}

/*
 * Optional slot permutation (Sec. IV-F "Tables in shared memory": symbols need
 * not occupy consecutive slots, and permuting them spreads bank accesses).
 * Seeded Fisher-Yates over the used slots with splitmix64 as the generator.
 * Digits stay attached to their slots; only positions move.
 * The paper prints no permuted table; the placement is pinned by a
 * hand-worked permutation from SplitMix64's published reference outputs
 * (a four-slot table and the stream encoded through it), besides the
 * generator's outputs themselves, the bijection of the used slots that
 * leaves the unused tail in place, and the round trip.
 */
static uint64_t splitmix64(uint64_t *s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* The first n outputs of the generator from `seed` (for pinning it against
 * the published reference outputs). */
void or_splitmix64_seq(uint64_t seed, int64_t n, uint64_t *out) {
  uint64_t s = seed;
  for (int64_t i = 0; i < n; ++i) out[i] = splitmix64(&s);
}

/* ------------------------------------------------------------------------ */
/* Symbol resolution                                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint32_t first, mult;
  int32_t esc;
} or_sym;

typedef struct {
  uint64_t key;
  int64_t idx;
} or_ki;

static int cmp_ki(const void *a, const void *b) {
  const or_ki *x = (const or_ki *)a, *y = (const or_ki *)b;
  return x->key < y->key ? -1 : (x->key > y->key ? 1 : 0);
}

typedef struct {
  const or_table *t;
  or_ki *sorted; /* kept keys sorted by key */
  /* per-slot placement of the digit when a permutation is active */
  uint32_t *perm; /* perm[canonical slot] = stored slot, or NULL */
} or_resolver;

static or_sym resolve(const or_resolver *R, uint64_t key) {
  const or_table *t = R->t;
  int64_t lo = 0, hi = t->nkept - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (R->sorted[mid].key == key) {
      int64_t s = R->sorted[mid].idx;
      return (or_sym){t->kept_first[s], t->kept_mult[s], 0};
    }
    if (R->sorted[mid].key < key)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return (or_sym){t->esc_first, t->esc_mult, 1};
}

static int resolver_init(or_resolver *R, const or_table *t) {
  R->t = t;
  R->perm = NULL;
  R->sorted = (or_ki *)malloc(sizeof(or_ki) * (size_t)(t->nkept > 0 ? t->nkept : 1));
  if (!R->sorted) return -1;
  for (int64_t s = 0; s < t->nkept; ++s) R->sorted[s] = (or_ki){t->kept_key[s], s};
  qsort(R->sorted, (size_t)t->nkept, sizeof(or_ki), cmp_ki);
  return 0;
}

static or_sym pad_sym(const or_table *t) {
  if (t->pad_esc) return (or_sym){t->esc_first, t->esc_mult, 1};
  return (or_sym){t->kept_first[0], t->kept_mult[0], 0};
}

/* ------------------------------------------------------------------------ */
/* pack / unpack (Sec. IV-D "Words in v")                                    */
/* ------------------------------------------------------------------------ */
/* The o words are read as one number with w_1 most significant,
 *   N = sum_q w_q W^(o-q),  and slot i_k = floor(N / K^(k-1)) mod K,
 * i.e. i_1 is the least significant slot.  Worked example: (1,1,1)_4 = 21
 * = (2)_8 (5)_8, so i_1 = 5 and i_2 = 2. */

static void unpack(const or_params *P, const uint32_t *w, uint32_t *slots) {
  u128 N = 0;
  for (int q = 0; q < P->o; ++q) N = (N << P->logW) | (u128)w[q];
  const u128 kmask = (((u128)1) << P->logK) - 1;
  for (int k = 0; k < P->l; ++k) slots[k] = (uint32_t)((N >> (P->logK * k)) & kmask);
}

static void pack(const or_params *P, const uint32_t *slots, uint32_t *w) {
  u128 N = 0;
  for (int k = P->l - 1; k >= 0; --k) N = (N << P->logK) | (u128)slots[k];
  const u128 wmask = (((u128)1) << P->logW) - 1;
  for (int q = 0; q < P->o; ++q) w[q] = (uint32_t)((N >> (P->logW * (P->o - 1 - q))) & wmask);
}

/* ------------------------------------------------------------------------ */
/* Unit encoder (Sec. IV-E: forward base pass, backward digit pass)          */
/* ------------------------------------------------------------------------ */
/*
 * Decoder program that the encoder mirrors (Algorithm 3 with the readings
 * below), for a unit of n items split into nseg = ceil(n / (l/spi)) segments:
 *   read w_1..w_o; d = 0; r = 1;
 *   per segment j:
 *     unpack the l slots and look up (symbol, digit, base) of each;
 *     escape point: for slots k = 1..l in order, a non-pad slot holding the
 *       escape symbol reads its raw words (a value's low word first);
 *     for check q = 1..f: append the digits of slots (q-1)g+1..qg, g = l/f,
 *       to the state (d = d*base + digit, r = r*base); then, unless j is the
 *       last segment, if r >= W extract w_q = d mod W, d = floor(d/W),
 *       r = floor(r/W), else read w_q;
 *     unless j is the last segment, read w_{f+1}..w_o.
 * Readings (the paper's worked example fixes them):
 *   - check q follows the digits of group q, as in the Sec. IV-D example
 *     (check after returned digit 1, then after returned digit 2) and the
 *     4-digit accumulation of Sec. IV-F "Positioning of checks";
 *   - the last segment performs no check and reads nothing (Sec. IV-F "end
 *     of row": the trailing words are known to be zero and are not stored);
 *   - pads fill the last segment (Sec. IV-F) and read no raw words.
 * Output: body = [w_1..w_o of segment 0] + words in read order.  The row
 * length n is stored by the caller in front of it.
 */

typedef struct {
  int64_t n, nseg;
  uint32_t *body;
  int64_t nbody;
  uint8_t *load; /* [nseg * f]: 1 if the decoder reads at check q */
  int32_t *nraw; /* [nseg]: raw words read at the escape point */
} or_unit;

static void unit_free(or_unit *u) {
  free(u->body);
  free(u->load);
  free(u->nraw);
  u->body = NULL;
  u->load = NULL;
  u->nraw = NULL;
}

/*
 * Chained units (an option beside the paper's one sequence per unit, the
 * "several rows per thread" of its conclusion): the units of one lane in C
 * consecutive slices form ONE dtANS sequence.  Each unit keeps its own
 * segments (its last segment padded), and only the chain's final segment is
 * "last" (no checks, no reads); every other segment, a unit's last segment
 * included, checks and reads as usual, so the decoder state runs on into the
 * lane's next unit and the unit's trailing state words are not stored.  With
 * one unit per chain this is exactly the per-unit encoder above.
 */
typedef struct {
  int nk;          /* units in the chain */
  int64_t S;       /* segments of the whole chain */
  int64_t n[64], nseg[64], seg0[64];
  int32_t cont[64]; /* 1: a later unit of the chain has items */
  uint32_t *body;  /* [w_1..w_o] + words in read order (empty when S = 0) */
  int64_t nbody;
  uint8_t *load;   /* [S * f] */
  int32_t *nraw;   /* [S] */
} or_chain;

static void chain_free(or_chain *c) {
  free(c->body);
  free(c->load);
  free(c->nraw);
  c->body = NULL;
  c->load = NULL;
  c->nraw = NULL;
}

/* syms[k]: n[k]*spi keys of unit k, item-major.  Returns 0, or -1
 * (allocation), -2 (a symbol needs the escape symbol but the table has
 * none), -3 (state invariant). */
static int encode_chain(const or_params *P, or_resolver *R /* [spi] */, const or_table *const *tabs, int nk,
                        const int64_t *n, const uint64_t *const *syms, or_chain *c) {
  const int l = P->l, o = P->o, f = P->f, spi = P->spi, ips = P->l / P->spi, g = P->l / P->f;
  const u128 W = ((u128)1) << P->logW;
  memset(c, 0, sizeof(*c));
  if (nk < 1 || nk > 64) return -1;
  c->nk = nk;
  int64_t S = 0;
  for (int k = 0; k < nk; ++k) {
    c->n[k] = n[k];
    c->nseg[k] = (n[k] + ips - 1) / ips;
    c->seg0[k] = S;
    S += c->nseg[k];
  }
  for (int k = 0; k < nk; ++k) {
    c->cont[k] = 0;
    for (int k2 = k + 1; k2 < nk; ++k2)
      if (n[k2] > 0) c->cont[k] = 1;
  }
  c->S = S;
  if (S == 0) return 0;
  or_sym *ss = (or_sym *)malloc(sizeof(or_sym) * (size_t)(S * l));
  int32_t *valid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(S * l));
  const uint64_t **segsym = (const uint64_t **)malloc(sizeof(uint64_t *) * (size_t)S);
  int64_t *segitem0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)S);
  c->load = (uint8_t *)calloc((size_t)(S * f), 1);
  c->nraw = (int32_t *)calloc((size_t)S, sizeof(int32_t));
  /* words: o initial + per segment at most (o + l*2) */
  int64_t cap = o + S * (int64_t)(o + 2 * l) + 4;
  uint32_t *out = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)cap);
  c->body = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)cap);
  if (!ss || !valid || !segsym || !segitem0 || !c->load || !c->nraw || !out || !c->body) {
    free(ss), free(valid), free(segsym), free(segitem0), free(out);
    chain_free(c);
    return -1;
  }
  /* segment G of the chain is segment j of unit k: items j*ips .. of unit k;
   * slots of items at or past n[k] are pads */
  for (int k = 0; k < nk; ++k)
    for (int64_t j = 0; j < c->nseg[k]; ++j) {
      const int64_t G = c->seg0[k] + j;
      segsym[G] = syms[k];
      segitem0[G] = j * ips;
      for (int p = 0; p < l; ++p) {
        const int64_t item = j * ips + p / spi;
        const int dom = p % spi;
        if (item < n[k]) {
          ss[G * l + p] = resolve(&R[dom], syms[k][item * spi + dom]);
          valid[G * l + p] = 1;
          if (ss[G * l + p].esc) {
            if (!tabs[dom]->has_esc) {
              free(ss), free(valid), free(segsym), free(segitem0), free(out);
              chain_free(c);
              return -2;
            }
            c->nraw[G] += P->raw_words[dom];
          }
        } else {
          ss[G * l + p] = pad_sym(tabs[dom]);
          valid[G * l + p] = 0;
        }
      }
    }

  /* base pass (forward): the radix alone decides every branch. */
  {
    u128 r = 1;
    for (int64_t G = 0; G + 1 < S; ++G)
      for (int q = 0; q < f; ++q) {
        for (int p = q * g; p < (q + 1) * g; ++p) r *= ss[G * l + p].mult;
        if (r >= W)
          r /= W; /* extraction */
        else
          c->load[G * f + q] = 1;
      }
  }

  /* digit pass (backward) */
  u128 d = 0;
  uint32_t nxt[8] = {0}, slots[16];
  int64_t no = 0;
  for (int64_t G = S - 1; G >= 0; --G) {
    const int last = (G == S - 1);
    if (!last)
      for (int q = o - 1; q >= f; --q) out[no++] = nxt[q];
    for (int q = f - 1; q >= 0; --q) {
      if (!last) {
        if (!c->load[G * f + q])
          d = d * W + nxt[q];
        else
          out[no++] = nxt[q];
      }
      for (int p = (q + 1) * g - 1; p >= q * g; --p) {
        const or_sym sy = ss[G * l + p];
        uint32_t dig = (uint32_t)(d % sy.mult);
        d /= sy.mult;
        slots[p] = sy.first + dig;
      }
    }
    /* escape raws of segment G, pushed in reverse */
    for (int p = l - 1; p >= 0; --p) {
      if (!valid[G * l + p] || !ss[G * l + p].esc) continue;
      const int dom = p % spi;
      const int64_t item = segitem0[G] + p / spi;
      const uint64_t key = segsym[G][item * spi + dom];
      for (int wq = P->raw_words[dom] - 1; wq >= 0; --wq) out[no++] = (uint32_t)(key >> (32 * wq));
    }
    if (R[0].perm || (spi > 1 && R[1].perm))
      for (int p = 0; p < l; ++p) {
        const or_resolver *rr = &R[p % spi];
        if (rr->perm) slots[p] = rr->perm[slots[p]];
      }
    pack(P, slots, nxt);
  }
  free(ss), free(valid), free(segsym), free(segitem0);
  if (d != 0) {
    free(out);
    chain_free(c);
    return -3;
  }
  for (int q = 0; q < o; ++q) c->body[q] = nxt[q];
  for (int64_t i = 0; i < no; ++i) c->body[o + i] = out[no - 1 - i];
  c->nbody = o + no;
  free(out);
  return 0;
}

/* One unit on its own: a chain of one unit. */
static int encode_unit(const or_params *P, or_resolver *R /* [spi] */, const or_table *const *tabs, int64_t n,
                       const uint64_t *syms, or_unit *u) {
  or_chain c;
  const uint64_t *sy[1] = {syms};
  memset(u, 0, sizeof(*u));
  u->n = n;
  const int rc = encode_chain(P, R, tabs, 1, &n, sy, &c);
  if (rc) return rc;
  u->nseg = c.S;
  u->body = c.body;
  u->nbody = c.nbody;
  u->load = c.load;
  u->nraw = c.nraw;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Warp interleaving (Sec. II "Interleaving for warps", Sec. IV-B)            */
/* ------------------------------------------------------------------------ */
/*
 * A slice holds up to `slice` consecutive units, one per lane.  The lanes'
 * words are merged in the order a lock-step decoder consumes them: program
 * points P_n, P_w1..P_wo, then for every segment j: E_j (each lane's raw
 * words of segment j, contiguous), C_j1..C_jf (lanes that read at check q),
 * U_j,f+1..U_j,o (lanes that are not in their last segment).  At each point
 * the participating lanes append their words in lane order, which is the
 * offset a warp gets from one ballot and two popcounts (Sec. IV-B).
 */

/* edst (NULL: raws stay in the stream) receives the escape points' words
 * instead, in the same order; *elen their count. */
static int64_t interleave_slice(const or_params *P, const or_unit *u, int nl, uint32_t *dst, uint32_t *edst,
                                int64_t *elen) {
  int64_t cur[64] = {0};
  int64_t pos = 0, maxseg = 0, epos = 0;
  for (int a = 0; a < nl; ++a) {
    dst[pos++] = (uint32_t)u[a].n;
    if (u[a].nseg > maxseg) maxseg = u[a].nseg;
  }
  for (int q = 0; q < P->o; ++q)
    for (int a = 0; a < nl; ++a)
      if (u[a].n > 0) dst[pos++] = u[a].body[cur[a]++];
  for (int64_t j = 0; j < maxseg; ++j) {
    for (int a = 0; a < nl; ++a)
      if (j < u[a].nseg)
        for (int32_t t = 0; t < u[a].nraw[j]; ++t) {
          if (edst)
            edst[epos++] = u[a].body[cur[a]++];
          else
            dst[pos++] = u[a].body[cur[a]++];
        }
    for (int q = 0; q < P->f; ++q)
      for (int a = 0; a < nl; ++a)
        if (j + 1 < u[a].nseg && u[a].load[j * P->f + q]) dst[pos++] = u[a].body[cur[a]++];
    for (int q = P->f; q < P->o; ++q)
      for (int a = 0; a < nl; ++a)
        if (j + 1 < u[a].nseg) dst[pos++] = u[a].body[cur[a]++];
  }
  if (elen) *elen = epos;
  return pos;
}

/*
 * Slice k of a chain (c[a]: lane a's chain, cur[a]: its body cursor, kept
 * across the chain's slices).  Program points: P_n, each lane's word
 * n | continues << 31 (continues: a later unit of the lane's chain has
 * items); at the chain's first slice P_w1..P_wo for lanes whose chain has
 * segments; then for every segment j of this slice's units E_j, C_j1..C_jf,
 * U_j as in interleave_slice, where only the chain's final segment skips the
 * checks and reads.  With chains of one slice this is interleave_slice.
 */
static int64_t interleave_chain_slice(const or_params *P, const or_chain *c, int nl, int k, int64_t *cur,
                                      uint32_t *dst, uint32_t *edst, int64_t *elen) {
  int64_t pos = 0, maxseg = 0, epos = 0;
  for (int a = 0; a < nl; ++a) {
    dst[pos++] = (uint32_t)c[a].n[k] | ((uint32_t)c[a].cont[k] << 31);
    if (c[a].nseg[k] > maxseg) maxseg = c[a].nseg[k];
  }
  if (k == 0)
    for (int q = 0; q < P->o; ++q)
      for (int a = 0; a < nl; ++a)
        if (c[a].S > 0) dst[pos++] = c[a].body[cur[a]++];
  for (int64_t j = 0; j < maxseg; ++j) {
    for (int a = 0; a < nl; ++a)
      if (j < c[a].nseg[k])
        for (int32_t t = 0; t < c[a].nraw[c[a].seg0[k] + j]; ++t) {
          if (edst)
            edst[epos++] = c[a].body[cur[a]++];
          else
            dst[pos++] = c[a].body[cur[a]++];
        }
    for (int q = 0; q < P->f; ++q)
      for (int a = 0; a < nl; ++a) {
        const int64_t G = c[a].seg0[k] + j;
        if (j < c[a].nseg[k] && G + 1 < c[a].S && c[a].load[G * P->f + q]) dst[pos++] = c[a].body[cur[a]++];
      }
    for (int q = P->f; q < P->o; ++q)
      for (int a = 0; a < nl; ++a)
        if (j < c[a].nseg[k] && c[a].seg0[k] + j + 1 < c[a].S) dst[pos++] = c[a].body[cur[a]++];
  }
  if (elen) *elen = epos;
  return pos;
}

/* ------------------------------------------------------------------------ */
/* Slice decoder: lock-step simulation of the lanes of one warp              */
/* ------------------------------------------------------------------------ */
/* Decodes one slice of nl units from stream words s[0..avail).  Outputs per
 * lane: n (out_n[a]) and the n*spi symbol keys at out_sym + out_off[a]*spi.
 * Returns the number of words consumed, or -1 on a corrupt stream (a read
 * past `avail`, an unused slot, an escape without raw bits). */
/* es (NULL: raws are in the stream) holds the slice's escape words, eavail of
 * them; *eused receives how many were read. */
static int64_t decode_slice(const or_params *P, const or_table *const *tabs, const uint32_t *perm_inv[2],
                            const uint32_t *s, int64_t avail, int nl, int64_t *out_n, const int64_t *out_off,
                            uint64_t *out_sym, const uint32_t *es, int64_t eavail, int64_t *eused) {
  const int l = P->l, o = P->o, f = P->f, spi = P->spi, ips = P->l / P->spi, g = P->l / P->f;
  const u128 W = ((u128)1) << P->logW;
  int64_t pos = 0, epos = 0;
  int64_t n[64], nseg[64], j;
  uint32_t w[64][8];
  u128 d[64], r[64];
  int64_t maxseg = 0;
#define RD(dst)                  \
  do {                           \
    if (pos >= avail) return -1; \
    (dst) = s[pos++];            \
  } while (0)
  for (int a = 0; a < nl; ++a) {
    uint32_t v;
    RD(v);
    n[a] = v;
    out_n[a] = v;
    nseg[a] = (n[a] + ips - 1) / ips;
    if (nseg[a] > maxseg) maxseg = nseg[a];
    d[a] = 0;
    r[a] = 1;
  }
  for (int q = 0; q < o; ++q)
    for (int a = 0; a < nl; ++a)
      if (n[a] > 0) RD(w[a][q]);
  for (j = 0; j < maxseg; ++j) {
    uint32_t slots[64][16];
    int32_t kind[64][16];
    uint32_t dig[64][16], base[64][16];
    /* unpack + lookups (independent per slot) */
    for (int a = 0; a < nl; ++a) {
      if (j >= nseg[a]) continue;
      unpack(P, w[a], slots[a]);
      for (int p = 0; p < l; ++p) {
        const int dom = p % spi;
        uint32_t sl = slots[a][p];
        if (perm_inv[dom]) sl = perm_inv[dom][sl];
        const or_table *t = tabs[dom];
        kind[a][p] = t->slot_kind[sl];
        if (kind[a][p] == 0) return -1;
        dig[a][p] = t->slot_digit[sl];
        base[a][p] = t->slot_base[sl];
        const int64_t item = j * ips + p / spi;
        if (item < n[a] && kind[a][p] == 1) out_sym[(out_off[a] + item) * spi + dom] = t->slot_key[sl];
      }
    }
    /* escape point E_j */
    for (int a = 0; a < nl; ++a) {
      if (j >= nseg[a]) continue;
      for (int p = 0; p < l; ++p) {
        const int dom = p % spi;
        const int64_t item = j * ips + p / spi;
        if (item >= n[a] || kind[a][p] != 2) continue;
        uint64_t key = 0;
        for (int wq = 0; wq < P->raw_words[dom]; ++wq) {
          uint32_t v;
          if (es) {
            if (epos >= eavail) return -1;
            v = es[epos++];
          } else {
            RD(v);
          }
          key |= ((uint64_t)v) << (32 * wq);
        }
        if (P->raw_words[dom] == 0) return -1;
        out_sym[(out_off[a] + item) * spi + dom] = key;
      }
    }
    /* checks C_j1..C_jf */
    for (int q = 0; q < f; ++q) {
      for (int a = 0; a < nl; ++a) {
        if (j >= nseg[a]) continue;
        for (int p = q * g; p < (q + 1) * g; ++p) {
          d[a] = d[a] * base[a][p] + dig[a][p];
          r[a] = r[a] * base[a][p];
        }
      }
      for (int a = 0; a < nl; ++a) {
        if (j + 1 >= nseg[a]) continue; /* last segment: no checks */
        if (r[a] >= W) {
          w[a][q] = (uint32_t)(d[a] % W);
          d[a] /= W;
          r[a] /= W;
        } else {
          RD(w[a][q]);
        }
      }
    }
    /* unconditional reads U_j */
    for (int q = f; q < o; ++q)
      for (int a = 0; a < nl; ++a)
        if (j + 1 < nseg[a]) RD(w[a][q]);
  }
#undef RD
  if (eused) *eused = epos;
  return pos;
}

/* Decodes slice `first ? 0 : k > 0` of a chain: like decode_slice, with the
 * lanes' state (w, d, r) carried in from the chain's previous slice; the
 * words P_n hold n | continues << 31; lanes read w_1..w_o at the chain's first
 * slice when they have items now or later; a unit's last segment checks and
 * reads unless the lane's chain ends there. */
static int64_t decode_chain_slice(const or_params *P, const or_table *const *tabs, const uint32_t *perm_inv[2],
                                  const uint32_t *s, int64_t avail, int nl, int first, uint32_t (*w)[8], u128 *d,
                                  u128 *r, int64_t *out_n, const int64_t *out_off, uint64_t *out_sym,
                                  const uint32_t *es, int64_t eavail, int64_t *eused) {
  const int l = P->l, o = P->o, f = P->f, spi = P->spi, ips = P->l / P->spi, g = P->l / P->f;
  const u128 W = ((u128)1) << P->logW;
  int64_t pos = 0, epos = 0;
  int64_t n[64], nseg[64], j;
  int cont[64];
  int64_t maxseg = 0;
#define RD(dst)                  \
  do {                           \
    if (pos >= avail) return -1; \
    (dst) = s[pos++];            \
  } while (0)
  for (int a = 0; a < nl; ++a) {
    uint32_t v;
    RD(v);
    n[a] = v & 0x7fffffffu;
    cont[a] = (int)(v >> 31);
    out_n[a] = n[a];
    nseg[a] = (n[a] + ips - 1) / ips;
    if (nseg[a] > maxseg) maxseg = nseg[a];
    if (first) {
      d[a] = 0;
      r[a] = 1;
    }
  }
  if (first)
    for (int q = 0; q < o; ++q)
      for (int a = 0; a < nl; ++a)
        if (n[a] > 0 || cont[a]) RD(w[a][q]);
  for (j = 0; j < maxseg; ++j) {
    uint32_t slots[64][16];
    int32_t kind[64][16];
    uint32_t dig[64][16], base[64][16];
    for (int a = 0; a < nl; ++a) {
      if (j >= nseg[a]) continue;
      unpack(P, w[a], slots[a]);
      for (int p = 0; p < l; ++p) {
        const int dom = p % spi;
        uint32_t sl = slots[a][p];
        if (perm_inv[dom]) sl = perm_inv[dom][sl];
        const or_table *t = tabs[dom];
        kind[a][p] = t->slot_kind[sl];
        if (kind[a][p] == 0) return -1;
        dig[a][p] = t->slot_digit[sl];
        base[a][p] = t->slot_base[sl];
        const int64_t item = j * ips + p / spi;
        if (item < n[a] && kind[a][p] == 1) out_sym[(out_off[a] + item) * spi + dom] = t->slot_key[sl];
      }
    }
    for (int a = 0; a < nl; ++a) {
      if (j >= nseg[a]) continue;
      for (int p = 0; p < l; ++p) {
        const int dom = p % spi;
        const int64_t item = j * ips + p / spi;
        if (item >= n[a] || kind[a][p] != 2) continue;
        uint64_t key = 0;
        for (int wq = 0; wq < P->raw_words[dom]; ++wq) {
          uint32_t v;
          if (es) {
            if (epos >= eavail) return -1;
            v = es[epos++];
          } else {
            RD(v);
          }
          key |= ((uint64_t)v) << (32 * wq);
        }
        if (P->raw_words[dom] == 0) return -1;
        out_sym[(out_off[a] + item) * spi + dom] = key;
      }
    }
    for (int q = 0; q < f; ++q) {
      for (int a = 0; a < nl; ++a) {
        if (j >= nseg[a]) continue;
        for (int p = q * g; p < (q + 1) * g; ++p) {
          d[a] = d[a] * base[a][p] + dig[a][p];
          r[a] = r[a] * base[a][p];
        }
      }
      for (int a = 0; a < nl; ++a) {
        if (j >= nseg[a] || (j + 1 >= nseg[a] && !cont[a])) continue; /* the chain's final segment */
        if (r[a] >= W) {
          w[a][q] = (uint32_t)(d[a] % W);
          d[a] /= W;
          r[a] /= W;
        } else {
          RD(w[a][q]);
        }
      }
    }
    for (int q = f; q < o; ++q)
      for (int a = 0; a < nl; ++a)
        if (j < nseg[a] && (j + 1 < nseg[a] || cont[a])) RD(w[a][q]);
  }
#undef RD
  if (eused) *eused = epos;
  return pos;
}

/* ------------------------------------------------------------------------ */
/* Plain symbol strings (the Sec. IV-D worked example)                       */
/* ------------------------------------------------------------------------ */

/* Encodes one symbol string with an explicit table (spi must be 1).  body
 * receives the stored words without n; returns the word count or < 0. */
int64_t or_encode_string(const or_params *P, const or_table *t, int64_t n, const uint64_t *syms, uint32_t *body,
                         int64_t cap, uint8_t *load_flags /* [nseg*f] or NULL */) {
  if (P->spi != 1) return -10;
  or_resolver R[1];
  if (resolver_init(&R[0], t)) return -1;
  const or_table *tabs[1] = {t};
  or_unit u;
  int rc = encode_unit(P, R, tabs, n, syms, &u);
  free(R[0].sorted);
  if (rc) return rc;
  if (u.nbody > cap) {
    unit_free(&u);
    return -4;
  }
  memcpy(body, u.body, sizeof(uint32_t) * (size_t)u.nbody);
  if (load_flags) memcpy(load_flags, u.load, (size_t)(u.nseg * P->f));
  int64_t nb = u.nbody;
  unit_free(&u);
  return nb;
}

/* Decodes [n] + body (one lane) back to n symbols; returns words used or < 0. */
int64_t or_decode_string(const or_params *P, const or_table *t, const uint32_t *stream, int64_t nwords,
                         uint64_t *syms_out, int64_t *n_out) {
  const or_table *tabs[1] = {t};
  const uint32_t *pinv[2] = {NULL, NULL};
  int64_t off = 0;
  return decode_slice(P, tabs, pinv, stream, nwords, 1, n_out, &off, syms_out, NULL, 0, NULL);
}

/* ------------------------------------------------------------------------ */
/* CSR layout: rows -> units (one unit per row, or split and reordered)      */
/* ------------------------------------------------------------------------ */
/*
 * unit_max_nnz U = 0: one unit per row, rows in their natural order (the
 * paper's mapping: a slice is 32 consecutive rows, Sec. II).
 * U > 0 (load balance, the remedy of Sec. V for irregular rows): a row of
 * length L becomes k = max(1, ceil(L/U)) units of near-equal length (the
 * first L mod k units one longer), each its own dtANS sequence whose first
 * delta is absolute.  With row_order = 1 the rows are then ordered by their
 * longest unit (descending, ties by row index; with U = 0 a row's one unit is
 * the whole row) so that a slice holds units of similar length; with
 * row_order = 0 the natural order is kept.  window > 0 (an option beside the
 * paper's format) restricts that ordering to consecutive blocks of `window`
 * rows: block b = rows [b*window, (b+1)*window) is ordered on its own and the
 * blocks keep their natural order, so a slice's rows stay within one block;
 * window <= 0 orders all rows as one block.
 */
typedef struct {
  int64_t len;
  int64_t row;
} or_lr;

static int cmp_lr(const void *a, const void *b) {
  const or_lr *x = (const or_lr *)a, *y = (const or_lr *)b;
  if (x->len != y->len) return x->len > y->len ? -1 : 1;
  return x->row < y->row ? -1 : (x->row > y->row ? 1 : 0);
}

/* Returns the number of units; fills unit_row/unit_start/unit_len when not
 * NULL (capacity = return value of a first call with NULL arrays). */
int64_t or_layout(int64_t m, const int64_t *row_ptr, int64_t U, int32_t row_order, int64_t window,
                  int64_t *unit_row, int64_t *unit_start, int64_t *unit_len) {
  or_lr *ord = (or_lr *)malloc(sizeof(or_lr) * (size_t)(m > 0 ? m : 1));
  if (!ord) return -1;
  for (int64_t i = 0; i < m; ++i) {
    const int64_t L = row_ptr[i + 1] - row_ptr[i];
    int64_t k = 1, ul = L;
    if (U > 0 && L > U) {
      k = (L + U - 1) / U;
      ul = (L + k - 1) / k;
    }
    ord[i] = (or_lr){ul, i};
  }
  if (row_order == 1) {
    const int64_t B = window > 0 ? window : (m > 0 ? m : 1);
    for (int64_t b = 0; b < m; b += B) {
      const int64_t e = b + B < m ? b + B : m;
      qsort(ord + b, (size_t)(e - b), sizeof(or_lr), cmp_lr);
    }
  }
  int64_t nu = 0;
  for (int64_t t = 0; t < m; ++t) {
    const int64_t i = ord[t].row;
    const int64_t L = row_ptr[i + 1] - row_ptr[i];
    const int64_t k = (U > 0 && L > U) ? (L + U - 1) / U : 1;
    const int64_t q = L / k, rem = L % k;
    int64_t st = 0;
    for (int64_t p = 0; p < k; ++p) {
      const int64_t len = q + (p < rem ? 1 : 0);
      if (unit_row) {
        unit_row[nu] = i;
        unit_start[nu] = st;
        unit_len[nu] = len;
      }
      st += len;
      ++nu;
    }
  }
  free(ord);
  return nu;
}

/* ------------------------------------------------------------------------ */
/* Matrix encode / decode                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t m, n, nnz, nunits, nslices, nwords;
  int64_t *unit_row, *unit_start, *unit_len;
  uint32_t *words;
  int64_t *slice_off; /* [nslices + 1] word offsets */
  /* escape_stream: the escape points' raw words, per slice, in their own array */
  int32_t esc_stream;
  int64_t nesc;
  uint32_t *esc_words;
  int64_t *esc_off; /* [nslices + 1] */
  /* per-unit statistics (for size checks) */
  int64_t *unit_words;  /* words stored for the unit, n word included */
  int64_t *unit_loads;  /* conditional reads */
  int64_t *unit_extr;   /* extractions */
  int64_t *unit_raw;    /* raw words */
  /* histogram of each domain (distinct keys, counts) */
  int64_t S[2];
  uint64_t *hkeys[2], *hcounts[2];
} or_matrix;

typedef struct {
  uint32_t col;
  int64_t k;
} or_ck;

static int cmp_ck(const void *a, const void *b) {
  const or_ck *x = (const or_ck *)a, *y = (const or_ck *)b;
  if (x->col != y->col) return x->col < y->col ? -1 : 1;
  return x->k < y->k ? -1 : (x->k > y->k ? 1 : 0); /* stable */
}

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Sorts each row's entries by column (stable: duplicates keep their input
 * order) into cols_s / vals_s.  Delta encoding (Sec. IV-A) works on these. */
void or_sort_rows(int64_t m, const int64_t *row_ptr, const uint32_t *cols, const uint64_t *vals, uint32_t *cols_s,
                  uint64_t *vals_s) {
  int64_t maxlen = 0;
  for (int64_t i = 0; i < m; ++i)
    if (row_ptr[i + 1] - row_ptr[i] > maxlen) maxlen = row_ptr[i + 1] - row_ptr[i];
  or_ck *tmp = (or_ck *)malloc(sizeof(or_ck) * (size_t)(maxlen > 0 ? maxlen : 1));
  for (int64_t i = 0; i < m; ++i) {
    const int64_t b = row_ptr[i], L = row_ptr[i + 1] - row_ptr[i];
    for (int64_t k = 0; k < L; ++k) tmp[k] = (or_ck){cols[b + k], k};
    qsort(tmp, (size_t)L, sizeof(or_ck), cmp_ck);
    for (int64_t k = 0; k < L; ++k) {
      cols_s[b + k] = tmp[k].col;
      vals_s[b + k] = vals[b + tmp[k].k];
    }
  }
  free(tmp);
}

/* Histogram of a key array: distinct keys ascending with counts. */
static int64_t histogram(int64_t nk, const uint64_t *k_in, uint64_t **keys, uint64_t **counts) {
  uint64_t *k = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nk > 0 ? nk : 1));
  memcpy(k, k_in, sizeof(uint64_t) * (size_t)nk);
  qsort(k, (size_t)nk, sizeof(uint64_t), cmp_u64);
  int64_t S = 0;
  for (int64_t i = 0; i < nk; ++i)
    if (i == 0 || k[i] != k[i - 1]) ++S;
  *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(S > 0 ? S : 1));
  *counts = (uint64_t *)calloc((size_t)(S > 0 ? S : 1), sizeof(uint64_t));
  int64_t s = -1;
  for (int64_t i = 0; i < nk; ++i) {
    if (i == 0 || k[i] != k[i - 1]) (*keys)[++s] = k[i];
    (*counts)[s] += 1;
  }
  free(k);
  return S;
}

void or_matrix_free(or_matrix *A) {
  if (!A) return;
  free(A->unit_row), free(A->unit_start), free(A->unit_len), free(A->words), free(A->slice_off);
  free(A->unit_words), free(A->unit_loads), free(A->unit_extr), free(A->unit_raw);
  free(A->esc_words), free(A->esc_off);
  for (int d = 0; d < 2; ++d) free(A->hkeys[d]), free(A->hcounts[d]);
  free(A);
}

/* Builds the per-unit symbol sequences: (delta, value) per item.  delta of a
 * unit's first item is its absolute column (Sec. IV-A: the first entry of a
 * row is an index, the rest are differences); duplicates give delta 0.  With
 * first_rel = 1 (an option beside the paper's format) the first delta is
 * instead the column minus the unit's row, modulo 2^32, so that a decoder
 * starting its running column at the row recovers the column by the same
 * 32-bit additions as for every other delta. */
static void unit_symbols(const int64_t *row_ptr, const uint32_t *cols_s, const uint64_t *vals_s, int64_t row,
                         int64_t start, int64_t len, int32_t first_rel, uint64_t *syms) {
  const int64_t b = row_ptr[row] + start;
  for (int64_t t = 0; t < len; ++t) {
    const uint32_t c = cols_s[b + t];
    const uint32_t prev = (t == 0) ? (first_rel ? (uint32_t)row : 0u) : cols_s[b + t - 1];
    syms[2 * t] = (uint64_t)(uint32_t)(c - prev);
    syms[2 * t + 1] = vals_s[b + t];
  }
}

/*
 * Encodes a CSR matrix into CSR-dtANS with the canonical parameters held in
 * P (spi must be 2).  vals are bit patterns (FP64, or FP32 zero-extended);
 * P->raw_words[1] is 2 for FP64 and 1 for FP32.  Tables are written to
 * tabs[0] (deltas) and tabs[1] (values); permutation seeds of 0 leave the
 * slot layout canonical; U, row_order and window give the rows-to-units
 * layout (see or_layout); first_rel selects the first-delta convention (see
 * unit_symbols); chain > 1 encodes each lane's units of `chain` consecutive
 * slices as one sequence (see encode_chain); esc_stream = 1 moves the escape
 * points' raw words into a separate array (esc_words, esc_off per slice; the
 * alternative of Sec. IV-F "Escaping rare values").  Returns the matrix or
 * NULL (*err set).
 */
or_matrix *or_encode_matrix(const or_params *P, int64_t m, int64_t n, const int64_t *row_ptr, const uint32_t *cols,
                            const uint64_t *vals, int64_t U, int32_t row_order, int64_t window, int32_t first_rel, int32_t chain,
                            int32_t esc_stream, or_table *tabD, or_table *tabV,
                            uint64_t perm_seed_d, uint64_t perm_seed_v, uint32_t *permD, uint32_t *permV,
                            int32_t *err) {
  *err = 0;
  if (P->spi != 2 || P->l % 2 || P->l % P->f || P->slice < 1 || P->slice > 64 || chain < 1 || chain > 64) {
    *err = -10;
    return NULL;
  }
  const int64_t nnz = row_ptr[m];
  or_matrix *A = (or_matrix *)calloc(1, sizeof(or_matrix));
  A->m = m, A->n = n, A->nnz = nnz;
  uint32_t *cols_s = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nnz > 0 ? nnz : 1));
  uint64_t *vals_s = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nnz > 0 ? nnz : 1));
  or_sort_rows(m, row_ptr, cols, vals, cols_s, vals_s);

  const int64_t nu = or_layout(m, row_ptr, U, row_order, window, NULL, NULL, NULL);
  A->nunits = nu;
  A->unit_row = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nu > 0 ? nu : 1));
  A->unit_start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nu > 0 ? nu : 1));
  A->unit_len = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nu > 0 ? nu : 1));
  or_layout(m, row_ptr, U, row_order, window, A->unit_row, A->unit_start, A->unit_len);

  /* histograms over all items of all units */
  int64_t maxlen = 0;
  for (int64_t a = 0; a < nu; ++a)
    if (A->unit_len[a] > maxlen) maxlen = A->unit_len[a];
  uint64_t *syms = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * maxlen + 2));
  {
    uint64_t *dk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nnz > 0 ? nnz : 1));
    uint64_t *vk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t t = 0;
    for (int64_t a = 0; a < nu; ++a) {
      unit_symbols(row_ptr, cols_s, vals_s, A->unit_row[a], A->unit_start[a], A->unit_len[a], first_rel, syms);
      for (int64_t i = 0; i < A->unit_len[a]; ++i, ++t) {
        dk[t] = syms[2 * i];
        vk[t] = syms[2 * i + 1];
      }
    }
    A->S[0] = histogram(nnz, dk, &A->hkeys[0], &A->hcounts[0]);
    A->S[1] = histogram(nnz, vk, &A->hkeys[1], &A->hcounts[1]);
    free(dk), free(vk);
  }
  if (or_build_table(P, 0, A->S[0], A->hkeys[0], A->hcounts[0], tabD) ||
      or_build_table(P, 1, A->S[1], A->hkeys[1], A->hcounts[1], tabV)) {
    *err = -1;
    free(cols_s), free(vals_s), free(syms);
    or_matrix_free(A);
    return NULL;
  }
  or_resolver R[2];
  resolver_init(&R[0], tabD);
  resolver_init(&R[1], tabV);
  /* optional slot permutations (off unless a seed is given) */
  uint32_t *perms[2] = {permD, permV};
  uint64_t seeds[2] = {perm_seed_d, perm_seed_v};
  or_table *tt[2] = {tabD, tabV};
  for (int d = 0; d < 2; ++d) {
    if (!seeds[d] || !perms[d]) continue;
    const int64_t K = (int64_t)1 << P->logK;
    int64_t used = 0;
    for (int64_t s = 0; s < K; ++s)
      if (tt[d]->slot_kind[s]) ++used;
    for (int64_t s = 0; s < K; ++s) perms[d][s] = (uint32_t)s;
    uint64_t st = seeds[d];
    for (int64_t i = used - 1; i > 0; --i) {
      int64_t jx = (int64_t)(splitmix64(&st) % (uint64_t)(i + 1));
      uint32_t tmp = perms[d][i];
      perms[d][i] = perms[d][jx];
      perms[d][jx] = tmp;
    }
    R[d].perm = perms[d];
  }
  const or_table *tabs[2] = {tabD, tabV};

  const int SW = P->slice;
  const int64_t ns = (nu + SW - 1) / SW;
  A->nslices = ns;
  A->slice_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ns + 1));
  A->unit_words = (int64_t *)calloc((size_t)(nu > 0 ? nu : 1), sizeof(int64_t));
  A->unit_loads = (int64_t *)calloc((size_t)(nu > 0 ? nu : 1), sizeof(int64_t));
  A->unit_extr = (int64_t *)calloc((size_t)(nu > 0 ? nu : 1), sizeof(int64_t));
  A->unit_raw = (int64_t *)calloc((size_t)(nu > 0 ? nu : 1), sizeof(int64_t));
  int64_t cap = 1024, pos = 0;
  A->words = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)cap);
  A->esc_stream = esc_stream ? 1 : 0;
  int64_t ecap = 1024, epos = 0;
  A->esc_words = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)ecap);
  A->esc_off = (int64_t *)calloc((size_t)(ns + 1), sizeof(int64_t));
  or_unit uu[64];
  if (chain > 1) {
    /* one sequence per lane over each run of `chain` slices */
    uint64_t *csyms[64][64];
    or_chain ch[64];
    for (int64_t c0 = 0; c0 < ns; c0 += chain) {
      const int nks = (int)(c0 + chain <= ns ? chain : ns - c0);
      int64_t cur[64] = {0};
      int nk_lane[64];
      int rc = 0;
      for (int a = 0; a < SW; ++a) {
        int64_t nn[64];
        int nk = 0;
        while (nk < nks && (c0 + nk) * SW + a < nu) {
          const int64_t ui = (c0 + nk) * SW + a;
          nn[nk] = A->unit_len[ui];
          csyms[a][nk] = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * A->unit_len[ui] + 2));
          unit_symbols(row_ptr, cols_s, vals_s, A->unit_row[ui], A->unit_start[ui], A->unit_len[ui], first_rel,
                       csyms[a][nk]);
          ++nk;
        }
        nk_lane[a] = nk;
        if (nk == 0) {
          memset(&ch[a], 0, sizeof(ch[a]));
          continue;
        }
        if (!rc) rc = encode_chain(P, R, tabs, nk, nn, (const uint64_t *const *)csyms[a], &ch[a]);
        else memset(&ch[a], 0, sizeof(ch[a]));
      }
      for (int k = 0; k < nks && !rc; ++k) {
        const int nl = (int)((c0 + k + 1) * SW <= nu ? SW : nu - (c0 + k) * SW);
        int64_t need = 0;
        for (int a = 0; a < nl; ++a) need += 1 + ch[a].nbody;
        while (pos + need > cap) {
          cap *= 2;
          A->words = (uint32_t *)realloc(A->words, sizeof(uint32_t) * (size_t)cap);
        }
        while (epos + need > ecap) {
          ecap *= 2;
          A->esc_words = (uint32_t *)realloc(A->esc_words, sizeof(uint32_t) * (size_t)ecap);
        }
        A->slice_off[c0 + k] = pos;
        A->esc_off[c0 + k] = epos;
        int64_t el = 0;
        pos += interleave_chain_slice(P, ch, nl, k, cur, A->words + pos, esc_stream ? A->esc_words + epos : NULL, &el);
        epos += el;
        /* per-unit statistics: the words the decoder reads for this unit */
        for (int a = 0; a < nl; ++a) {
          const int64_t ui = (c0 + k) * SW + a;
          int64_t raw = 0, loads = 0, extr = 0, uncond = 0;
          for (int64_t j = 0; j < ch[a].nseg[k]; ++j) {
            const int64_t G = ch[a].seg0[k] + j;
            raw += ch[a].nraw[G];
            if (G + 1 < ch[a].S) {
              for (int q = 0; q < P->f; ++q) {
                loads += ch[a].load[G * P->f + q];
                extr += !ch[a].load[G * P->f + q];
              }
              uncond += P->o - P->f;
            }
          }
          A->unit_raw[ui] = raw;
          A->unit_loads[ui] = loads;
          A->unit_extr[ui] = extr;
          A->unit_words[ui] = 1 + (k == 0 && ch[a].S > 0 ? P->o : 0) + raw + loads + uncond;
        }
      }
      for (int a = 0; a < SW; ++a) {
        for (int k = 0; k < nk_lane[a]; ++k) free(csyms[a][k]);
        chain_free(&ch[a]);
      }
      if (rc) {
        *err = rc;
        free(cols_s), free(vals_s), free(syms), free(R[0].sorted), free(R[1].sorted);
        or_matrix_free(A);
        return NULL;
      }
    }
    A->slice_off[ns] = pos;
    A->nwords = pos;
    A->esc_off[ns] = epos;
    A->nesc = epos;
    free(cols_s), free(vals_s), free(syms), free(R[0].sorted), free(R[1].sorted);
    return A;
  }
  for (int64_t sl = 0; sl < ns; ++sl) {
    const int nl = (int)((sl + 1) * SW <= nu ? SW : nu - sl * SW);
    int64_t need = 0;
    for (int a = 0; a < nl; ++a) {
      const int64_t ui = sl * SW + a;
      unit_symbols(row_ptr, cols_s, vals_s, A->unit_row[ui], A->unit_start[ui], A->unit_len[ui], first_rel, syms);
      int rc = encode_unit(P, R, tabs, A->unit_len[ui], syms, &uu[a]);
      if (rc) {
        *err = rc;
        for (int b = 0; b < a; ++b) unit_free(&uu[b]);
        free(cols_s), free(vals_s), free(syms), free(R[0].sorted), free(R[1].sorted);
        or_matrix_free(A);
        return NULL;
      }
      need += 1 + uu[a].nbody;
      A->unit_words[ui] = 1 + uu[a].nbody;
      int64_t raw = 0, loads = 0, extr = 0;
      for (int64_t j = 0; j < uu[a].nseg; ++j) {
        raw += uu[a].nraw[j];
        if (j + 1 < uu[a].nseg)
          for (int q = 0; q < P->f; ++q) {
            loads += uu[a].load[j * P->f + q];
            extr += !uu[a].load[j * P->f + q];
          }
      }
      A->unit_raw[ui] = raw;
      A->unit_loads[ui] = loads;
      A->unit_extr[ui] = extr;
    }
    while (pos + need > cap) {
      cap *= 2;
      A->words = (uint32_t *)realloc(A->words, sizeof(uint32_t) * (size_t)cap);
    }
    while (epos + need > ecap) {
      ecap *= 2;
      A->esc_words = (uint32_t *)realloc(A->esc_words, sizeof(uint32_t) * (size_t)ecap);
    }
    A->slice_off[sl] = pos;
    A->esc_off[sl] = epos;
    int64_t el = 0;
    pos += interleave_slice(P, uu, nl, A->words + pos, esc_stream ? A->esc_words + epos : NULL, &el);
    epos += el;
    for (int a = 0; a < nl; ++a) unit_free(&uu[a]);
  }
  A->slice_off[ns] = pos;
  A->nwords = pos;
  A->esc_off[ns] = epos;
  A->nesc = epos;
  free(cols_s), free(vals_s), free(syms), free(R[0].sorted), free(R[1].sorted);
  return A;
}

/* Accessors for the Python wrapper. */
int64_t or_matrix_get(const or_matrix *A, int32_t what) {
  switch (what) {
    case 0: return A->m;
    case 1: return A->n;
    case 2: return A->nnz;
    case 3: return A->nunits;
    case 4: return A->nslices;
    case 5: return A->nwords;
    case 6: return A->S[0];
    case 7: return A->S[1];
    case 8: return A->nesc;
    default: return -1;
  }
}

void or_matrix_copy(const or_matrix *A, uint32_t *words, int64_t *slice_off, int64_t *unit_row, int64_t *unit_start,
                    int64_t *unit_len, int64_t *unit_words, int64_t *unit_loads, int64_t *unit_extr,
                    int64_t *unit_raw) {
  memcpy(words, A->words, sizeof(uint32_t) * (size_t)A->nwords);
  memcpy(slice_off, A->slice_off, sizeof(int64_t) * (size_t)(A->nslices + 1));
  memcpy(unit_row, A->unit_row, sizeof(int64_t) * (size_t)A->nunits);
  memcpy(unit_start, A->unit_start, sizeof(int64_t) * (size_t)A->nunits);
  memcpy(unit_len, A->unit_len, sizeof(int64_t) * (size_t)A->nunits);
  memcpy(unit_words, A->unit_words, sizeof(int64_t) * (size_t)A->nunits);
  memcpy(unit_loads, A->unit_loads, sizeof(int64_t) * (size_t)A->nunits);
  memcpy(unit_extr, A->unit_extr, sizeof(int64_t) * (size_t)A->nunits);
  memcpy(unit_raw, A->unit_raw, sizeof(int64_t) * (size_t)A->nunits);
}

void or_matrix_copy_esc(const or_matrix *A, uint32_t *esc_words, int64_t *esc_off) {
  memcpy(esc_words, A->esc_words, sizeof(uint32_t) * (size_t)A->nesc);
  memcpy(esc_off, A->esc_off, sizeof(int64_t) * (size_t)(A->nslices + 1));
}

void or_matrix_hist(const or_matrix *A, int32_t dom, uint64_t *keys, uint64_t *counts) {
  memcpy(keys, A->hkeys[dom], sizeof(uint64_t) * (size_t)A->S[dom]);
  memcpy(counts, A->hcounts[dom], sizeof(uint64_t) * (size_t)A->S[dom]);
}

/*
 * Decodes slices [s0, s1) of an interleaved stream.  units of those slices
 * are written in unit order: out_n[u - 32*s0] and their symbols (delta,
 * value) item-major at out_sym + 2*(sum of earlier units' n).  Returns 0, or
 * -1 when the stream is corrupt, -2 when out_cap (items) is too small.
 */
int32_t or_decode_slices(const or_params *P, const or_table *tabD, const or_table *tabV, const uint32_t *permD_inv,
                         const uint32_t *permV_inv, const uint32_t *words, const int64_t *slice_off, int64_t nunits,
                         int64_t s0, int64_t s1, int32_t chain, const uint32_t *esc_words, const int64_t *esc_off,
                         int64_t *out_n, uint64_t *out_sym, int64_t out_cap) {
  const or_table *tabs[2] = {tabD, tabV};
  const uint32_t *pinv[2] = {permD_inv, permV_inv};
  const int SW = P->slice;
  int64_t items = 0;
  uint32_t cw[64][8];
  u128 cd[64], cr[64];
  memset(cw, 0, sizeof(cw));
  for (int a = 0; a < 64; ++a) cd[a] = 0, cr[a] = 1;
  if (SW > 64) return -1;
  for (int64_t sl = s0; sl < s1; ++sl) {
    const int nl = (int)((sl + 1) * SW <= nunits ? SW : nunits - sl * SW);
    const uint32_t *s = words + slice_off[sl];
    const int64_t avail = slice_off[sl + 1] - slice_off[sl];
    const uint32_t *es = esc_words ? esc_words + esc_off[sl] : NULL;
    const int64_t eavail = esc_words ? esc_off[sl + 1] - esc_off[sl] : 0;
    int64_t eused = 0;
    /* lengths first (the n point) to place each lane's output */
    int64_t off[64];
    int64_t acc = items;
    for (int a = 0; a < nl; ++a) {
      if (a >= avail) return -1;
      off[a] = acc;
      acc += chain > 1 ? (s[a] & 0x7fffffffu) : s[a];
    }
    if (acc > out_cap) return -2;
    int64_t used;
    if (chain > 1) {
      if (sl == s0 && sl % chain) return -1; /* decoding starts at a chain's first slice */
      used = decode_chain_slice(P, tabs, pinv, s, avail, nl, sl % chain == 0, cw, cd, cr, out_n + (sl - s0) * SW, off,
                                out_sym, es, eavail, &eused);
    } else {
      used = decode_slice(P, tabs, pinv, s, avail, nl, out_n + (sl - s0) * SW, off, out_sym, es, eavail, &eused);
    }
    if (es && eused != eavail) return -1;
    if (used != avail) return -1;
    items = acc;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Products (y = A x + beta y, Sec. III-A) with compensated arithmetic        */
/* ------------------------------------------------------------------------ */
/* Dot2 (Ogita, Rump and Oishi, 2005): TwoProduct through fma and TwoSum
 * (Knuth); the result is as accurate as if computed in twice the working
 * precision and then rounded.  A and x are given in FP64 (FP32 inputs are
 * widened exactly, so their products are exact). */

static inline void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}

static inline void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}

/* Y[:, b] = A X[:, b] + beta Y[:, b] for b < k (row-major n x k and m x k).
 * beta == 0 leaves Y unread.  abs_out (m x k, optional) = sum |a_ij x_jb|. */
void or_spmm_ref(int64_t m, const int64_t *row_ptr, const uint32_t *cols, const double *vals, int64_t k,
                 const double *X, double beta, const double *Y_in, double *Y_out, double *abs_out) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t b = 0; b < k; ++b) {
      double s = 0.0, c = 0.0, ab = 0.0, p, e, e2;
      for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
        const double a = vals[q], x = X[(int64_t)cols[q] * k + b];
        two_prod(a, x, &p, &e);
        two_sum(s, p, &s, &e2);
        c += e + e2;
        ab += fabs(a * x);
      }
      if (beta != 0.0) {
        two_prod(beta, Y_in[i * k + b], &p, &e);
        two_sum(s, p, &s, &e2);
        c += e + e2;
        ab += fabs(beta * Y_in[i * k + b]);
      }
      Y_out[i * k + b] = s + c;
      if (abs_out) abs_out[i * k + b] = ab;
    }
}

/* XG[:, b] = A^T G[:, b] + beta XG[:, b] (G is m x k, XG is n x k). */
void or_spmm_t_ref(int64_t m, int64_t n, const int64_t *row_ptr, const uint32_t *cols, const double *vals, int64_t k,
                   const double *G, double beta, const double *XG_in, double *XG_out, double *abs_out) {
  double *s = (double *)calloc((size_t)(n * k > 0 ? n * k : 1), sizeof(double));
  double *c = (double *)calloc((size_t)(n * k > 0 ? n * k : 1), sizeof(double));
  double *ab = (double *)calloc((size_t)(n * k > 0 ? n * k : 1), sizeof(double));
  for (int64_t i = 0; i < m; ++i)
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      const int64_t j = cols[q];
      for (int64_t b = 0; b < k; ++b) {
        double p, e, e2;
        two_prod(vals[q], G[i * k + b], &p, &e);
        two_sum(s[j * k + b], p, &s[j * k + b], &e2);
        c[j * k + b] += e + e2;
        ab[j * k + b] += fabs(vals[q] * G[i * k + b]);
      }
    }
  for (int64_t t = 0; t < n * k; ++t) {
    double v = s[t], cc = c[t], a = ab[t];
    if (beta != 0.0) {
      double p, e, e2;
      two_prod(beta, XG_in[t], &p, &e);
      two_sum(v, p, &v, &e2);
      cc += e + e2;
      a += fabs(beta * XG_in[t]);
    }
    XG_out[t] = v + cc;
    if (abs_out) abs_out[t] = a;
  }
  free(s), free(c), free(ab);
}

/* vals_grad[q] = sum_b G[i, b] X[j, b] for each stored entry q = (i, j) in the
 * given CSR order (the gradient of sum(G .* (A X)) with respect to a_ij). */
void or_vals_grad_ref(int64_t m, const int64_t *row_ptr, const uint32_t *cols, int64_t k, const double *G,
                      const double *X, double *out, double *abs_out) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
      const int64_t j = cols[q];
      double s = 0.0, c = 0.0, ab = 0.0, p, e, e2;
      for (int64_t b = 0; b < k; ++b) {
        two_prod(G[i * k + b], X[j * k + b], &p, &e);
        two_sum(s, p, &s, &e2);
        c += e + e2;
        ab += fabs(G[i * k + b] * X[j * k + b]);
      }
      out[q] = s + c;
      if (abs_out) abs_out[q] = ab;
    }
}

/* Brute force on a materialised dense matrix: y_i = sum_j A_ij x_j over all
 * columns j in ascending order (plain FP64 sums; used on small integer-valued
 * cases, where every sum is exact). */
void or_dense_spmv(int64_t m, int64_t n, const int64_t *row_ptr, const uint32_t *cols, const double *vals,
                   const double *x, double *y) {
  double *Ad = (double *)calloc((size_t)(m * n > 0 ? m * n : 1), sizeof(double));
  for (int64_t i = 0; i < m; ++i)
    for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) Ad[i * n + cols[q]] += vals[q];
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += Ad[i * n + j] * x[j];
    y[i] = s;
  }
  free(Ad);
}

// Host encoder of CSR-dtANS (arXiv 2603.01915, Sec. II "Encoding", Sec. IV).
//
// Pipeline: sort each row by column and delta-encode it (Sec. IV-A); split rows
// into units and order them (load-balancing layout, off by default); histogram
// the delta and value domains; build one coding table per domain (Sec. III-D,
// IV-C, IV-F "Escaping rare values"); encode every unit with a forward base
// pass and a backward digit pass (Sec. IV-E); interleave the 32 units of each
// slice in the order a warp reads them (Sec. II, IV-B).  Work is spread over
// host threads; the output is deterministic and independent of the thread
// count.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <thread>

#include "dtans_internal.h"

namespace dtans {
namespace {

int pick_threads(int requested) {
  if (requested > 0) return requested;
  unsigned hc = std::thread::hardware_concurrency();
  return hc ? (int)std::min(hc, 64u) : 4;
}

// Runs fn(begin, end, thread_index) over [0, count) in contiguous chunks.
void parallel_for(int64_t count, int nthreads, const std::function<void(int64_t, int64_t, int)> &fn) {
  if (count <= 0) return;
  int nt = (int)std::min<int64_t>(nthreads, std::max<int64_t>(1, count / 256 + 1));
  if (nt <= 1) {
    fn(0, count, 0);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    int64_t b = count * t / nt, e = count * (t + 1) / nt;
    th.emplace_back([=, &fn] { fn(b, e, t); });
  }
  for (auto &x : th) x.join();
}

// Open-addressing counter keyed by u64 (linear probing; separate occupancy).
struct Counter {
  std::vector<uint64_t> keys, counts;
  std::vector<uint8_t> used;
  uint64_t mask = 0;
  int64_t size = 0;
  static uint64_t mix(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
  }
  void init(int64_t cap) {
    uint64_t c = 16;
    while ((int64_t)c < 2 * cap) c <<= 1;
    keys.assign(c, 0);
    counts.assign(c, 0);
    used.assign(c, 0);
    mask = c - 1;
    size = 0;
  }
  void grow() {
    std::vector<uint64_t> k2 = std::move(keys), c2 = std::move(counts);
    std::vector<uint8_t> u2 = std::move(used);
    init((int64_t)(k2.size()));
    for (size_t i = 0; i < k2.size(); ++i)
      if (u2[i]) add(k2[i], c2[i]);
  }
  void add(uint64_t k, uint64_t c) {
    if ((uint64_t)(size + 1) * 2 > mask + 1) grow();
    uint64_t i = mix(k) & mask;
    while (used[i]) {
      if (keys[i] == k) {
        counts[i] += c;
        return;
      }
      i = (i + 1) & mask;
    }
    used[i] = 1;
    keys[i] = k;
    counts[i] = c;
    ++size;
  }
};

// Key -> kept-symbol index lookup for the (at most K) kept symbols.
struct SymIndex {
  std::vector<uint64_t> keys;
  std::vector<int32_t> idx;
  uint64_t mask = 0;
  void build(const Table &t) {
    uint64_t c = 16;
    while (c < 4 * (t.kept_key.size() + 1)) c <<= 1;
    keys.assign(c, 0);
    idx.assign(c, -1);
    mask = c - 1;
    for (size_t s = 0; s < t.kept_key.size(); ++s) {
      uint64_t i = Counter::mix(t.kept_key[s]) & mask;
      while (idx[i] >= 0) i = (i + 1) & mask;
      keys[i] = t.kept_key[s];
      idx[i] = (int32_t)s;
    }
  }
  int32_t find(uint64_t k) const {
    uint64_t i = Counter::mix(k) & mask;
    while (idx[i] >= 0) {
      if (keys[i] == k) return idx[i];
      i = (i + 1) & mask;
    }
    return -1;
  }
};

// Max-heap entry for the slot allocation: larger gain first, then lower index.
struct Gain {
  double g;
  int32_t s;
};
inline bool before(const Gain &a, const Gain &b) { return a.g > b.g || (a.g == b.g && a.s < b.s); }

struct GainHeap {
  std::vector<Gain> h;
  void clear() { h.clear(); }
  void push(Gain e) {
    h.push_back(e);
    size_t i = h.size() - 1;
    while (i > 0) {
      size_t p = (i - 1) >> 1;
      if (!before(h[i], h[p])) break;
      std::swap(h[i], h[p]);
      i = p;
    }
  }
  Gain pop() {
    Gain top = h[0];
    h[0] = h.back();
    h.pop_back();
    size_t i = 0, n = h.size();
    for (;;) {
      size_t a = 2 * i + 1, b = a + 1, best = i;
      if (a < n && before(h[a], h[best])) best = a;
      if (b < n && before(h[b], h[best])) best = b;
      if (best == i) break;
      std::swap(h[i], h[best]);
      i = best;
    }
    return top;
  }
};

// Water-filling of the K slots among `ns` symbols with counts c (rank order,
// escape last): every symbol gets one slot, then each further slot goes to the
// largest gain c*(log2(m+1) - log2(m)) with m < M.  Maximises sum c*log2(m).
void fill_slots(int ns, const uint64_t *c, const double *lg, uint32_t *m, GainHeap &heap) {
  heap.clear();
  for (int s = 0; s < ns; ++s) {
    m[s] = 1;
    heap.push({(double)c[s] * (lg[2] - lg[1]), s});
  }
  int spare = kK - ns;
  while (spare > 0 && !heap.h.empty()) {
    Gain top = heap.pop();
    uint32_t mm = ++m[top.s];
    --spare;
    if (mm < (uint32_t)kM) heap.push({(double)c[top.s] * (lg[mm + 1] - lg[mm]), top.s});
  }
}

}  // namespace

// Table construction.  The paper asks for P' close to P (minimal cross
// entropy, Sec. III-D), caps multiplicities at M (Sec. IV-C) and escapes rare
// symbols so that the expected total size is minimal (Sec. IV-F).  Search used:
// rank symbols by (count desc, key asc); for every kept-set size T (all S
// symbols when they fit in K slots, otherwise at most K - 1 plus the escape
// symbol) water-fill the slots and price the result as the coded bits (summed
// in rank order, escape last) plus raw bits of escaped entries; keep the
// cheapest, ties to the larger T.  Layout: kept symbols in rank order on
// consecutive slots, then the escape symbol.
void build_table(std::vector<std::pair<uint64_t, uint64_t>> kc, int raw_bits, int nthreads, Table &t) {
  t = Table();
  t.slot_key.assign(kK, 0);
  t.slot_digit.assign(kK, 0);
  t.slot_base.assign(kK, 0);
  t.slot_kind.assign(kK, 0);
  const int64_t S = (int64_t)kc.size();
  if (S == 0) return;
  std::sort(kc.begin(), kc.end(), [](const std::pair<uint64_t, uint64_t> &a, const std::pair<uint64_t, uint64_t> &b) {
    if (a.second != b.second) return a.second > b.second;
    return a.first < b.first;
  });
  double lg[kM + 2];
  lg[0] = 0.0;
  for (int v = 1; v <= kM + 1; ++v) lg[v] = std::log2((double)v);
  const int64_t Tmax = S <= kK ? S : kK - 1;
  std::vector<uint64_t> prefix(Tmax + 1, 0);  // prefix[T] = total count of ranks < T
  for (int64_t T = 1; T <= Tmax; ++T) prefix[T] = prefix[T - 1] + kc[T - 1].second;
  uint64_t total = 0;
  for (auto &p : kc) total += p.second;

  std::vector<double> cost(Tmax + 1);
  int nt = (int)std::min<int64_t>(pick_threads(nthreads), Tmax + 1);
  std::vector<std::thread> th;
  for (int w = 0; w < nt; ++w)
    th.emplace_back([&, w] {
      std::vector<uint64_t> c(kK + 1);
      std::vector<uint32_t> m(kK + 1);
      GainHeap heap;
      heap.h.reserve(kK + 1);
      for (int64_t T = w; T <= Tmax; T += nt) {
        const uint64_t E = total - prefix[T];
        const int ns = (int)T + (E > 0 ? 1 : 0);
        for (int64_t s = 0; s < T; ++s) c[s] = kc[s].second;
        if (E > 0) c[T] = E;
        fill_slots(ns, c.data(), lg, m.data(), heap);
        double bits = 0.0;
        for (int s = 0; s < ns; ++s) bits += (double)c[s] * ((double)kLogK - lg[m[s]]);
        bits += (double)E * (double)raw_bits;
        cost[T] = bits;
      }
    });
  for (auto &x : th) x.join();
  int64_t best = 0;
  for (int64_t T = 1; T <= Tmax; ++T)
    if (cost[T] <= cost[best]) best = T;

  const int64_t T = best;
  const uint64_t E = total - prefix[T];
  const int ns = (int)T + (E > 0 ? 1 : 0);
  std::vector<uint64_t> c(ns);
  std::vector<uint32_t> m(ns);
  for (int64_t s = 0; s < T; ++s) c[s] = kc[s].second;
  if (E > 0) c[T] = E;
  GainHeap heap;
  fill_slots(ns, c.data(), lg, m.data(), heap);
  uint32_t slot = 0;
  for (int64_t s = 0; s < T; ++s) {
    t.kept_key.push_back(kc[s].first);
    t.kept_first.push_back(slot);
    t.kept_mult.push_back(m[s]);
    for (uint32_t d = 0; d < m[s]; ++d, ++slot) {
      t.slot_key[slot] = kc[s].first;
      t.slot_digit[slot] = (uint16_t)d;
      t.slot_base[slot] = (uint16_t)m[s];
      t.slot_kind[slot] = 1;
    }
  }
  if (E > 0) {
    t.has_esc = true;
    t.esc_first = slot;
    t.esc_mult = m[T];
    for (uint32_t d = 0; d < m[T]; ++d, ++slot) {
      t.slot_digit[slot] = (uint16_t)d;
      t.slot_base[slot] = (uint16_t)m[T];
      t.slot_kind[slot] = 2;
    }
  }
  t.cost_bits = cost[best];
}

void make_permutation(Table &t, uint64_t seed) {
  t.perm.clear();
  if (!seed) return;
  uint32_t used = 0;
  for (int s = 0; s < kK; ++s) used += t.slot_kind[s] ? 1 : 0;
  t.perm.resize(kK);
  for (int s = 0; s < kK; ++s) t.perm[s] = (uint32_t)s;
  uint64_t st = seed;
  auto next = [&st]() {  // splitmix64
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (int64_t i = (int64_t)used - 1; i > 0; --i) {
    uint64_t j = next() % (uint64_t)(i + 1);
    std::swap(t.perm[i], t.perm[j]);
  }
}

namespace {

// A symbol as the coder sees it: its slot range and whether it is escaped.
struct Coded {
  uint32_t first, mult;
  bool esc;
};

// One lane's chain before interleaving: the lane's units of up to 64
// consecutive slices encoded as one dtANS sequence (a chain of one unit is the
// paper's one sequence per unit).  Each unit keeps its own segments, its last
// one padded; only the chain's final segment skips the checks and reads.
struct ChainOut {
  int nk = 0;                          // units in the chain
  uint32_t S = 0;                      // segments of the whole chain
  uint32_t n[64], nseg[64], seg0[64];  // per unit: entries, segments, first segment
  uint8_t cont[64];                    // per unit: a later unit of the chain has entries
  std::vector<uint32_t> body;          // w1..w3 of segment 0, then words in read order
  std::vector<uint8_t> reads;          // per segment: bit q set if check q reads
  std::vector<uint8_t> nraw;           // per segment: raw words at the escape point
};

struct Encoder {
  const Table *tab[2];
  SymIndex idx[2];
  int raw_v;  // raw words of an escaped value: 2 (FP64) or 1 (FP32)
  Coded pad[2];

  Coded code(int dom, uint64_t key) const {
    int32_t s = idx[dom].find(key);
    if (s >= 0) return {tab[dom]->kept_first[s], tab[dom]->kept_mult[s], false};
    return {tab[dom]->esc_first, tab[dom]->esc_mult, true};
  }

  // Unit k of the chain has n[k] entries with deltas dl[k] and value keys vk[k].
  void encode_chain(int nk, const uint32_t *n, const uint32_t *const *dl, const uint64_t *const *vk, ChainOut &u,
                    std::vector<Coded> &cs) const {
    u.nk = nk;
    u.body.clear();
    u.reads.clear();
    u.nraw.clear();
    uint32_t S = 0;
    for (int k = 0; k < nk; ++k) {
      u.n[k] = n[k];
      u.nseg[k] = (n[k] + kItemsPerSeg - 1) / kItemsPerSeg;
      u.seg0[k] = S;
      S += u.nseg[k];
    }
    for (int k = nk - 1, later = 0; k >= 0; --k) {
      u.cont[k] = (uint8_t)later;
      if (n[k]) later = 1;
    }
    u.S = S;
    if (S == 0) return;
    cs.resize((size_t)S * kSlots);
    u.reads.assign(S, 0);
    u.nraw.assign(S, 0);
    std::vector<uint32_t> seg_unit(S);
    for (int k = 0; k < nk; ++k)
      for (uint32_t j = 0; j < u.nseg[k]; ++j) {
        const uint32_t G = u.seg0[k] + j;
        seg_unit[G] = (uint32_t)k;
        for (int it = 0; it < kItemsPerSeg; ++it) {
          const uint32_t item = j * kItemsPerSeg + it;
          Coded *c = &cs[(size_t)G * kSlots + 2 * it];
          if (item < n[k]) {
            c[0] = code(0, dl[k][item]);
            c[1] = code(1, vk[k][item]);
            u.nraw[G] += (c[0].esc ? 1 : 0) + (c[1].esc ? raw_v : 0);
          } else {
            c[0] = pad[0];
            c[1] = pad[1];
          }
        }
      }
    // Forward base pass (Sec. IV-E): the radix alone decides each check.
    uint64_t r = 1;
    for (uint32_t G = 0; G + 1 < S; ++G)
      for (int q = 0; q < kChecks; ++q) {
        const Coded *c = &cs[(size_t)G * kSlots + q * kGroup];
        uint64_t R = (uint64_t)c[0].mult * c[1].mult * c[2].mult * c[3].mult;
        r *= R;  // r < 2^32 and R <= 2^32
        if (r >> 32)
          r >>= 32;
        else
          u.reads[G] |= (uint8_t)(1u << q);
      }
    // Backward digit pass (Sec. IV-E): choose slots and stored words.
    std::vector<uint32_t> rev;
    rev.reserve((size_t)S * 4 + 8);
    uint64_t d = 0;
    uint32_t nxt[3] = {0, 0, 0};
    uint32_t slot[kSlots];
    for (int64_t G = (int64_t)S - 1; G >= 0; --G) {
      const bool last = (G == (int64_t)S - 1);
      const Coded *c = &cs[(size_t)G * kSlots];
      if (!last) rev.push_back(nxt[2]);
      for (int q = kChecks - 1; q >= 0; --q) {
        if (!last) {
          if (u.reads[G] >> q & 1)
            rev.push_back(nxt[q]);
          else
            d = (d << 32) | nxt[q];
        }
        for (int p = q * kGroup + kGroup - 1; p >= q * kGroup; --p) {
          const uint32_t b = c[p].mult;
          slot[p] = c[p].first + (uint32_t)(d % b);
          d /= b;
        }
      }
      const int k = (int)seg_unit[G];
      const uint32_t j = (uint32_t)G - u.seg0[k];
      for (int p = kSlots - 1; p >= 0; --p) {
        const uint32_t item = j * kItemsPerSeg + p / 2;
        if (item >= n[k] || !c[p].esc) continue;
        if (p & 1) {
          const uint64_t key = vk[k][item];
          if (raw_v == 2) rev.push_back((uint32_t)(key >> 32));
          rev.push_back((uint32_t)key);
        } else {
          rev.push_back(dl[k][item]);
        }
      }
      for (int p = 0; p < kSlots; ++p) slot[p] = tab[p & 1]->stored(slot[p]);
      // pack: N = sum slot_k 2^(12k), w_1 the most significant word
      nxt[2] = slot[0] | slot[1] << 12 | slot[2] << 24;
      nxt[1] = slot[2] >> 8 | slot[3] << 4 | slot[4] << 16 | slot[5] << 28;
      nxt[0] = slot[5] >> 4 | slot[6] << 8 | slot[7] << 20;
    }
    // d == 0 here: the decoder starts from d = 0, and d < r holds throughout.
    u.body.reserve(3 + rev.size());
    u.body.push_back(nxt[0]);
    u.body.push_back(nxt[1]);
    u.body.push_back(nxt[2]);
    for (size_t i = rev.size(); i-- > 0;) u.body.push_back(rev[i]);
  }
};

// Merges slice k of the lanes' chains in warp read order (see dtans.h): the
// units' words n | continues << 31, at the chain's first slice the initial
// words of lanes whose chain has segments, then per segment the escape point,
// the conditional reads and the unconditional read (none after the chain's
// final segment).  cur: each lane's position in its body, across the chain.
// esc (null: in the stream) receives the escape points' raw words instead.
void interleave(const ChainOut *u, int nl, int k, size_t *cur, std::vector<uint32_t> &dst,
                std::vector<uint32_t> *esc) {
  std::vector<uint32_t> &raw = esc ? *esc : dst;
  uint32_t maxseg = 0;
  for (int a = 0; a < nl; ++a) {
    dst.push_back(u[a].n[k] | (uint32_t)u[a].cont[k] << 31);
    maxseg = std::max(maxseg, u[a].nseg[k]);
  }
  if (k == 0)
    for (int q = 0; q < kWords; ++q)
      for (int a = 0; a < nl; ++a)
        if (u[a].S) dst.push_back(u[a].body[cur[a]++]);
  for (uint32_t j = 0; j < maxseg; ++j) {
    for (int a = 0; a < nl; ++a)
      if (j < u[a].nseg[k])
        for (int t = 0; t < u[a].nraw[u[a].seg0[k] + j]; ++t) raw.push_back(u[a].body[cur[a]++]);
    for (int q = 0; q < kChecks; ++q)
      for (int a = 0; a < nl; ++a) {
        const uint32_t G = u[a].seg0[k] + j;
        if (j < u[a].nseg[k] && G + 1 < u[a].S && (u[a].reads[G] >> q & 1)) dst.push_back(u[a].body[cur[a]++]);
      }
    for (int a = 0; a < nl; ++a)
      if (j < u[a].nseg[k] && u[a].seg0[k] + j + 1 < u[a].S) dst.push_back(u[a].body[cur[a]++]);
  }
}

}  // namespace

dtans_status encode_matrix(int64_t m, int64_t n, const int64_t *row_ptr, const uint32_t *col_idx, const void *vals,
                           dtans_dtype dtype, const dtans_encode_opts &opts, dtans_handle_s &H) {
  if (m < 0 || n < 0 || m >= (1ll << 31) || n >= (1ll << 31)) return set_error(DTANS_ERR_ARG, "shape out of range");
  if (dtype != DTANS_F32 && dtype != DTANS_F64) return set_error(DTANS_ERR_ARG, "dtype must be F32 or F64");
  if (opts.unit_max_nnz < 0 || opts.row_order < 0 || opts.row_order > 1 || opts.first_delta < 0 ||
      opts.first_delta > 1 || opts.chain_slices < 0 || opts.chain_slices > 64 || opts.escape_stream < 0 ||
      opts.escape_stream > 1 || opts.order_window < 0)
    return set_error(DTANS_ERR_ARG, "bad encode options");
  if (!row_ptr) return set_error(DTANS_ERR_ARG, "row_ptr is null");
  if (row_ptr[0] != 0) return set_error(DTANS_ERR_ARG, "row_ptr[0] != 0");
  for (int64_t i = 0; i < m; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return set_error(DTANS_ERR_ARG, "row_ptr decreases");
  const int64_t nnz = row_ptr[m];
  if (nnz > 0 && (!col_idx || !vals)) return set_error(DTANS_ERR_ARG, "col_idx or vals is null");
  for (int64_t q = 0; q < nnz; ++q)
    if ((int64_t)col_idx[q] >= n) return set_error(DTANS_ERR_ARG, "column index out of range");
  const int nthreads = pick_threads(opts.num_threads);
  const bool f64 = dtype == DTANS_F64;
  H.m = m, H.n = n, H.nnz = nnz, H.dtype = dtype, H.opts = opts;

  // 1. sort rows by column (stable), values as bit patterns.
  std::vector<uint32_t> cols(nnz);
  std::vector<uint64_t> vk(nnz);
  parallel_for(m, nthreads, [&](int64_t b, int64_t e, int) {
    std::vector<int64_t> ord;
    for (int64_t i = b; i < e; ++i) {
      const int64_t s = row_ptr[i], L = row_ptr[i + 1] - row_ptr[i];
      bool sorted = true;
      for (int64_t k = 1; k < L; ++k)
        if (col_idx[s + k] < col_idx[s + k - 1]) {
          sorted = false;
          break;
        }
      ord.resize(L);
      for (int64_t k = 0; k < L; ++k) ord[k] = k;
      if (!sorted)
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int64_t a, int64_t c) { return col_idx[s + a] < col_idx[s + c]; });
      for (int64_t k = 0; k < L; ++k) {
        cols[s + k] = col_idx[s + ord[k]];
        if (f64) {
          uint64_t bits;
          std::memcpy(&bits, (const double *)vals + s + ord[k], 8);
          vk[s + k] = bits;
        } else {
          uint32_t bits;
          std::memcpy(&bits, (const float *)vals + s + ord[k], 4);
          vk[s + k] = bits;
        }
      }
    }
  });

  // 2. layout: rows -> units.
  const int64_t U = opts.unit_max_nnz;
  std::vector<uint32_t> order(m);
  std::vector<int64_t> nparts(m), ulen(m);
  for (int64_t i = 0; i < m; ++i) {
    const int64_t L = row_ptr[i + 1] - row_ptr[i];
    int64_t k = (U > 0 && L > U) ? (L + U - 1) / U : 1;
    nparts[i] = k;
    ulen[i] = (L + k - 1) / k;
    order[i] = (uint32_t)i;
  }
  if (opts.row_order == 1) {  // longest unit first (with U = 0, the whole row), ties by row
    // each block of order_window rows on its own (0: all rows are one block)
    const int64_t B = opts.order_window > 0 ? opts.order_window : std::max<int64_t>(m, 1);
    for (int64_t b = 0; b < m; b += B)
      std::stable_sort(order.begin() + b, order.begin() + std::min(m, b + B),
                       [&](uint32_t a, uint32_t c) { return ulen[a] > ulen[c]; });
  }
  int64_t nu = 0;
  for (int64_t i = 0; i < m; ++i) nu += nparts[i];
  H.nunits = nu;
  H.unit_row.resize(nu);
  H.unit_len.resize(nu);
  H.unit_pos.resize(nu);
  H.row_split.assign(m, 0);
  {
    int64_t u = 0;
    for (int64_t t = 0; t < m; ++t) {
      const uint32_t i = order[t];
      const int64_t L = row_ptr[i + 1] - row_ptr[i], k = nparts[i], q = L / k, rem = L % k;
      int64_t st = 0;
      for (int64_t p = 0; p < k; ++p, ++u) {
        const int64_t len = q + (p < rem ? 1 : 0);
        H.unit_row[u] = i;
        H.unit_len[u] = (uint32_t)len;
        H.unit_pos[u] = (uint64_t)(row_ptr[i] + st);
        st += len;
      }
      if (k > 1) H.row_split[i] = 1;
    }
  }
  H.identity_layout = true;
  for (int64_t u = 0; u < nu && H.identity_layout; ++u)
    if (H.unit_row[u] != (uint32_t)u) H.identity_layout = false;
  if (nu != m) H.identity_layout = false;
  H.any_split = nu != m;

  // 3. per-unit delta symbols: the first delta is the absolute column
  // (Sec. IV-A) or, with first_delta = 1, the column minus the unit's row
  // (modulo 2^32); the others are differences of consecutive columns.
  std::vector<uint32_t> deltas(nnz);
  parallel_for(nu, nthreads, [&](int64_t b, int64_t e, int) {
    for (int64_t u = b; u < e; ++u) {
      const uint64_t p = H.unit_pos[u];
      const uint32_t origin = opts.first_delta ? H.unit_row[u] : 0u;
      for (uint32_t t = 0; t < H.unit_len[u]; ++t)
        deltas[p + t] = t == 0 ? cols[p] - origin : cols[p + t] - cols[p + t - 1];
    }
  });

  // 4. histograms.
  for (int dom = 0; dom < 2; ++dom) {
    std::vector<Counter> part(nthreads);
    parallel_for(nnz, nthreads, [&](int64_t b, int64_t e, int t) {
      part[t].init(1024);
      for (int64_t q = b; q < e; ++q) part[t].add(dom == 0 ? (uint64_t)deltas[q] : vk[q], 1);
    });
    Counter all;
    all.init(1024);
    for (auto &p : part)
      for (size_t i = 0; i < p.keys.size(); ++i)
        if (p.used[i]) all.add(p.keys[i], p.counts[i]);
    std::vector<std::pair<uint64_t, uint64_t>> kc;
    kc.reserve(all.size);
    for (size_t i = 0; i < all.keys.size(); ++i)
      if (all.used[i]) kc.push_back({all.keys[i], all.counts[i]});
    build_table(std::move(kc), dom == 0 ? 32 : (f64 ? 64 : 32), nthreads, H.tab[dom]);
  }
  make_permutation(H.tab[0], opts.perm_seed_delta);
  make_permutation(H.tab[1], opts.perm_seed_value);

  // 5. encode + interleave, slice by slice.
  Encoder enc;
  enc.raw_v = f64 ? 2 : 1;
  for (int dom = 0; dom < 2; ++dom) {
    enc.tab[dom] = &H.tab[dom];
    enc.idx[dom].build(H.tab[dom]);
    const Table &t = H.tab[dom];
    if (!t.kept_key.empty())
      enc.pad[dom] = {t.kept_first[0], t.kept_mult[0], false};
    else
      enc.pad[dom] = {t.esc_first, std::max<uint32_t>(1, t.esc_mult), true};
  }
  const int64_t ns = (nu + kSlice - 1) / kSlice;
  H.nslices = ns;
  const int64_t C = std::max(1, opts.chain_slices);  // slices per chain
  const int64_t nchains = (ns + C - 1) / C;
  std::vector<std::vector<uint32_t>> sw(ns), se(opts.escape_stream ? ns : 0);
  std::atomic<int> bad{0};
  parallel_for(nchains, nthreads, [&](int64_t b, int64_t e, int) {
    std::vector<ChainOut> lanes(kSlice);
    std::vector<Coded> cs;
    for (int64_t c = b; c < e; ++c) {
      const int64_t s0 = c * C, nks = std::min<int64_t>(C, ns - s0);
      for (int a = 0; a < kSlice; ++a) {
        uint32_t nn[64];
        const uint32_t *dl[64];
        const uint64_t *vv[64];
        int nk = 0;
        for (; nk < nks && (s0 + nk) * kSlice + a < nu; ++nk) {
          const int64_t u = (s0 + nk) * kSlice + a;
          const uint64_t p = H.unit_pos[u];
          nn[nk] = H.unit_len[u];
          dl[nk] = deltas.data() + p;
          vv[nk] = vk.data() + p;
        }
        enc.encode_chain(nk, nn, dl, vv, lanes[a], cs);
      }
      size_t cur[kSlice] = {0};
      for (int64_t k = 0; k < nks; ++k) {
        const int nl = (int)std::min<int64_t>(kSlice, nu - (s0 + k) * kSlice);
        interleave(lanes.data(), nl, (int)k, cur, sw[s0 + k], opts.escape_stream ? &se[s0 + k] : nullptr);
      }
    }
  });
  if (bad.load()) return set_error(DTANS_ERR_CORRUPT, "encoder invariant violated");
  H.esc_words.clear();
  H.esc_off.clear();
  if (opts.escape_stream) {
    H.esc_off.assign(ns + 1, 0);
    for (int64_t s = 0; s < ns; ++s) H.esc_off[s + 1] = H.esc_off[s] + se[s].size();
    H.esc_words.reserve(H.esc_off[ns]);
    for (int64_t s = 0; s < ns; ++s) H.esc_words.insert(H.esc_words.end(), se[s].begin(), se[s].end());
  }
  H.slice_off.assign(ns + 1, 0);
  for (int64_t s = 0; s < ns; ++s) H.slice_off[s + 1] = H.slice_off[s] + sw[s].size();
  H.nwords = (int64_t)H.slice_off[ns];
  H.words.resize(H.nwords);
  parallel_for(ns, nthreads, [&](int64_t b, int64_t e, int) {
    for (int64_t s = b; s < e; ++s) {
      if (!sw[s].empty()) std::memcpy(H.words.data() + H.slice_off[s], sw[s].data(), sw[s].size() * 4);
      std::vector<uint32_t>().swap(sw[s]);
    }
  });
  build_table_image(H);
  return DTANS_OK;
}

int64_t table_image_bytes(dtans_dtype dt) { return (int64_t)kK * 8 + (int64_t)kK * (dt == DTANS_F64 ? 16 : 8); }

namespace {

// Integer coefficients of an FP64 value table: every kept value is written
// as c * 2^e with one exponent e for the whole table and integers
// |c| <= kIntCoefMax (zero has c = 0).  Returns false when some kept value
// is not finite or needs a larger c; else coef[slot] holds c for kept slots
// (0 for escape and unused slots) and *exp the common e.
constexpr int64_t kIntCoefMax = (1 << 15) - 1;

bool integer_coefficients(const Table &t, std::vector<int32_t> &coef, int32_t *exp) {
  struct Dec {
    int64_t m;  // odd (or zero) signed integer
    int32_t e;  // value = m * 2^e
  };
  std::vector<Dec> dec(t.kept_key.size());
  int32_t emin = INT32_MAX;
  for (size_t q = 0; q < t.kept_key.size(); ++q) {
    const uint64_t b = t.kept_key[q];
    const uint32_t be = (uint32_t)(b >> 52) & 0x7ffu;
    const uint64_t frac = b & ((1ull << 52) - 1);
    if (be == 0x7ffu) return false;  // infinity or NaN
    uint64_t m = be ? (frac | 1ull << 52) : frac;
    int32_t e = be ? (int32_t)be - 1075 : -1074;
    if (m == 0) {
      dec[q] = {0, 0};
      continue;
    }
    while (!(m & 1)) {
      m >>= 1;
      ++e;
    }
    if (m > (uint64_t)kIntCoefMax) return false;
    dec[q] = {(b >> 63) ? -(int64_t)m : (int64_t)m, e};
    emin = std::min(emin, e);
  }
  if (emin == INT32_MAX) emin = 0;  // no nonzero kept value
  coef.assign(kK, 0);
  for (size_t q = 0; q < dec.size(); ++q) {
    int64_t c = dec[q].m;
    if (c != 0) {
      const int32_t sh = dec[q].e - emin;
      if (sh > 15) return false;
      c *= (int64_t)1 << sh;
      if (c > kIntCoefMax || c < -kIntCoefMax) return false;
    }
    for (uint32_t s = t.kept_first[q]; s < t.kept_first[q] + t.kept_mult[q]; ++s) coef[t.stored(s)] = (int32_t)c;
  }
  *exp = emin;
  return true;
}

}  // namespace

// Device image of both tables, indexed by stored slot:
//   deltas: uint2 {delta, meta}; values: FP32 uint2 {bits, meta},
//   FP64 uint4 {lo, hi, meta, c};  meta = digit | flags | base << 16, and c
//   the slot's integer coefficient when the whole FP64 table has integer
//   coefficients (see integer_coefficients; else 0).  Also records whether
//   the integer-coefficient products apply and the longest unit.
void build_table_image(dtans_handle_s &H) {
  const bool f64 = H.dtype == DTANS_F64;
  H.table_image.assign((size_t)table_image_bytes(H.dtype), 0);
  uint32_t *D = (uint32_t *)H.table_image.data();
  uint32_t *V = D + 2 * kK;
  H.max_unit_len = 0;
  for (uint32_t L : H.unit_len) H.max_unit_len = std::max<int64_t>(H.max_unit_len, L);
  {
    bool full[2] = {false, false};  // some used slot belongs to a symbol of multiplicity M
    for (int dom = 0; dom < 2; ++dom)
      for (int s = 0; s < kK && !full[dom]; ++s) full[dom] = H.tab[dom].slot_kind[s] && H.tab[dom].slot_base[s] == kM;
    H.radix_w = full[0] && full[1];
  }
  std::vector<int32_t> coef;
  H.int_exp = 0;
  H.int_ok = f64 && integer_coefficients(H.tab[1], coef, &H.int_exp);
  for (int dom = 0; dom < 2; ++dom) {
    const Table &t = H.tab[dom];
    for (int s = 0; s < kK; ++s) {
      const uint32_t st = t.stored((uint32_t)s);
      uint32_t meta;
      if (t.slot_kind[s] == 0)
        meta = kMetaUnused | 1u << 16;  // base 1, digit 0: harmless if a corrupt stream selects it
      else
        meta = (uint32_t)t.slot_digit[s] | (uint32_t)t.slot_base[s] << 16 | (t.slot_kind[s] == 2 ? kMetaEsc : 0u);
      const uint64_t key = t.slot_key[s];
      if (dom == 0) {
        D[2 * st] = (uint32_t)key;
        D[2 * st + 1] = meta;
      } else if (f64) {
        V[4 * st] = (uint32_t)key;
        V[4 * st + 1] = (uint32_t)(key >> 32);
        V[4 * st + 2] = meta;
        V[4 * st + 3] = H.int_ok ? (uint32_t)coef[st] : 0u;
      } else {
        V[2 * st] = (uint32_t)key;
        V[2 * st + 1] = meta;
      }
    }
  }
}

}  // namespace dtans

// Internal declarations shared by the host encoder, the handle code and the
// CUDA launchers of the CSR-dtANS library.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "dtans.h"

namespace dtans {

// Fixed CSR-dtANS parameters (arXiv 2603.01915, Sec. IV-D): K = 2^12 slots per
// table, W = 2^32, M = 2^8, l = 8 slots (4 nonzeros) per segment unpacked from
// o = 3 words, f = 2 conditional checks, each after a group of g = 4 slots.
constexpr int kLogK = 12;
constexpr int kK = 1 << kLogK;
constexpr int kM = 256;
constexpr int kSlots = 8;
constexpr int kWords = 3;
constexpr int kChecks = 2;
constexpr int kGroup = 4;
constexpr int kItemsPerSeg = 4;
constexpr int kSlice = 32;

// Meta word of a device table entry: digit (bits 0-7) | flags | base << 16
// (base = the symbol's multiplicity, 1..256).
constexpr uint32_t kMetaEsc = 1u << 15;
constexpr uint32_t kMetaUnused = 1u << 14;

// Host form of one domain's coding table, in canonical slot order.
struct Table {
  std::vector<uint64_t> slot_key;
  std::vector<uint16_t> slot_digit, slot_base;
  std::vector<uint8_t> slot_kind;  // 0 unused, 1 kept, 2 escape
  std::vector<uint64_t> kept_key;  // rank order
  std::vector<uint32_t> kept_first, kept_mult;
  bool has_esc = false;
  uint32_t esc_first = 0, esc_mult = 0;
  double cost_bits = 0.0;
  std::vector<uint32_t> perm;  // canonical slot -> stored slot; empty = identity
  uint32_t stored(uint32_t s) const { return perm.empty() ? s : perm[s]; }
};

// Builds a table from (key, count) pairs (any order).  raw_bits prices an
// escaped symbol.  nthreads parallelises the search over kept-set sizes.
void build_table(std::vector<std::pair<uint64_t, uint64_t>> kc, int raw_bits, int nthreads, Table &t);

// Applies a seeded Fisher-Yates shuffle of the used slots (splitmix64).
void make_permutation(Table &t, uint64_t seed);

struct HostIO;  // device buffers, streams and events of dtans_spmv_host (host_io.cpp)

}  // namespace dtans

struct dtans_handle_s {
  int64_t m = 0, n = 0, nnz = 0, nunits = 0, nslices = 0, nwords = 0;
  dtans_dtype dtype = DTANS_F64;
  dtans_encode_opts opts{};
  bool identity_layout = true;  // unit u is row u
  bool any_split = false;       // some row spans several units
  bool radix_w = true;          // both tables hold a symbol of multiplicity M (a check group can have radix W)

  // host data
  std::vector<uint32_t> words;
  std::vector<uint64_t> slice_off;
  std::vector<uint32_t> unit_row;   // row of each unit; bit 31 of the device copy marks split rows
  std::vector<uint32_t> unit_len;
  std::vector<uint64_t> unit_pos;   // sorted-CSR position of each unit's first entry
  std::vector<uint32_t> esc_words;  // separate escape stream (escape_stream = 1), else empty
  std::vector<uint64_t> esc_off;    // its offset per slice (nslices + 1), else empty
  std::vector<uint8_t> row_split;   // per row: 1 if the row has more than one unit
  dtans::Table tab[2];
  std::vector<uint8_t> table_image; // device image: delta table then value table

  // device data
  bool uploaded = false;
  int device = -1;
  uint32_t *d_words = nullptr;
  uint64_t *d_slice_off = nullptr;
  uint8_t *d_tables = nullptr;
  uint32_t *d_unit_row = nullptr;   // null for the identity layout
  uint64_t *d_unit_pos = nullptr;
  uint32_t *d_esc_words = nullptr;   // separate escape stream, or null
  uint64_t *d_esc_off = nullptr;
  int32_t *d_err = nullptr;
  uint16_t *d_vrank = nullptr;      // codebook gradient: bin of each stored value slot (built on first use)
  uint32_t *d_warp_slice[2] = {nullptr, nullptr};  // per-warp slice ranges (32- and 16-warp CTAs)
  int64_t warp_slice_n[2] = {0, 0};                 // warps those ranges were computed for
  int32_t grid = 0, block = 0;       // 0 = automatic
  int32_t warps = 0;                 // warps per CTA of the single-vector persistent kernel (0 = automatic)
  int32_t scatter = 0;               // dtans_set_scatter: 0 one atomic per entry, 1 warp-aggregated
  int32_t tile_policy = 0;           // 0: 8-column persistent tiles; 1: one 16-column pass when >= 16 columns are left
  bool use_persistent = true;        // k = 1 products use the persistent ring kernel
  dtans::HostIO *host_io = nullptr;  // created by the first dtans_spmv_host call

  // Integer-coefficient products (FP64 tables whose kept values are small
  // integers times one power of two; see spmv.cu)
  bool int_ok = false;               // the value table has integer coefficients
  int32_t int_exp = 0;               // their common power of two
  int64_t max_unit_len = 0;          // entries of the longest unit
  int32_t accumulate = 0;            // dtans_set_accumulate: 0 FP64 fused multiply-adds, 1 integer coefficients
  void *d_xfix = nullptr;            // fixed-point copy of x (n x 16 bytes), allocated on first use
  int64_t xfix_n = 0;
  int32_t *d_xexp = nullptr;         // largest exponent of x, written by the prepass
};

namespace dtans {

dtans_status set_error(dtans_status st, const std::string &msg);
dtans_status encode_matrix(int64_t m, int64_t n, const int64_t *row_ptr, const uint32_t *col_idx, const void *vals,
                           dtans_dtype dtype, const dtans_encode_opts &opts, dtans_handle_s &H);
void build_table_image(dtans_handle_s &H);
int64_t table_image_bytes(dtans_dtype dt);
// Persistent decode-fused products (spmv.cu) for one tile of kt columns
// (c0 .. c0 + kt - 1 of row-major blocks with leading dimension ld);
// beta_mode 0: y = Ax, 1: y += Ax, 2: y = Ax + beta y (split rows add
// atomically into a pre-scaled y).  persistent_tile_ok tells whether a tile
// qualifies (kt in {1, 2, 4, 8}, and 16 or 32 for FP32, filling 16-byte
// vectors, aligned blocks).
bool persistent_tile_ok(const dtans_handle_s &H, int kt, const void *x, const void *y, int64_t ld, int64_t c0);
// Whether single-vector products of the handle use the integer-coefficient
// kernels (spmv.cu).
bool int_products(const dtans_handle_s &H);
// Releases the state of dtans_spmv_host (waits for its copies first).
void free_host_io(dtans_handle_s &H);
dtans_status spmv_persistent(dtans_handle_s &H, int kt, const void *x, void *y, int64_t ld, int64_t c0, double beta,
                             int32_t beta_mode, void *stream);
// The value gradient of 32 FP32 columns c0 .. c0 + 31 with the persistent
// kernel (FP32 handles without a separate escape stream; G and X rows 16-byte
// aligned at c0): out[p] (sorted-CSR order) = <G[row, cols], X[col, cols]>,
// added to out when acc_out.
dtans_status vals_grad_persistent(dtans_handle_s &H, const void *G, const void *X, void *out, int64_t ld, int64_t c0,
                                  bool acc_out, void *stream);
// The codebook gradient of 32 FP32 columns c0 .. c0 + 31 with the persistent
// kernel (same conditions): out[vrank[slot]] += <G[row, cols], X[col, cols]>
// for each entry's value-table slot; nbins = kept symbols + 1 (<= K + 1).
dtans_status codebook_grad_persistent(dtans_handle_s &H, const void *G, const void *X, void *out, int64_t ld,
                                      int64_t c0, const uint16_t *vrank, int32_t nbins, void *stream);

}  // namespace dtans

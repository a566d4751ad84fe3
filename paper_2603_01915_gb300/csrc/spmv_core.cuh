// Per-warp machinery of the persistent CSR-dtANS decoder, shared by the
// single-matrix SpMV (spmv.cu) and the batched SpMV (batch.cu): the warp's
// bulk-copy ring of stream words and the segment decoder (Algorithm 3 with the
// readings of Sec. IV-D/IV-F).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "decode_common.cuh"
#include "dtans_internal.h"


namespace dtans {
namespace core {

using namespace dev;

constexpr uint32_t kNumChunks = 8;         // ring chunks (one mbarrier each) per warp
constexpr uint32_t kSpinLimit = 1u << 20;  // polls per wait before giving up

// Ring of kRingWords words (4 KB) per warp.  A slice whose words fit the ring
// (up to ~900 words) is fetched whole and decoded without ring checks; the
// 512-byte chunks keep the waits and copies per slice few.  Measured against a
// 2 KB ring of 256-byte chunks on GB300: 4.5% faster on the 27-point stencil,
// and it keeps every slice of the power-law layouts resident.
constexpr uint32_t kRingWords = 1024;

// Warp-private ring of RW stream words in kNumChunks chunks.  All lanes hold
// the same state; lane 0 issues the copies.
template <uint32_t RW>
struct Ring {
  static constexpr uint32_t kChunk = RW / kNumChunks;  // words per bulk copy
  static constexpr uint32_t kMask = RW - 1;
  static_assert((RW & kMask) == 0 && kChunk % 4 == 0, "ring of whole 16-byte chunks");
  const uint32_t *src;  // global address of word 0 of the warp's range (16-byte aligned)
  uint32_t bar;         // shared address of barrier 0
  uint32_t total;       // words in the range (multiple of 4)
  uint32_t nchunks, issued, ready;
  uint32_t phase_bits;  // next-phase parity of each of the kNumChunks barriers
  const uint32_t *ring; // generic pointer to the ring

  __device__ void issue_upto(uint32_t lim, int lane) {
    if (issued >= lim) return;
    __syncwarp();  // every lane is done with the chunks being recycled
    fence_proxy_async();
    for (uint32_t c = issued; c < lim; ++c) {
      const uint32_t w0 = c * kChunk;
      const uint32_t nw = min(kChunk, total - w0);
      bulk_load(lane == 0, smem_addr(ring) + (c % kNumChunks) * kChunk * 4, src + w0, nw * 4,
                bar + (c % kNumChunks) * 8);
    }
    issued = lim;
  }
  // Keeps the ring full: chunks below the one holding `pos` are consumed.
  __device__ void refill(uint32_t pos, int lane) {
    const uint32_t lim = min(nchunks, pos / kChunk + kNumChunks);
    issue_upto(lim, lane);
  }
  // Makes words [.., end) readable; false on a timed-out wait.
  __device__ bool ensure(uint32_t pos, uint32_t end, int lane) {
    const uint32_t need = (end + kChunk - 1) / kChunk;
    if (need <= ready) return true;
    if (end > total) return false;  // past the warp's range: corrupt stream
    refill(pos, lane);
    while (ready < need) {
      if (ready >= issued) return false;  // would read past what the ring can hold
      if (!wait_chunk(ready)) return false;
      ++ready;
    }
    return true;
  }
  __device__ uint32_t at(uint32_t pos) const { return ring[pos & kMask]; }
  // Barrier c % kNumChunks guards ring slot c % kNumChunks; phase_bits holds
  // the parity of the next phase of each barrier (it carries over between
  // ranges decoded by the same warp).
  __device__ bool wait_chunk(uint32_t c) {
    const uint32_t b = c % kNumChunks;
    if (!mbar_wait_warp(bar + b * 8, (phase_bits >> b) & 1u, kSpinLimit)) return false;
    phase_bits ^= 1u << b;
    return true;
  }
  // Waits (bounded) for every copy still in flight.
  __device__ void drain() {
    while (ready < issued) {
      if (!wait_chunk(ready)) break;
      ++ready;
    }
  }
};

// Decoder state of one lane (one unit) while a warp decodes a slice.
struct LaneState {
  uint32_t w0, w1, w2;  // the three words unpacked into the next segment
  uint32_t d, r;        // dtANS decoder state (digit, radix), both < 2^32
  uint32_t col;         // running column (the first delta is absolute)
  uint32_t n, nseg;     // entries and segments of the unit
  uint32_t cont;        // 1: the lane's chain goes on after this unit (its last segment reads on)
};

// Where the products go: KT right-hand-side columns c0 .. c0 + KT - 1 of a
// row-major block with leading dimension ld.
template <typename V>
struct Dense {
  const V *__restrict__ x;
  V *__restrict__ y;
  uint32_t ld, c0;
  const int4 *__restrict__ xfix;  // integer-coefficient products: x as fixed point (IntCols), else null
  int32_t scale;                  // ... the power of two of one unit of their sums
  int32_t coef_exp;               // ... and of one unit of the table's coefficients
  int32_t radixw = 1;             // 0: no check group can have radix W (the tables hold no symbol of
                                  // multiplicity M in one of the domains), so that test is skipped
  int32_t x32 = 0;                // rows of x (KT > 1) start on 32-byte boundaries at column c0
  uint4 *stage = nullptr;         // this warp's staging area in shared memory (TCols32)
  // value gradient (DotCols32): G's rows (leading dimension ld, column c0),
  // 32-byte aligned when g32; the sorted-CSR position of each unit's first
  // entry; add to the output instead of writing it when acc_out
  const V *__restrict__ g = nullptr;
  const uint64_t *__restrict__ unit_pos = nullptr;
  int32_t g32 = 0, acc_out = 0;
  uint64_t nnz = 0;     // ... entries (a position past it is a corrupt stream)
  int32_t *err = nullptr;
  // codebook gradient (DotCols32<true>): the bin of each value-table slot
  // (the kept symbol's rank, or the last bin) and the CTA's bins in shared memory
  const uint16_t *__restrict__ vrank = nullptr;
  V *bins = nullptr;
};

// Zeros that pad slots of the 32-byte row loads read instead of a row of X.
static __device__ __align__(128) double g_zero_row[16];

// Per-lane accumulators for KT columns.  KT = 1 gathers x as soon as a column
// is known; KT > 1 gathers each row of X (KT contiguous values) after the
// state update, with 32-byte loads when the rows are a whole number of
// 32-byte sectors and start on sector boundaries (each sector then passes
// L1TEX once; the 32 lanes gather 32 different rows), else 16-byte loads.
template <typename V, int KT>
struct Cols {
  static constexpr int kVec = 16 / (int)sizeof(V);  // values per 16-byte load
  static constexpr int kV32 = 32 / (int)sizeof(V);  // values per 32-byte load
  // rows of whole sectors read with 32-byte loads; not the 64-byte FP64 rows,
  // whose 8 FP64 FMAs per entry bound the kernel (measured on GB300: k = 8
  // 0.324 ms with 32-byte loads, 0.312 ms with 16-byte ones)
  static constexpr bool k32 = (KT * sizeof(V)) % 32 == 0 && (sizeof(V) == 4 || KT * sizeof(V) <= 32);
  static_assert(KT % kVec == 0, "KT must fill whole 16-byte vectors");
  V acc[KT];
  uint32_t cc[4];
  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int c = 0; c < KT; ++c) acc[c] = V(0);
  }
  __device__ __forceinline__ void at_column(int t, uint32_t col, const Dense<V> &D) { cc[t] = col; }
  __device__ __forceinline__ void skip(int t) { cc[t] = 0xffffffffu; }
  // KT values of a row at p: 32-byte loads (kW32; p on a sector boundary) or
  // 16-byte ones.
  template <bool kW32>
  __device__ __forceinline__ static void load_row(const V *p, V *r) {
    if constexpr (kW32) {
#pragma unroll
      for (int c = 0; c < KT; c += kV32) ldg32(p + c, r + c);
    } else {
#pragma unroll
      for (int c = 0; c < KT; c += kVec) {
        if constexpr (sizeof(V) == 8) {
          const double2 q = __ldg((const double2 *)(p + c));
          r[c] = q.x;
          r[c + 1] = q.y;
        } else {
          const float4 q = __ldg((const float4 *)(p + c));
          r[c] = q.x;
          r[c + 1] = q.y;
          r[c + 2] = q.z;
          r[c + 3] = q.w;
        }
      }
    }
  }
  // Rows wider than 32 bytes (FP64, 8 columns; FP32, 16 or 32): two entries'
  // rows are loaded together, a pad reading zeros instead (16-byte loads:
  // predicated, not branched; 32-byte loads: from a zero row), so both are in
  // flight before the first FMA waits; an entry slot that is a pad in every
  // lane costs no FMA.  Measured on GB300: 6.7 % faster for 8 FP64 columns,
  // 2 % slower for 32-byte rows, which keep the branched form below.
  // 128-byte rows (32 FP32 columns) go one entry at a time, so that the
  // loaded row and the 32 accumulators fit the registers of a 16-warp CTA.
  template <bool kW32>
  __device__ __forceinline__ void accumulate_wide(const V (&v)[4], const Dense<V> &D) {
    constexpr int kG = KT * sizeof(V) > 64 ? 1 : 2;
#pragma unroll
    for (int g = 0; g < 4; g += kG) {
      V xr[kG][KT];
#pragma unroll
      for (int t = 0; t < kG; ++t) {
        const bool live = cc[g + t] != 0xffffffffu;
        if constexpr (kW32) {
          load_row<true>(live ? D.x + (size_t)cc[g + t] * D.ld + D.c0 : (const V *)g_zero_row, xr[t]);
        } else {
          const V *row = D.x + (size_t)(live ? cc[g + t] : 0u) * D.ld + D.c0;
#pragma unroll
          for (int c = 0; c < KT; c += kVec) {
            if constexpr (sizeof(V) == 8) {
              const double2 q = live ? __ldg((const double2 *)(row + c)) : make_double2(0.0, 0.0);
              xr[t][c] = q.x;
              xr[t][c + 1] = q.y;
            } else {
              const float4 q = live ? __ldg((const float4 *)(row + c)) : make_float4(0.f, 0.f, 0.f, 0.f);
              xr[t][c] = q.x;
              xr[t][c + 1] = q.y;
              xr[t][c + 2] = q.z;
              xr[t][c + 3] = q.w;
            }
          }
        }
      }
#pragma unroll
      for (int t = 0; t < kG; ++t) {
        if (!__any_sync(kFull, cc[g + t] != 0xffffffffu)) continue;
#pragma unroll
        for (int c = 0; c < KT; ++c) acc[c] = fma(v[g + t], xr[t][c], acc[c]);
      }
    }
  }
  // Rows of up to 32 bytes: per entry slot, a branch around a pad.
  template <bool kW32>
  __device__ __forceinline__ void accumulate_rows(const V (&v)[4], const Dense<V> &D) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (cc[t] == 0xffffffffu) continue;  // a pad: no gather, no FMA (skipped by the warp if no lane has it)
      V xr[KT];
      load_row<kW32>(D.x + (size_t)cc[t] * D.ld + D.c0, xr);
#pragma unroll
      for (int c = 0; c < KT; ++c) acc[c] = fma(v[t], xr[c], acc[c]);
    }
  }
  __device__ __forceinline__ void accumulate(const V (&v)[4], const Dense<V> &D) {
    if constexpr (KT * sizeof(V) > 32) {
      if constexpr (k32) {
        if (D.x32) {
          accumulate_wide<true>(v, D);
          return;
        }
      }
      accumulate_wide<false>(v, D);
    } else {
      if constexpr (k32) {
        if (D.x32) {
          accumulate_rows<true>(v, D);
          return;
        }
      }
      accumulate_rows<false>(v, D);
    }
  }
  __device__ __forceinline__ void accumulate_n(const V (&v)[4], uint32_t, const Dense<V> &D) { accumulate(v, D); }
  __device__ __forceinline__ V total(int c) const { return acc[c]; }
};

// 32 FP32 columns with the accumulators transposed: lane c owns column c,
// and acc[l] is column c of the row of lane l's unit in this slice.  At each
// segment the lanes publish their entries (the row of X each one multiplies,
// or the zero row for a pad, and the value) in the warp's staging area; the
// warp then reads each entry's 128-byte row of X with one coalesced load,
// lane c taking column c: one line per load, where row-per-lane loads gather
// 32 different lines per load and bind the L1TEX data pipe.  The slice's
// rows are written by the whole warp at the end (store_rows).
constexpr int kStageBytes = 4 * 32 * 16;  // staging area per warp: 4 slots x 32 lanes x 16 bytes

struct TCols32 {
  float acc[32];
  uint32_t cc[4];
  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int l = 0; l < 32; ++l) acc[l] = 0.f;
  }
  __device__ __forceinline__ void at_column(int t, uint32_t col, const Dense<float> &) { cc[t] = col; }
  __device__ __forceinline__ void skip(int t) { cc[t] = 0xffffffffu; }
  // Each entry is staged as its row's address (the zero row for a pad) and
  // its value: the warp's loop per entry is then one broadcast shared load,
  // one coalesced load and one FMA.  (Staging the column index and testing
  // for pads in that loop measured 24 % slower on GB300.)
  __device__ __forceinline__ void accumulate(const float (&v)[4], const Dense<float> &D) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const float *row = cc[t] != 0xffffffffu ? D.x + (size_t)cc[t] * D.ld + D.c0 : (const float *)g_zero_row;
      const unsigned long long p = (unsigned long long)row;
      D.stage[t * 32 + lane] = make_uint4((uint32_t)p, (uint32_t)(p >> 32), __float_as_uint(v[t]), 0u);
    }
    __syncwarp();
#pragma unroll 1
    for (int t = 0; t < 4; ++t) {
      const uint4 *st = D.stage + t * 32;
#pragma unroll
      for (int l = 0; l < 32; ++l) {
        const uint4 e = st[l];  // the same 16 bytes for every lane: one broadcast
        const float *row = (const float *)(((unsigned long long)e.y << 32) | e.x);
        acc[l] = fmaf(__uint_as_float(e.z), __ldg(row + lane), acc[l]);
      }
    }
    __syncwarp();  // the area is written again at the next segment
  }
  __device__ __forceinline__ void accumulate_n(const float (&v)[4], uint32_t, const Dense<float> &D) {
    accumulate(v, D);
  }
  // y rows of the slice: lane l's unit (live in `has`) adds to row `row`
  // (atomically when `split`); every lane of the warp takes part.
  __device__ __forceinline__ void store_rows(const Dense<float> &D, uint32_t row, bool has, bool split,
                                             int32_t beta_mode, float beta) const {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t mh = __ballot_sync(kFull, has), ms = __ballot_sync(kFull, has && split);
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const uint32_t r = __shfl_sync(kFull, row, l);
      if (!((mh >> l) & 1u)) continue;
      float *yp = D.y + (size_t)r * D.ld + D.c0 + lane;
      if ((ms >> l) & 1u)
        atomicAdd(yp, acc[l]);
      else if (beta_mode == 0)
        *yp = acc[l];
      else if (beta_mode == 1)
        *yp = acc[l] + *yp;
      else
        *yp = fmaf(beta, *yp, acc[l]);
    }
  }
};

// The value gradient of 32 FP32 columns on the compressed pattern:
// out[p] = <G[row, c0 : c0 + 32], X[col, c0 : c0 + 32]> for each entry p
// (sorted-CSR position, the unit's first position plus the entry's index in
// it).  Each lane loads its unit's G row once per slice and each entry's X
// row with 32-byte loads when the rows are sector-aligned.  kCode: the
// codebook gradient instead, each dot product added to the shared-memory
// bin of the entry's value symbol (the rank of the kept symbol that owns its
// table slot, escaped values in the last bin).
template <bool kCode>
struct DotCols32 {
  float gv[32];
  uint32_t cc[4];
  uint32_t vs[4];  // kCode: value-table slots of the segment's entries
  uint64_t opos;   // position of the lane's entry in slot 0 of the next segment
  __device__ __forceinline__ void reset() {}
  __device__ __forceinline__ void begin(const Dense<float> &D, uint32_t row, bool live, uint64_t pos) {
    opos = pos;
    if (!live) {
#pragma unroll
      for (int c = 0; c < 32; ++c) gv[c] = 0.f;
      return;
    }
    const float *gr = D.g + (size_t)row * D.ld + D.c0;
    if (D.g32) {
#pragma unroll
      for (int c = 0; c < 32; c += 8) ldg32(gr + c, gv + c);
    } else {
#pragma unroll
      for (int c = 0; c < 32; c += 4) {
        const float4 q = __ldg((const float4 *)(gr + c));
        gv[c] = q.x, gv[c + 1] = q.y, gv[c + 2] = q.z, gv[c + 3] = q.w;
      }
    }
  }
  __device__ __forceinline__ void at_column(int t, uint32_t col, const Dense<float> &) { cc[t] = col; }
  __device__ __forceinline__ void skip(int t) { cc[t] = 0xffffffffu; }
  // byte offsets o[2t + 1] of the segment's value-table entries
  __device__ __forceinline__ void value_slots(const uint32_t (&o)[8]) {
#pragma unroll
    for (int t = 0; t < 4; ++t) vs[t] = o[2 * t + 1] / (uint32_t)sizeof(ValueEntry<float>);
  }
  template <bool kW32>
  __device__ __forceinline__ void dots(const Dense<float> &D) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (cc[t] == 0xffffffffu) continue;  // a pad
      const float *xr = D.x + (size_t)cc[t] * D.ld + D.c0;
      float r[32];
      if constexpr (kW32) {
#pragma unroll
        for (int c = 0; c < 32; c += 8) ldg32(xr + c, r + c);
      } else {
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          const float4 q = __ldg((const float4 *)(xr + c));
          r[c] = q.x, r[c + 1] = q.y, r[c + 2] = q.z, r[c + 3] = q.w;
        }
      }
      float s0 = 0.f, s1 = 0.f;
#pragma unroll
      for (int c = 0; c < 32; c += 2) {
        s0 = fmaf(gv[c], r[c], s0);
        s1 = fmaf(gv[c + 1], r[c + 1], s1);
      }
      if constexpr (kCode) {
        atomicAdd(D.bins + __ldg(D.vrank + vs[t]), s0 + s1);
        continue;
      }
      if (opos + t >= D.nnz) {  // a unit longer than its place in CSR order: corrupt
        atomicExch(D.err, kErrOverrun);
        continue;
      }
      float *o = D.y + opos + t;
      *o = D.acc_out ? *o + (s0 + s1) : s0 + s1;
    }
  }
  __device__ __forceinline__ void accumulate(const float (&)[4], const Dense<float> &D) {
    if (D.x32)
      dots<true>(D);
    else
      dots<false>(D);
    opos += 4;
  }
  __device__ __forceinline__ void accumulate_n(const float (&v)[4], uint32_t, const Dense<float> &D) {
    accumulate(v, D);
  }
};

template <typename Acc>
constexpr bool is_dotcols() {
  return std::is_same<Acc, DotCols32<false>>::value || std::is_same<Acc, DotCols32<true>>::value;
}
template <typename Acc>
constexpr bool wants_value_slots() {
  return std::is_same<Acc, DotCols32<true>>::value;
}

template <typename Acc>
constexpr bool is_tcols() {
  return std::is_same<Acc, TCols32>::value;
}

// One right-hand side.  FP32 keeps two independent FMA chains.  FP64 products
// go through GB300's narrow FP64 pipe, which bounds the whole kernel, so the
// FP64 path spends exactly one pipe operation per stored entry: one chain
// (no final add) and no FMA for a slot that is a pad in every lane.
template <typename V>
struct Cols<V, 1> {
  static constexpr bool kOneChain = sizeof(V) == 8;
  V acc0, acc1, xg[4];
  __device__ __forceinline__ void reset() { acc0 = acc1 = V(0); }
  __device__ __forceinline__ void at_column(int t, uint32_t col, const Dense<V> &D) { xg[t] = __ldg(D.x + col); }
  __device__ __forceinline__ void skip(int t) { xg[t] = V(0); }
  __device__ __forceinline__ void accumulate(const V (&v)[4], const Dense<V> &) {
    if constexpr (kOneChain) {
      acc0 = fma(v[0], xg[0], acc0);
      acc0 = fma(v[1], xg[1], acc0);
      acc0 = fma(v[2], xg[2], acc0);
      acc0 = fma(v[3], xg[3], acc0);
    } else {
      acc0 = fma(v[0], xg[0], acc0);
      acc1 = fma(v[1], xg[1], acc1);
      acc0 = fma(v[2], xg[2], acc0);
      acc1 = fma(v[3], xg[3], acc1);
    }
  }
  // Slots t >= nvalid of a lane are pads (v = x = 0).  Slot 0 is live in some
  // lane whenever a segment runs.
  __device__ __forceinline__ void accumulate_n(const V (&v)[4], uint32_t nvalid, const Dense<V> &D) {
    if constexpr (sizeof(V) == 8) {
      // A warp-uniform loop over the live slots (operands picked by
      // selects): written as tests on the live count, the slot FMAs were
      // if-converted into unconditional ones (28 FP64 FMAs per 27-entry
      // stencil row on GB300), and the FP64 pipe bounds this path.
      const uint32_t nv = __reduce_max_sync(kFull, nvalid);
      acc0 = fma(v[0], xg[0], acc0);
#pragma unroll 1
      for (uint32_t t = 1; t < nv; ++t) {
        const V a = t == 1 ? v[1] : (t == 2 ? v[2] : v[3]);
        const V b = t == 1 ? xg[1] : (t == 2 ? xg[2] : xg[3]);
        acc0 = fma(a, b, acc0);
      }
    } else {
      accumulate(v, D);
    }
  }
  __device__ __forceinline__ V total(int) const {
    if constexpr (kOneChain) return acc0;
    return acc0 + acc1;
  }
};

// The exact sum T = a0 + a1 2^32 + a2 2^64 (signed 64-bit parts) times
// 2^scale, rounded once to FP64 (round to nearest, ties to even), with
// integer operations only: T as a 128-bit two's complement hi:lo, its
// magnitude normalised so bit 127 is set, the top 64 bits kept with every
// lower bit folded into their lowest one (it lies below the rounding
// position, so it only acts as the sticky bit), then rounded to 53 bits and
// assembled with the exponent.  Results outside the normal range (overflow,
// subnormals) are scaled by scalbn instead.
static __device__ __noinline__ double fixed_to_double_slow(bool neg, unsigned long long top, int32_t e2) {
  const double r = scalbn(__ull2double_rn(top), e2);
  return neg ? -r : r;
}

__device__ __forceinline__ double fixed_to_double(long long a0, long long a1, long long a2, int32_t scale) {
  unsigned long long lo = (unsigned long long)a0 + ((unsigned long long)a1 << 32);
  const unsigned long long carry = lo < ((unsigned long long)a1 << 32) ? 1ull : 0ull;
  long long hi = (a0 >> 63) + (a1 >> 32) + a2 + (long long)carry;
  if ((hi | (long long)lo) == 0) return 0.0;
  const bool neg = hi < 0;
  if (neg) {  // 128-bit negation
    lo = 0ull - lo;
    hi = ~hi + (lo == 0ull ? 1 : 0);
  }
  const unsigned long long uh = (unsigned long long)hi;
  unsigned long long top;
  int lz;
  if (uh) {
    lz = __clzll((long long)uh);
    unsigned long long rest;
    if (lz) {
      top = (uh << lz) | (lo >> (64 - lz));
      rest = lo << lz;
    } else {
      top = uh;
      rest = lo;
    }
    top |= rest != 0ull ? 1ull : 0ull;
  } else {
    lz = 64 + __clzll((long long)lo);
    top = lo << (lz - 64);
  }
  // |T| = top 2^(64 - lz) (up to the sticky bit); value = |T| 2^scale
  unsigned long long m = top >> 11;  // 53 bits, the leading one at bit 52
  const uint32_t low = (uint32_t)top & 0x7ffu;
  m += (low > 0x400u || (low == 0x400u && (m & 1ull))) ? 1ull : 0ull;
  int32_t be = 1150 - lz + scale;  // biased exponent of m 2^(75 - lz + scale) with m in [2^52, 2^53)
  if (m >> 53) {
    m >>= 1;
    ++be;
  }
  if (be < 1 || be > 2046) return fixed_to_double_slow(neg, top, 64 - lz + scale);
  const unsigned long long bits =
      (neg ? 1ull << 63 : 0ull) | ((unsigned long long)be << 52) | (m & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// One right-hand side of an FP64 matrix whose kept values are all c * 2^e
// with small integers c (|c| < 2^15; dtans_handle_s::int_ok).  Every x
// arrives as exact fixed point, x 2^F = S0 + S1 2^32 + S2 2^64 with signed
// 32-bit limbs, plus a flag for x outside the window the limbs cover (see
// the prepass in spmv.cu), so an entry adds c * S_k to three 64-bit
// accumulators (one 32 x 32 -> 64-bit multiply-add each, on the integer
// pipe) and the unit's sum of c_j x_j 2^F is exact; it is rounded to FP64
// once at the end.  Two kinds of entries go through an FP64 FMA chain
// instead: a flagged x (its limbs hold x's raw bits, S2 = 0; the rare path
// takes their products back out of the accumulators, exactly, and adds
// c 2^e * x) and an escaped value (read raw from the stream; the escape
// symbol's coefficient is 0, and the entry's FMA is taken as soon as its
// column is known, see escaped()).  Every limb, raw bits included, lies in
// [-2^31, 2^31), so for a unit of length L the accumulators hold
// |a_k| < L 2^46, inside 64 bits for L <= 2^16.
// d = a * b + c for signed 32-bit a, b and a 64-bit c (one 32 x 32 -> 64-bit
// multiply-add; written out so the product is not widened to 64 x 64).
__device__ __forceinline__ long long mad_wide(int32_t a, int32_t b, long long c) {
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

struct IntCols {
  long long a0, a1, a2;
  double fb;
  int4 xq[4];
  __device__ __forceinline__ void reset() {
    a0 = a1 = a2 = 0;
    fb = 0.0;
  }
  __device__ __forceinline__ void at_column(int t, uint32_t col, const Dense<double> &D) {
    xq[t] = __ldg(D.xfix + col);
  }
  __device__ __forceinline__ void skip(int t) { xq[t] = make_int4(0, 0, 0, 0); }
  // An entry whose value v was escaped: FMA with the true x at once, and no
  // fixed-point term (xq cleared: the escape symbol's coefficient is 0, and a
  // flagged x must not reach the rare path).  Only the column pass of a
  // segment in which some lane has an escaped value calls it (a separate,
  // warp-uniform pass), so the common pass issues no FP64 instruction: a
  // per-slot test there is if-converted into a predicated FMA per slot, and
  // on this GPU's FP64 pipe a predicated-off FMA still takes its 16 cycles.
  __device__ __forceinline__ void escaped(int t, uint32_t col, double v, const Dense<double> &D) {
    fb = fma(v, __ldg(D.x + col), fb);
    xq[t] = make_int4(0, 0, 0, 0);
  }
  __device__ __forceinline__ void accumulate(const ValueEntry<double> (&eV)[4], const Dense<double> &D) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int32_t c = eV[t].coef;
      a0 = mad_wide(c, xq[t].x, a0);
      a1 = mad_wide(c, xq[t].y, a1);
      a2 = mad_wide(c, xq[t].z, a2);
    }
    if (__any_sync(kFull, xq[0].w | xq[1].w | xq[2].w | xq[3].w)) {
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (xq[t].w) {
          const int32_t c = eV[t].coef;
          a0 = mad_wide(-c, xq[t].x, a0);
          a1 = mad_wide(-c, xq[t].y, a1);
          fb = fma(scalbn((double)c, D.coef_exp), __hiloint2double(xq[t].y, xq[t].x), fb);
        }
    }
  }
  __device__ __forceinline__ double total(int, int32_t scale) const {
    return fixed_to_double(a0, a1, a2, scale) + fb;
  }
};

template <typename Acc>
constexpr bool is_int_acc() {
  return std::is_same<Acc, IntCols>::value;
}

// Escape point of a segment (Sec. IV-F "Escape symbols"): each lane's raw
// words of this segment in slot order (a delta, then a value, per nonzero;
// a value's low word first), lanes in order.  Slots t >= nvalid are pads and
// read nothing (kAll: every slot is live).  Returns false when no lane has an
// escaped slot; otherwise anyv (some lane has an escaped value), off (this
// lane's first raw word, relative to the escape point) and tot (raw words of
// the warp).  The lane's counts are sums of the escape flags (bit 15 of a
// table entry's meta word), so no per-slot mask is built.
template <typename V, bool kAll>
__device__ __forceinline__ bool escape_plan(const DeltaEntry (&eD)[4], const ValueEntry<V> (&eV)[4],
                                            uint32_t nvalid, uint32_t lt, bool &anyv, uint32_t &off,
                                            uint32_t &tot) {
  static_assert(kMetaEsc == 1u << 15, "escape flag is bit 15 of a table entry's meta word");
  constexpr uint32_t kRawV = RawWords<V>::kValue;
  uint32_t ed = 0, ev = 0;  // escaped live slots of each domain, times 2^15
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (kAll || (uint32_t)t < nvalid) {
      ed += eD[t].meta & kMetaEsc;
      ev += eV[t].meta & kMetaEsc;
    }
  if (!__any_sync(kFull, (ed | ev) != 0u)) return false;
  const uint32_t cd = ed >> 15, cv = ev >> 15;
  anyv = __any_sync(kFull, cv != 0u);
  if (!anyv)  // deltas only: at most 4 raw words per lane
    off = warp_prefix8(cd, lt, tot);
  else
    off = warp_prefix16(cd + kRawV * cv, lt, tot);
  return true;
}

// Entries of the segment whose value is escaped (bit t), live slots only.
template <typename V, bool kAll>
__device__ __forceinline__ uint32_t escaped_values(const ValueEntry<V> (&eV)[4], uint32_t nvalid) {
  uint32_t mv = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if ((kAll || (uint32_t)t < nvalid) && (eV[t].meta & kMetaEsc)) mv |= 1u << t;
  return mv;
}

// Reads the raw words planned by escape_plan, starting at stream position p;
// rd(q) returns stream word q.
template <typename V, bool kAll, typename Rd>
__device__ __forceinline__ void escape_read(DeltaEntry (&eD)[4], ValueEntry<V> (&eV)[4], uint32_t nvalid, bool anyv,
                                            uint32_t p, Rd rd) {
  constexpr uint32_t kRawV = RawWords<V>::kValue;
  if (!anyv) {
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if ((kAll || (uint32_t)t < nvalid) && (eD[t].meta & kMetaEsc)) eD[t].delta = rd(p++);
    return;
  }
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (!kAll && (uint32_t)t >= nvalid) continue;
    if (eD[t].meta & kMetaEsc) eD[t].delta = rd(p++);
    if (eV[t].meta & kMetaEsc) {
      if constexpr (kRawV == 2) {
        const uint32_t lo = rd(p), hi = rd(p + 1);
        eV[t].v = __hiloint2double((int)hi, (int)lo);
      } else {
        eV[t].v = __uint_as_float(rd(p));
      }
      p += kRawV;
    }
  }
}

// One segment of four nonzeros (Algorithm 3, one iteration): unpack, table
// lookups, escape point, x gathers, two checks and the unconditional read,
// FMAs.  kFast: every lane of a full slice is live and not in its last
// segment.  kResident: the whole slice is already in the ring, so no read
// needs a ring check.  `lim` bounds pos (the slice end when resident, else the
// warp's range end); returns false when a read would pass it or the ring could
// not supply the words.
template <typename V, int KT, uint32_t RW, bool kFast, bool kResident, typename Acc>
__device__ __forceinline__ bool segment(LaneState &L, Acc &A, Ring<RW> &rg, uint32_t &pos, uint32_t lim,
                                        uint32_t j, const uint8_t *tD, const uint8_t *tV, const Dense<V> &Dn,
                                        uint32_t nm1, uint32_t lt, int lane) {
  using VE = ValueEntry<V>;
  constexpr int VS = sizeof(VE);
  uint32_t o[8];
  unpack_offsets<8, VS>(L.w0, L.w1, L.w2, o);
  if constexpr (wants_value_slots<Acc>()) A.value_slots(o);
  if (!kResident) rg.refill(pos, lane);  // a resident slice was fetched whole at its start
  DeltaEntry eD[4];
  VE eV[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    eD[t] = *(const DeltaEntry *)(tD + o[2 * t]);
    eV[t] = *(const VE *)(tV + o[2 * t + 1]);
  }
  const uint32_t nvalid = kFast ? 4u : (j < L.nseg ? min(4u, L.n - 4 * j) : 0u);
  uint32_t vesc = 0;   // entries whose value was escaped (integer-coefficient products only)
  bool vany = false;   // some lane has one (warp-uniform)
  {
    uint32_t off, tot;
    bool anyv;
    if (escape_plan<V, kFast>(eD, eV, nvalid, lt, anyv, off, tot)) {
      if (pos + tot > lim) return false;
      if (!kResident && !rg.ensure(pos, pos + tot, lane)) return false;
      if constexpr (is_int_acc<Acc>()) {
        vany = anyv;
        vesc = anyv ? escaped_values<V, kFast>(eV, nvalid) : 0u;
      }
      escape_read<V, kFast>(eD, eV, nvalid, anyv, pos + off, [&](uint32_t q) { return rg.at(q); });
      pos += tot;
    }
  }
  // columns (clamped: every gather stays inside x); with KT = 1 the gathers
  // are issued here and consumed after the state update
  // esc: entries whose escaped value takes the FMA at once (integer products)
  auto columns = [&](uint32_t esc) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (kFast || (uint32_t)t < nvalid) {
        L.col += eD[t].delta;
        if constexpr (is_int_acc<Acc>()) {
          if ((esc >> t) & 1u) {
            A.escaped(t, min(L.col, nm1), eV[t].v, Dn);
            continue;
          }
        }
        A.at_column(t, min(L.col, nm1), Dn);
      } else {
        A.skip(t);
        eV[t].v = V(0);
      }
    }
  };
  if (is_int_acc<Acc>() && vany)
    columns(vesc);
  else
    columns(0u);
  // the checks and the unconditional read take at most 3 * 32 words
  if (pos > lim) return false;
  if (!kResident && !rg.ensure(pos, min(pos + 3 * kSlice, lim), lane)) return false;
  const bool more = kFast || (j < L.nseg && (j + 1 < L.nseg || L.cont));
  {
    // both check groups, then their conditional reads (Sec. IV-B: one ballot,
    // two popcounts each; C1's words come before C2's in the stream)
    bool need0 = false, need1 = false;
    if (kFast || more) {
      need0 = group_step(eD[0].meta, eV[0].meta, eD[1].meta, eV[1].meta, L.d, L.r, L.w0);
      need1 = group_step(eD[2].meta, eV[2].meta, eD[3].meta, eV[3].meta, L.d, L.r, L.w1);
    }
    const uint32_t m0 = __ballot_sync(kFull, need0), m1 = __ballot_sync(kFull, need1);
    if (m0 | m1) {  // warp-uniform
      const uint32_t c0 = __popc(m0);
      const uint32_t v0 = rg.at(pos + __popc(m0 & lt));
      const uint32_t v1 = rg.at(pos + c0 + __popc(m1 & lt));
      L.w0 = need0 ? v0 : L.w0;
      L.w1 = need1 ? v1 : L.w1;
      pos += c0 + __popc(m1);
    }
  }
  if (kFast) {
    L.w2 = rg.at(pos + lane);
    pos += kSlice;
  } else {
    const uint32_t m = __ballot_sync(kFull, more);
    const uint32_t v = rg.at(pos + __popc(m & lt));
    L.w2 = more ? v : L.w2;
    pos += __popc(m);
  }
  if constexpr (is_int_acc<Acc>()) {
    A.accumulate(eV, Dn);
  } else {
    const V vals[4] = {eV[0].v, eV[1].v, eV[2].v, eV[3].v};
    if (kFast)
      A.accumulate(vals, Dn);
    else
      A.accumulate_n(vals, nvalid, Dn);
  }
  // A valid stream never reads past `lim`.  Every segment in which some lane
  // is not in its last segment advances pos, so this check also bounds the
  // number of segments a corrupt row length can cause.
  return pos <= lim;
}

// The first `nfast` segments of a resident slice in which all 32 lanes are
// live and none is in its last segment, for one right-hand side: the same
// program as segment<V, 1, RW, true, true>, written as one straight loop over
// plain registers (one uniform branch per rare event: escapes, conditional
// reads, and the range check).  Returns false when a read passes `lim`.
template <typename V, uint32_t RW, typename Acc>
__device__ __forceinline__ bool fast_run_kt1(LaneState &L, Acc &A, const uint32_t *ring, uint32_t &pos_io,
                                             uint32_t lim, uint32_t nfast, const uint8_t *tD, const uint8_t *tV,
                                             const Dense<V> &Dn, uint32_t nm1, uint32_t lt, uint32_t lane) {
  using VE = ValueEntry<V>;
  constexpr int VS = sizeof(VE);
  constexpr uint32_t kMask = RW - 1;
  uint32_t w0 = L.w0, w1 = L.w1, w2 = L.w2, d = L.d, r = L.r, col = L.col, pos = pos_io;
  bool ok = true;
  for (uint32_t j = 0; j < nfast; ++j) {
    uint32_t o[8];
    unpack_offsets<8, VS>(w0, w1, w2, o);
    DeltaEntry eD[4];
    VE eV[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      eD[t] = *(const DeltaEntry *)(tD + o[2 * t]);
      eV[t] = *(const VE *)(tV + o[2 * t + 1]);
    }
    uint32_t vesc = 0;
    bool vany = false;
    {
      uint32_t off, tot;
      bool anyv;
      if (escape_plan<V, true>(eD, eV, 4u, lt, anyv, off, tot)) {
        if constexpr (is_int_acc<Acc>()) {
          vany = anyv;
          vesc = anyv ? escaped_values<V, true>(eV, 4u) : 0u;
        }
        escape_read<V, true>(eD, eV, 4u, anyv, pos + off, [&](uint32_t q) { return ring[q & kMask]; });
        pos += tot;
      }
    }
    auto columns = [&](uint32_t esc) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        col += eD[t].delta;
        if constexpr (is_int_acc<Acc>()) {
          if ((esc >> t) & 1u) {
            A.escaped(t, min(col, nm1), eV[t].v, Dn);
            continue;
          }
        }
        A.at_column(t, min(col, nm1), Dn);
      }
    };
    if (is_int_acc<Acc>() && vany)
      columns(vesc);
    else
      columns(0u);
    bool radix = false;
    if (Dn.radixw) {
      const uint32_t all8 = eD[0].meta & eV[0].meta & eD[1].meta & eV[1].meta & eD[2].meta & eV[2].meta &
                            eD[3].meta & eV[3].meta;
      radix = __all_sync(kFull, all_base_w(all8));
    }
    if (radix) {
      // every group of every lane has radix W: both checks extract, state unchanged
      w0 = pack_digits(eD[0].meta, eV[0].meta, eD[1].meta, eV[1].meta);
      w1 = pack_digits(eD[2].meta, eV[2].meta, eD[3].meta, eV[3].meta);
    } else {
      // The second group's state update does not wait for the first group's
      // read (that word only enters the next segment), so both checks come
      // first and their reads follow together: C1's words, then C2's.
      const bool need0 = group_step(eD[0].meta, eV[0].meta, eD[1].meta, eV[1].meta, d, r, w0);
      const bool need1 = group_step(eD[2].meta, eV[2].meta, eD[3].meta, eV[3].meta, d, r, w1);
      const uint32_t m0 = __ballot_sync(kFull, need0), m1 = __ballot_sync(kFull, need1);
      if (m0 | m1) {
        const uint32_t c0 = __popc(m0);
        const uint32_t v0 = ring[(pos + __popc(m0 & lt)) & kMask];
        const uint32_t v1 = ring[(pos + c0 + __popc(m1 & lt)) & kMask];
        w0 = need0 ? v0 : w0;
        w1 = need1 ? v1 : w1;
        pos += c0 + __popc(m1);
      }
    }
    w2 = ring[(pos + lane) & kMask];
    pos += kSlice;
    if constexpr (is_int_acc<Acc>()) {
      A.accumulate(eV, Dn);
    } else {
      const V vals[4] = {eV[0].v, eV[1].v, eV[2].v, eV[3].v};
      A.accumulate(vals, Dn);
    }
    if (pos > lim) {  // a corrupt row length; each segment advances pos by >= 32
      ok = false;
      break;
    }
  }
  L.w0 = w0, L.w1 = w1, L.w2 = w2, L.d = d, L.r = r, L.col = col;
  pos_io = pos;
  return ok;
}

// The last segment when every lane of a full slice is in its last segment
// (all units of the slice have the same number of segments) and no lane's
// chain goes on: no checks and no reads but the escape point; items past a
// lane's length are pads.
template <typename V, uint32_t RW, typename Acc>
__device__ __forceinline__ bool last_segment_kt1(LaneState &L, Acc &A, const uint32_t *ring, uint32_t &pos,
                                                 uint32_t lim, uint32_t j, const uint8_t *tD, const uint8_t *tV,
                                                 const Dense<V> &Dn, uint32_t nm1, uint32_t lt) {
  using VE = ValueEntry<V>;
  constexpr int VS = sizeof(VE);
  constexpr uint32_t kMask = RW - 1;
  uint32_t o[8];
  unpack_offsets<8, VS>(L.w0, L.w1, L.w2, o);
  DeltaEntry eD[4];
  VE eV[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    eD[t] = *(const DeltaEntry *)(tD + o[2 * t]);
    eV[t] = *(const VE *)(tV + o[2 * t + 1]);
  }
  const uint32_t nvalid = L.n - 4 * j;  // 1..4
  uint32_t vesc = 0;
  bool vany = false;
  {
    uint32_t off, tot;
    bool anyv;
    if (escape_plan<V, false>(eD, eV, nvalid, lt, anyv, off, tot)) {
      if constexpr (is_int_acc<Acc>()) {
        vany = anyv;
        vesc = anyv ? escaped_values<V, false>(eV, nvalid) : 0u;
      }
      escape_read<V, false>(eD, eV, nvalid, anyv, pos + off, [&](uint32_t q) { return ring[q & kMask]; });
      pos += tot;
    }
  }
  auto columns = [&](uint32_t esc) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if ((uint32_t)t < nvalid) {
        L.col += eD[t].delta;
        if constexpr (is_int_acc<Acc>()) {
          if ((esc >> t) & 1u) {
            A.escaped(t, min(L.col, nm1), eV[t].v, Dn);
            continue;
          }
        }
        A.at_column(t, min(L.col, nm1), Dn);
      } else {
        A.skip(t);
        eV[t].v = V(0);
      }
    }
  };
  if (is_int_acc<Acc>() && vany)
    columns(vesc);
  else
    columns(0u);
  if constexpr (is_int_acc<Acc>()) {
    A.accumulate(eV, Dn);
  } else {
    const V vals[4] = {eV[0].v, eV[1].v, eV[2].v, eV[3].v};
    A.accumulate_n(vals, nvalid, Dn);
  }
  return pos <= lim;
}

template <typename V, int KT, uint32_t RW, bool kResident, typename Acc>
__device__ __forceinline__ bool decode_unit_segments(LaneState &L, Acc &A, Ring<RW> &rg, uint32_t &pos,
                                                     uint32_t lim, uint32_t minseg, uint32_t maxseg, const uint8_t *tD,
                                                     const uint8_t *tV, const Dense<V> &Dn, uint32_t nm1,
                                                     uint32_t lt, int lane) {
  uint32_t j = 0;
  if constexpr (KT == 1 && kResident) {
    if (minseg >= 2) {
      if (!fast_run_kt1<V, RW>(L, A, rg.ring, pos, lim, minseg - 1, tD, tV, Dn, nm1, lt, (uint32_t)lane))
        return false;
      j = minseg - 1;
    }
    if (minseg >= 1 && minseg == maxseg && !__any_sync(kFull, L.cont))  // every lane ends here
      return last_segment_kt1<V, RW>(L, A, rg.ring, pos, lim, j, tD, tV, Dn, nm1, lt);
  } else {
    for (; j + 1 < minseg; ++j)
      if (!segment<V, KT, RW, true, kResident>(L, A, rg, pos, lim, j, tD, tV, Dn, nm1, lt, lane)) return false;
  }
  for (; j < maxseg; ++j)
    if (!segment<V, KT, RW, false, kResident>(L, A, rg, pos, lim, j, tD, tV, Dn, nm1, lt, lane)) return false;
  return true;
}

template <typename V>
constexpr int table_bytes() {
  return kK * 8 + kK * (int)sizeof(ValueEntry<V>);
}

// Shared memory of the persistent kernels: tables, one ring and kNumChunks
// barriers per warp, and one barrier for the bulk copy of the tables.
template <typename V>
constexpr int persistent_smem_bytes(int warps, uint32_t ring_words, int stage_bytes = 0) {
  return ((table_bytes<V>() + warps * (int)(ring_words * 4) + warps * (int)kNumChunks * 8 + 8 + 15) & ~15) +
         warps * stage_bytes;
}

// The table image is copied into shared memory in chunks of this many bytes.
constexpr uint32_t kTableChunk = 16384;
template <typename V>
constexpr uint32_t table_chunks() {
  static_assert(table_bytes<V>() % kTableChunk == 0, "table image is a whole number of chunks");
  return table_bytes<V>() / kTableChunk;
}

// Starts the copy of a table image (global, 16-byte aligned) into shared
// memory with bulk copies, one chunk per lane of the calling warp, completing
// on barrier `tbar` (initialised with table_chunks<V>() arrivals).
template <typename V>
__device__ __forceinline__ void stage_tables_bulk(uint8_t *smem, const uint8_t *tables, uint32_t tbar, int lane) {
  static_assert(table_chunks<V>() <= 32, "one chunk per lane");
  const uint32_t c = (uint32_t)lane;
  bulk_load(c < table_chunks<V>(), smem_addr(smem) + c * kTableChunk, tables + (size_t)c * kTableChunk,
            kTableChunk, tbar);
}

// Copies a table image (global, 16-byte aligned) into shared memory with all
// threads of the CTA (the caller synchronises).
template <typename V>
__device__ __forceinline__ void stage_tables(uint8_t *smem, const uint8_t *tables) {
  const uint4 *src = (const uint4 *)tables;
  uint4 *dst = (uint4 *)smem;
  for (int i = threadIdx.x; i < table_bytes<V>() / 16; i += blockDim.x) dst[i] = __ldg(src + i);
}

// Decodes slices [s0, s1) of one matrix with one warp and writes KT columns
// of y.  The warp's ring (ring_base, bars: barriers initialised for this
// warp, phase parities in phase_bits, no copy in flight) streams the words.
// first_rel: a unit's first delta is relative to its row (the running column
// starts at the row instead of 0).  chain: slices per chain (the lanes'
// decoder state runs on from one slice of a chain into the next; s0 is a
// chain's first slice; kChain = false compiles the one-slice chains of the
// paper's format only).  tbar != 0: the tables are still arriving on that
// barrier (phase 0); the warp waits for them after starting its ring.
// kInt (FP64, KT = 1): integer-coefficient products (IntCols; Dn.xfix and
// Dn.scale set).  Returns 0 or an error code.
template <typename V, int KT, uint32_t RW, bool kChain = true, bool kInt = false, int kGrad = 0>
__device__ int32_t warp_spmv_range(const uint32_t *__restrict__ words, const uint64_t *__restrict__ slice_off,
                                   const uint32_t *__restrict__ unit_row, int64_t nunits, uint32_t ncols,
                                   bool first_rel, uint32_t chain, uint32_t s0, uint32_t s1, const uint8_t *tD, const uint8_t *tV,
                                   uint32_t *ring_base, uint64_t *bars, const Dense<V> &Dn, V beta,
                                   int32_t beta_mode, int32_t *err, uint32_t &phase_bits, int lane,
                                   uint32_t tbar = 0) {
  using RingT = Ring<RW>;
  if (s0 >= s1) return 0;
  const uint64_t gbeg = slice_off[s0], gend = slice_off[s1];
  const uint64_t g0 = gbeg & ~3ull;
  const uint64_t span = ((gend + 3) & ~3ull) - g0;
  if (span >= (1ull << 31)) return kErrRange;
  RingT rg;
  rg.src = words + g0;
  rg.bar = smem_addr(bars);
  rg.ring = ring_base;
  rg.total = (uint32_t)span;
  rg.nchunks = (rg.total + RingT::kChunk - 1) / RingT::kChunk;
  rg.issued = 0;
  rg.ready = 0;
  rg.phase_bits = phase_bits;
  rg.refill(0, lane);
  const uint32_t lt = lanemask_lt();
  const uint32_t nm1 = ncols - 1;
  uint32_t pos = (uint32_t)(gbeg - g0);
  int32_t fail = 0;
  // Slice offsets relative to g0, 32 at a time: lane i holds that of slice
  // sb + i (one coalesced load per 31 slices instead of two per slice).
  uint32_t sb = s0;
  uint32_t offv = (uint32_t)(slice_off[min(sb + (uint32_t)lane, s1)] - g0);
  if (tbar && !mbar_wait_warp(tbar, 0, kSpinLimit)) {
    rg.drain();
    phase_bits = rg.phase_bits;
    return kErrTimeout;
  }
  // the lane's decoder state (L.w0..w2, L.d, L.r) runs on from one slice of
  // a chain to the next
  LaneState L;
  L.w0 = L.w1 = L.w2 = 0;
  L.d = 0;
  L.r = 1;
  uint32_t kc = 0;  // slice index within the current chain

  for (uint32_t s = s0; s < s1; ++s) {
    if (s + 1 - sb >= kSlice) {
      sb = s;
      offv = (uint32_t)(slice_off[min(sb + (uint32_t)lane, s1)] - g0);
    }
    const uint32_t so = __shfl_sync(kFull, offv, s - sb);
    const uint32_t se = __shfl_sync(kFull, offv, s + 1 - sb);
    // every slice must start where the previous one ended (a corrupt stream
    // is caught here; reads in between stay inside the ring by masking)
    if (pos != so) {
      fail = kErrOverrun;
      break;
    }
    const int64_t u0 = (int64_t)s * kSlice;
    const uint32_t nl = (uint32_t)min((int64_t)kSlice, nunits - u0);
    const bool has = (uint32_t)lane < nl;
    if (!rg.ensure(pos, pos + nl, lane)) {
      fail = kErrOverrun;
      break;
    }
    std::conditional_t<kInt, IntCols,
                       std::conditional_t<kGrad != 0, DotCols32<kGrad == 2>,
                                          std::conditional_t<(KT == 32 && sizeof(V) == 4), TCols32, Cols<V, KT>>>>
        A;
    {
      const uint32_t nw = has ? rg.at(pos + lane) : 0u;  // n | continues << 31
      L.n = nw & 0x7fffffffu;
      L.cont = kChain ? nw >> 31 : 0u;
    }
    pos += nl;
    if (!kChain || kc == 0) {  // a chain starts: lanes with entries now or later read their initial words
      const bool act = L.n > 0 || L.cont;
      const uint32_t m = __ballot_sync(kFull, act);
      const uint32_t cnt = __popc(m), rk = __popc(m & lt);
      if (!rg.ensure(pos, pos + 3 * cnt, lane)) {
        fail = kErrOverrun;
        break;
      }
      L.w0 = L.w1 = L.w2 = 0;
      if (act) {
        L.w0 = rg.at(pos + rk);
        L.w1 = rg.at(pos + cnt + rk);
        L.w2 = rg.at(pos + 2 * cnt + rk);
      }
      pos += 3 * cnt;
      L.d = 0;
      L.r = 1;
    }
    if (kChain && ++kc == chain) kc = 0;
    L.nseg = (L.n + 3) >> 2;
    const uint32_t maxseg = __reduce_max_sync(kFull, L.nseg);
    const uint32_t minseg = __reduce_min_sync(kFull, L.nseg);  // lanes past nl count as 0
    L.col = 0;
    if (first_rel) L.col = unit_row ? (has ? __ldg(unit_row + u0 + lane) & 0x7fffffffu : 0u) : (uint32_t)(u0 + lane);
    A.reset();
    if constexpr (is_dotcols<decltype(A)>()) {
      uint32_t row = (uint32_t)(u0 + lane);
      if (unit_row && has) row = __ldg(unit_row + u0 + lane) & 0x7fffffffu;
      A.begin(Dn, row, has && L.n > 0, has ? __ldg(Dn.unit_pos + u0 + lane) : 0ull);
    }
    // A slice whose words all fit in the ring window is made resident once;
    // its segments then read without ring checks.
    const bool resident = se - (pos & ~(RingT::kChunk - 1)) <= RW && se <= rg.total;
    bool ok;
    if (resident) {
      ok = rg.ensure(pos, se, lane) &&
           decode_unit_segments<V, KT, RW, true>(L, A, rg, pos, se, minseg, maxseg, tD, tV, Dn, nm1, lt, lane);
    } else {
      ok = decode_unit_segments<V, KT, RW, false>(L, A, rg, pos, rg.total, minseg, maxseg, tD, tV, Dn, nm1, lt,
                                                  lane);
    }
    if (!ok) {
      fail = kErrOverrun;
      break;
    }
    if constexpr (is_dotcols<decltype(A)>()) {
      if (has && L.n > 0 && L.col > nm1) atomicExch(err, kErrColumn);  // the products went out per entry
    } else if constexpr (is_tcols<decltype(A)>()) {
      uint32_t row = (uint32_t)(u0 + lane);
      bool split = false;
      if (has) {
        if (L.n > 0 && L.col > nm1) atomicExch(err, kErrColumn);
        if (unit_row) {
          const uint32_t ur = __ldg(unit_row + u0 + lane);
          row = ur & 0x7fffffffu;
          split = (ur >> 31) != 0;
        }
      }
      A.store_rows(Dn, row, has, split, beta_mode, beta);
    } else if (has) {
      if (L.n > 0 && L.col > nm1) atomicExch(err, kErrColumn);
      uint32_t row = (uint32_t)(u0 + lane);
      bool split = false;
      if (unit_row) {
        const uint32_t ur = __ldg(unit_row + u0 + lane);
        row = ur & 0x7fffffffu;
        split = (ur >> 31) != 0;
      }
      V *yp = KT == 1 ? Dn.y + row : Dn.y + (size_t)row * Dn.ld + Dn.c0;
#pragma unroll
      for (int c = 0; c < KT; ++c) {
        V acc;
        if constexpr (kInt)
          acc = A.total(c, Dn.scale);
        else
          acc = A.total(c);
        if (split)
          atomicAdd(yp + c, acc);
        else if (beta_mode == 0)
          yp[c] = acc;
        else if (beta_mode == 1)
          yp[c] = acc + yp[c];
        else
          yp[c] = fma(beta, yp[c], acc);
      }
    }
  }
  if (!fail && pos != (uint32_t)(gend - g0)) fail = kErrOverrun;
  rg.drain();
  phase_bits = rg.phase_bits;
  return fail;
}

}  // namespace core
}  // namespace dtans

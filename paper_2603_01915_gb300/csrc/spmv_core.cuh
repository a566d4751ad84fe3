// Per-warp machinery of the persistent CSR-dtANS decoder, shared by the
// single-matrix SpMV (spmv.cu) and the batched SpMV (batch.cu): the warp's
// bulk-copy ring of stream words and the segment decoder (Algorithm 3 with the
// readings of Sec. IV-D/IV-F).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "decode_common.cuh"
#include "dtans_internal.h"

namespace dtans {
namespace core {

using namespace dev;

constexpr uint32_t kRing = 512;                   // words per warp
constexpr uint32_t kChunk = 64;                   // words per bulk copy (256 B)
constexpr uint32_t kNumChunks = kRing / kChunk;   // 8
constexpr uint32_t kSpinLimit = 1u << 20;  // polls per wait before giving up

// Warp-private ring of stream words.  All lanes hold the same state; lane 0
// issues the copies.
struct Ring {
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
  __device__ uint32_t at(uint32_t pos) const { return ring[pos & (kRing - 1)]; }
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
};

// Where the products go: KT right-hand-side columns c0 .. c0 + KT - 1 of a
// row-major block with leading dimension ld.
template <typename V>
struct Dense {
  const V *__restrict__ x;
  V *__restrict__ y;
  uint32_t ld, c0;
};

// Per-lane accumulators for KT columns.  KT = 1 keeps two independent FMA
// chains and gathers x as soon as a column is known; KT > 1 gathers each
// row of X (KT contiguous values, 16-byte vector loads) after the state update.
template <typename V, int KT>
struct Cols {
  static constexpr int kVec = 16 / (int)sizeof(V);  // values per 16-byte load
  static_assert(KT % kVec == 0, "KT must fill whole 16-byte vectors");
  V acc[KT];
  uint32_t cc[4];
  __device__ __forceinline__ void reset() {
#pragma unroll
    for (int c = 0; c < KT; ++c) acc[c] = V(0);
  }
  __device__ __forceinline__ void at_column(int t, uint32_t col, const Dense<V> &D) { cc[t] = col; }
  __device__ __forceinline__ void skip(int t) { cc[t] = 0xffffffffu; }
  __device__ __forceinline__ void accumulate(const V (&v)[4], const Dense<V> &D) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (cc[t] == 0xffffffffu) continue;
      const V *row = D.x + (size_t)cc[t] * D.ld + D.c0;
      V xr[KT];
#pragma unroll
      for (int c = 0; c < KT; c += kVec) {
        if constexpr (sizeof(V) == 8) {
          const double2 q = __ldg((const double2 *)(row + c));
          xr[c] = q.x;
          xr[c + 1] = q.y;
        } else {
          const float4 q = __ldg((const float4 *)(row + c));
          xr[c] = q.x;
          xr[c + 1] = q.y;
          xr[c + 2] = q.z;
          xr[c + 3] = q.w;
        }
      }
#pragma unroll
      for (int c = 0; c < KT; ++c) acc[c] = fma(v[t], xr[c], acc[c]);
    }
  }
  __device__ __forceinline__ V total(int c) const { return acc[c]; }
};

template <typename V>
struct Cols<V, 1> {
  V acc0, acc1, xg[4];
  __device__ __forceinline__ void reset() { acc0 = acc1 = V(0); }
  __device__ __forceinline__ void at_column(int t, uint32_t col, const Dense<V> &D) { xg[t] = __ldg(D.x + col); }
  __device__ __forceinline__ void skip(int t) { xg[t] = V(0); }
  __device__ __forceinline__ void accumulate(const V (&v)[4], const Dense<V> &D) {
    acc0 = fma(v[0], xg[0], acc0);
    acc1 = fma(v[1], xg[1], acc1);
    acc0 = fma(v[2], xg[2], acc0);
    acc1 = fma(v[3], xg[3], acc1);
  }
  __device__ __forceinline__ V total(int) const { return acc0 + acc1; }
};

// One segment of four nonzeros (Algorithm 3, one iteration): unpack, table
// lookups, escape point, x gathers, two checks and the unconditional read,
// FMAs.  kFast: every lane of a full slice is live and not in its last
// segment.  kResident: the whole slice is already in the ring, so no read
// needs a ring check.  `lim` bounds pos (the slice end when resident, else the
// warp's range end); returns false when a read would pass it or the ring could
// not supply the words.
template <typename V, int KT, bool kFast, bool kResident>
__device__ __forceinline__ bool segment(LaneState &L, Cols<V, KT> &A, Ring &rg, uint32_t &pos, uint32_t lim,
                                        uint32_t j, const uint8_t *tD, const uint8_t *tV, const Dense<V> &Dn,
                                        uint32_t nm1, uint32_t lt, int lane) {
  using VE = ValueEntry<V>;
  constexpr int VS = sizeof(VE);
  constexpr uint32_t kRawV = RawWords<V>::kValue;
  uint32_t o[8];
  unpack_offsets<8, VS>(L.w0, L.w1, L.w2, o);
  if (!kResident) rg.refill(pos, lane);  // a resident slice was fetched whole at its start
  DeltaEntry eD[4];
  VE eV[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    eD[t] = *(const DeltaEntry *)(tD + o[2 * t]);
    eV[t] = *(const VE *)(tV + o[2 * t + 1]);
  }
  const uint32_t nvalid = kFast ? 4u : (j < L.nseg ? min(4u, L.n - 4 * j) : 0u);
  uint32_t escbits = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if (kFast || (uint32_t)t < nvalid) escbits |= eD[t].meta | eV[t].meta;
  if (__any_sync(kFull, escbits & kMetaEsc)) {
    // escape point: each lane's raw words of this segment, slot order, lanes in order
    uint32_t nraw = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (kFast || (uint32_t)t < nvalid)
        nraw += ((eD[t].meta & kMetaEsc) ? 1u : 0u) + ((eV[t].meta & kMetaEsc) ? kRawV : 0u);
    uint32_t tot;
    uint32_t p = pos + warp_prefix16(nraw, lt, tot);
    if (pos + tot > lim) return false;
    if (!kResident && !rg.ensure(pos, pos + tot, lane)) return false;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (!kFast && (uint32_t)t >= nvalid) continue;
      if (eD[t].meta & kMetaEsc) eD[t].delta = rg.at(p++);
      if (eV[t].meta & kMetaEsc) {
        if constexpr (kRawV == 2) {
          const uint32_t lo = rg.at(p), hi = rg.at(p + 1);
          eV[t].v = __hiloint2double((int)hi, (int)lo);
        } else {
          eV[t].v = __uint_as_float(rg.at(p));
        }
        p += kRawV;
      }
    }
    pos += tot;
  }
  // columns (clamped: every gather stays inside x); with KT = 1 the gathers
  // are issued here and consumed after the state update
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (kFast || (uint32_t)t < nvalid) {
      L.col += eD[t].delta;
      A.at_column(t, min(L.col, nm1), Dn);
    } else {
      A.skip(t);
      eV[t].v = V(0);
    }
  }
  // the checks and the unconditional read take at most 3 * 32 words
  if (pos > lim) return false;
  if (!kResident && !rg.ensure(pos, min(pos + 3 * kSlice, lim), lane)) return false;
  const bool more = kFast || j + 1 < L.nseg;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    bool need = false;
    uint32_t w = q == 0 ? L.w0 : L.w1;
    if (kFast || more)
      need = group_step(eD[2 * q].meta, eV[2 * q].meta, eD[2 * q + 1].meta, eV[2 * q + 1].meta, L.d, L.r, w);
    const uint32_t m = __ballot_sync(kFull, need);
    if (m) {  // warp-uniform; conditional reads (Sec. IV-B: one ballot, two popcounts)
      const uint32_t v = rg.at(pos + __popc(m & lt));
      w = need ? v : w;
      pos += __popc(m);
    }
    if (q == 0) L.w0 = w; else L.w1 = w;
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
  const V vals[4] = {eV[0].v, eV[1].v, eV[2].v, eV[3].v};
  A.accumulate(vals, Dn);
  // A valid stream never reads past `lim`.  Every segment in which some lane
  // is not in its last segment advances pos, so this check also bounds the
  // number of segments a corrupt row length can cause.
  return pos <= lim;
}

// The first `nfast` segments of a resident slice in which all 32 lanes are
// live and none is in its last segment, for one right-hand side: the same
// program as segment<V, 1, true, true>, written as one straight loop over
// plain registers (one uniform branch per rare event: escapes, conditional
// reads, and the range check).  Returns false when a read passes `lim`.
template <typename V>
__device__ __forceinline__ bool fast_run_kt1(LaneState &L, Cols<V, 1> &A, const uint32_t *ring, uint32_t &pos_io,
                                             uint32_t lim, uint32_t nfast, const uint8_t *tD, const uint8_t *tV,
                                             const V *__restrict__ x, uint32_t nm1, uint32_t lt, uint32_t lane) {
  using VE = ValueEntry<V>;
  constexpr int VS = sizeof(VE);
  constexpr uint32_t kRawV = RawWords<V>::kValue;
  constexpr uint32_t kMask = kRing - 1;
  uint32_t w0 = L.w0, w1 = L.w1, w2 = L.w2, d = L.d, r = L.r, col = L.col, pos = pos_io;
  V acc0 = A.acc0, acc1 = A.acc1;
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
    const uint32_t esc = (eD[0].meta | eD[1].meta | eD[2].meta | eD[3].meta | eV[0].meta | eV[1].meta |
                          eV[2].meta | eV[3].meta) & kMetaEsc;
    if (__any_sync(kFull, esc)) {
      uint32_t nraw = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        nraw += ((eD[t].meta & kMetaEsc) ? 1u : 0u) + ((eV[t].meta & kMetaEsc) ? kRawV : 0u);
      uint32_t tot;
      uint32_t p = pos + warp_prefix16(nraw, lt, tot);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (eD[t].meta & kMetaEsc) eD[t].delta = ring[p++ & kMask];
        if (eV[t].meta & kMetaEsc) {
          if constexpr (kRawV == 2) {
            const uint32_t lo = ring[p & kMask], hi = ring[(p + 1) & kMask];
            eV[t].v = __hiloint2double((int)hi, (int)lo);
          } else {
            eV[t].v = __uint_as_float(ring[p & kMask]);
          }
          p += kRawV;
        }
      }
      pos += tot;
    }
    V xg[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      col += eD[t].delta;
      xg[t] = __ldg(x + min(col, nm1));
    }
    const uint32_t all8 = eD[0].meta & eV[0].meta & eD[1].meta & eV[1].meta & eD[2].meta & eV[2].meta &
                          eD[3].meta & eV[3].meta;
    if (__all_sync(kFull, all_base_w(all8))) {
      // every group of every lane has radix W: both checks extract, state unchanged
      w0 = pack_digits(eD[0].meta, eV[0].meta, eD[1].meta, eV[1].meta);
      w1 = pack_digits(eD[2].meta, eV[2].meta, eD[3].meta, eV[3].meta);
    } else {
      const bool need0 = group_step(eD[0].meta, eV[0].meta, eD[1].meta, eV[1].meta, d, r, w0);
      uint32_t m = __ballot_sync(kFull, need0);
      if (m) {
        const uint32_t v = ring[(pos + __popc(m & lt)) & kMask];
        w0 = need0 ? v : w0;
        pos += __popc(m);
      }
      const bool need1 = group_step(eD[2].meta, eV[2].meta, eD[3].meta, eV[3].meta, d, r, w1);
      m = __ballot_sync(kFull, need1);
      if (m) {
        const uint32_t v = ring[(pos + __popc(m & lt)) & kMask];
        w1 = need1 ? v : w1;
        pos += __popc(m);
      }
    }
    w2 = ring[(pos + lane) & kMask];
    pos += kSlice;
    acc0 = fma(eV[0].v, xg[0], acc0);
    acc1 = fma(eV[1].v, xg[1], acc1);
    acc0 = fma(eV[2].v, xg[2], acc0);
    acc1 = fma(eV[3].v, xg[3], acc1);
    if (pos > lim) {  // a corrupt row length; each segment advances pos by >= 32
      ok = false;
      break;
    }
  }
  L.w0 = w0, L.w1 = w1, L.w2 = w2, L.d = d, L.r = r, L.col = col;
  A.acc0 = acc0, A.acc1 = acc1;
  pos_io = pos;
  return ok;
}

// The last segment when every lane of a full slice is in its last segment
// (all units of the slice have the same number of segments): no checks and
// no reads but the escape point; items past a lane's length are pads.
template <typename V>
__device__ __forceinline__ bool last_segment_kt1(LaneState &L, Cols<V, 1> &A, const uint32_t *ring, uint32_t &pos,
                                                 uint32_t lim, uint32_t j, const uint8_t *tD, const uint8_t *tV,
                                                 const V *__restrict__ x, uint32_t nm1, uint32_t lt) {
  using VE = ValueEntry<V>;
  constexpr int VS = sizeof(VE);
  constexpr uint32_t kRawV = RawWords<V>::kValue;
  constexpr uint32_t kMask = kRing - 1;
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
  uint32_t escbits = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t)
    if ((uint32_t)t < nvalid) escbits |= eD[t].meta | eV[t].meta;
  if (__any_sync(kFull, escbits & kMetaEsc)) {
    uint32_t nraw = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if ((uint32_t)t < nvalid)
        nraw += ((eD[t].meta & kMetaEsc) ? 1u : 0u) + ((eV[t].meta & kMetaEsc) ? kRawV : 0u);
    uint32_t tot;
    uint32_t p = pos + warp_prefix16(nraw, lt, tot);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if ((uint32_t)t >= nvalid) continue;
      if (eD[t].meta & kMetaEsc) eD[t].delta = ring[p++ & kMask];
      if (eV[t].meta & kMetaEsc) {
        if constexpr (kRawV == 2) {
          const uint32_t lo = ring[p & kMask], hi = ring[(p + 1) & kMask];
          eV[t].v = __hiloint2double((int)hi, (int)lo);
        } else {
          eV[t].v = __uint_as_float(ring[p & kMask]);
        }
        p += kRawV;
      }
    }
    pos += tot;
  }
  V xg[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if ((uint32_t)t < nvalid) {
      L.col += eD[t].delta;
      xg[t] = __ldg(x + min(L.col, nm1));
    } else {
      xg[t] = V(0);
      eV[t].v = V(0);
    }
  }
  A.acc0 = fma(eV[0].v, xg[0], A.acc0);
  A.acc1 = fma(eV[1].v, xg[1], A.acc1);
  A.acc0 = fma(eV[2].v, xg[2], A.acc0);
  A.acc1 = fma(eV[3].v, xg[3], A.acc1);
  return pos <= lim;
}

template <typename V, int KT, bool kResident>
__device__ __forceinline__ bool decode_unit_segments(LaneState &L, Cols<V, KT> &A, Ring &rg, uint32_t &pos,
                                                     uint32_t lim, uint32_t minseg, uint32_t maxseg, const uint8_t *tD,
                                                     const uint8_t *tV, const Dense<V> &Dn, uint32_t nm1,
                                                     uint32_t lt, int lane) {
  uint32_t j = 0;
  if constexpr (KT == 1 && kResident) {
    if (minseg >= 2) {
      if (!fast_run_kt1<V>(L, A, rg.ring, pos, lim, minseg - 1, tD, tV, Dn.x, nm1, lt, (uint32_t)lane)) return false;
      j = minseg - 1;
    }
    if (minseg >= 1 && minseg == maxseg)  // every lane is now in its last segment
      return last_segment_kt1<V>(L, A, rg.ring, pos, lim, j, tD, tV, Dn.x, nm1, lt);
  } else {
    for (; j + 1 < minseg; ++j)
      if (!segment<V, KT, true, kResident>(L, A, rg, pos, lim, j, tD, tV, Dn, nm1, lt, lane)) return false;
  }
  for (; j < maxseg; ++j)
    if (!segment<V, KT, false, kResident>(L, A, rg, pos, lim, j, tD, tV, Dn, nm1, lt, lane)) return false;
  return true;
}

template <typename V>
constexpr int table_bytes() {
  return kK * 8 + kK * (int)sizeof(ValueEntry<V>);
}

template <typename V>
constexpr int persistent_smem_bytes(int warps) {
  return table_bytes<V>() + warps * (int)(kRing * 4) + warps * (int)kNumChunks * 8;
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
// Returns 0 or an error code.
template <typename V, int KT>
__device__ int32_t warp_spmv_range(const uint32_t *__restrict__ words, const uint64_t *__restrict__ slice_off,
                                   const uint32_t *__restrict__ unit_row, int64_t nunits, uint32_t ncols,
                                   uint32_t s0, uint32_t s1, const uint8_t *tD, const uint8_t *tV,
                                   uint32_t *ring_base, uint64_t *bars, const Dense<V> &Dn, V beta,
                                   int32_t beta_mode, int32_t *err, uint32_t &phase_bits, int lane) {
  if (s0 >= s1) return 0;
  const uint64_t gbeg = slice_off[s0], gend = slice_off[s1];
  const uint64_t g0 = gbeg & ~3ull;
  const uint64_t span = ((gend + 3) & ~3ull) - g0;
  if (span >= (1ull << 31)) return kErrRange;
  Ring rg;
  rg.src = words + g0;
  rg.bar = smem_addr(bars);
  rg.ring = ring_base;
  rg.total = (uint32_t)span;
  rg.nchunks = (rg.total + kChunk - 1) / kChunk;
  rg.issued = 0;
  rg.ready = 0;
  rg.phase_bits = phase_bits;
  rg.refill(0, lane);
  const uint32_t lt = lanemask_lt();
  const uint32_t nm1 = ncols - 1;
  uint32_t pos = (uint32_t)(gbeg - g0);
  int32_t fail = 0;

  for (uint32_t s = s0; s < s1; ++s) {
    // every slice must start where the previous one ended (a corrupt stream
    // is caught here; reads in between stay inside the ring by masking)
    if (pos != (uint32_t)(slice_off[s] - g0)) {
      fail = kErrOverrun;
      break;
    }
    const int64_t u0 = (int64_t)s * kSlice;
    const uint32_t nl = (uint32_t)min((int64_t)kSlice, nunits - u0);
    if (!rg.ensure(pos, pos + nl, lane)) {
      fail = kErrOverrun;
      break;
    }
    LaneState L;
    Cols<V, KT> A;
    const bool has = (uint32_t)lane < nl;
    L.n = has ? rg.at(pos + lane) : 0u;
    pos += nl;
    L.w0 = L.w1 = L.w2 = 0;
    {
      const uint32_t m = __ballot_sync(kFull, L.n > 0);
      const uint32_t cnt = __popc(m), rk = __popc(m & lt);
      if (!rg.ensure(pos, pos + 3 * cnt, lane)) {
        fail = kErrOverrun;
        break;
      }
      if (L.n > 0) {
        L.w0 = rg.at(pos + rk);
        L.w1 = rg.at(pos + cnt + rk);
        L.w2 = rg.at(pos + 2 * cnt + rk);
      }
      pos += 3 * cnt;
    }
    L.nseg = (L.n + 3) >> 2;
    const uint32_t maxseg = __reduce_max_sync(kFull, L.nseg);
    const uint32_t minseg = __reduce_min_sync(kFull, L.nseg);  // lanes past nl count as 0
    L.d = 0;
    L.r = 1;
    L.col = 0;
    A.reset();
    // A slice whose words all fit in the ring window is made resident once;
    // its segments then read without ring checks.
    const uint32_t se = (uint32_t)(slice_off[s + 1] - g0);
    const bool resident = se - (pos & ~(kChunk - 1)) <= kRing && se <= rg.total;
    bool ok;
    if (resident) {
      ok = rg.ensure(pos, se, lane) &&
           decode_unit_segments<V, KT, true>(L, A, rg, pos, se, minseg, maxseg, tD, tV, Dn, nm1, lt, lane);
    } else {
      ok = decode_unit_segments<V, KT, false>(L, A, rg, pos, rg.total, minseg, maxseg, tD, tV, Dn, nm1, lt, lane);
    }
    if (!ok) {
      fail = kErrOverrun;
      break;
    }
    if (has) {
      if (L.n > 0 && L.col > nm1) atomicExch(err, kErrColumn);
      const int64_t u = u0 + lane;
      uint32_t row = (uint32_t)u;
      bool split = false;
      if (unit_row) {
        const uint32_t ur = __ldg(unit_row + u);
        row = ur & 0x7fffffffu;
        split = (ur >> 31) != 0;
      }
      V *yp = KT == 1 ? Dn.y + row : Dn.y + (size_t)row * Dn.ld + Dn.c0;
#pragma unroll
      for (int c = 0; c < KT; ++c) {
        const V acc = A.total(c);
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

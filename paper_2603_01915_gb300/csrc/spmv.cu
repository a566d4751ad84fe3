// Decode-fused single-vector SpMV of CSR-dtANS for GB300 (sm_103a).
//
// Persistent kernel, one CTA of 32 warps per SM.  Each warp owns a contiguous
// range of slices whose interleaved words form one contiguous range of the
// stream; the warp streams that range into a private 2 KB shared-memory ring
// with 1-D bulk copies (cp.async.bulk, 256 B each, completion on one mbarrier
// per ring chunk), up to 8 chunks ahead of the word it is decoding.  All
// stream reads of the lock-step decoder (row lengths, initial words, escaped
// raw symbols, conditional and unconditional reads; Algorithm 3 and Sec. IV-B)
// are then shared-memory loads.  Both coding tables sit in shared memory
// (Sec. IV-F).  The x gathers of a segment are issued as soon as its columns
// are known and consumed after the state update, so their latency overlaps
// the decoder's work.  Segments in which every lane of a full slice is past
// its first and before its last segment take a path without per-lane
// predicates.
//
// Every wait on a ring chunk is bounded: after the limit the warp records an
// error, waits (bounded) for its own copies in flight and stops.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "decode_common.cuh"
#include "dtans_internal.h"

namespace dtans {
namespace {

using namespace dev;

constexpr int kThreads = 1024;
constexpr int kWarpsPerCta = kThreads / 32;
constexpr uint32_t kRing = 512;                   // words per warp
constexpr uint32_t kChunk = 64;                   // words per bulk copy (256 B)
constexpr uint32_t kNumChunks = kRing / kChunk;   // 8
constexpr uint32_t kSpinLimit = 1u << 20;  // polls per wait before giving up

template <typename V>
struct SpmvArgs {
  const uint32_t *words;
  const uint64_t *slice_off;
  const uint8_t *tables;
  const uint32_t *unit_row;    // null: unit u is row u
  const uint32_t *warp_slice;  // [nwarps + 1] first slice of each warp
  int64_t nunits;
  uint32_t ncols;
  int32_t *err;
  const V *x;
  V *y;
  V beta;
  int32_t beta_mode;  // 0: y = Ax, 1: y += Ax (y pre-scaled), 2: y = Ax + beta y
};

template <typename V>
constexpr int table_bytes() {
  return kK * 8 + kK * (int)sizeof(ValueEntry<V>);
}

template <typename V>
constexpr int spmv_smem_bytes() {
  return table_bytes<V>() + kWarpsPerCta * (int)(kRing * 4) + kWarpsPerCta * (int)kNumChunks * 8;
}

// Warp-private ring of stream words.  All lanes hold the same state; lane 0
// issues the copies.
struct Ring {
  const uint32_t *src;  // global address of word 0 of the warp's range (16-byte aligned)
  uint32_t buf;         // shared address of the ring
  uint32_t bar;         // shared address of barrier 0
  uint32_t total;       // words in the range (multiple of 4)
  uint32_t nchunks, issued, ready;
  const uint32_t *ring; // generic pointer to the ring

  __device__ void issue_upto(uint32_t lim, int lane) {
    if (issued >= lim) return;
    __syncwarp();  // every lane is done with the chunks being recycled
    fence_proxy_async();
    for (uint32_t c = issued; c < lim; ++c) {
      const uint32_t w0 = c * kChunk;
      const uint32_t nw = min(kChunk, total - w0);
      bulk_load(lane == 0, buf + (c % kNumChunks) * kChunk * 4, src + w0, nw * 4, bar + (c % kNumChunks) * 8);
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
      if (!mbar_wait_warp(bar + (ready % kNumChunks) * 8, (ready / kNumChunks) & 1u, kSpinLimit)) return false;
      ++ready;
    }
    return true;
  }
  __device__ uint32_t at(uint32_t pos) const { return ring[pos & (kRing - 1)]; }
  // Waits (bounded) for every copy still in flight.
  __device__ void drain() {
    while (ready < issued) {
      if (!mbar_wait_warp(bar + (ready % kNumChunks) * 8, (ready / kNumChunks) & 1u, kSpinLimit)) break;
      ++ready;
    }
  }
};

// Decoder state of one lane (one unit) while a warp decodes a slice.
template <typename V>
struct LaneState {
  uint32_t w0, w1, w2;  // the three words unpacked into the next segment
  uint32_t d, r;        // dtANS decoder state (digit, radix), both < 2^32
  uint32_t col;         // running column (the first delta is absolute)
  uint32_t n, nseg;     // entries and segments of the unit
  V acc0, acc1;         // two partial sums (independent FMA chains)
};

// One segment of four nonzeros (Algorithm 3, one iteration): unpack, table
// lookups, escape point, x gathers, two checks and the unconditional read,
// FMAs.  kFast: every lane of a full slice is live and not in its last
// segment.  kResident: the whole slice is already in the ring, so no read
// needs a ring check.  `lim` bounds pos (the slice end when resident, else the
// warp's range end); returns false when a read would pass it or the ring could
// not supply the words.
template <typename V, bool kFast, bool kResident>
__device__ __forceinline__ bool segment(LaneState<V> &L, Ring &rg, uint32_t &pos, uint32_t lim, uint32_t j,
                                        const uint8_t *tD, const uint8_t *tV, const V *__restrict__ x, uint32_t nm1,
                                        uint32_t lt, int lane) {
  using VE = ValueEntry<V>;
  constexpr int VS = sizeof(VE);
  constexpr uint32_t kRawV = RawWords<V>::kValue;
  uint32_t o[8];
  unpack_offsets<8, VS>(L.w0, L.w1, L.w2, o);
  rg.refill(pos, lane);
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
  // gathers of x as soon as the columns are known; consumed after the state update
  V xg[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (kFast || (uint32_t)t < nvalid) {
      L.col += eD[t].delta;
      xg[t] = __ldg(x + min(L.col, nm1));
    } else {
      xg[t] = V(0);
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
  L.acc0 = fma(eV[0].v, xg[0], L.acc0);
  L.acc1 = fma(eV[1].v, xg[1], L.acc1);
  L.acc0 = fma(eV[2].v, xg[2], L.acc0);
  L.acc1 = fma(eV[3].v, xg[3], L.acc1);
  // A valid stream never reads past `lim`.  Every segment in which some lane
  // is not in its last segment advances pos, so this check also bounds the
  // number of segments a corrupt row length can cause.
  return pos <= lim;
}

template <typename V, bool kResident>
__device__ __forceinline__ bool decode_unit_segments(LaneState<V> &L, Ring &rg, uint32_t &pos, uint32_t lim,
                                                     uint32_t minseg, uint32_t maxseg, const uint8_t *tD,
                                                     const uint8_t *tV, const V *__restrict__ x, uint32_t nm1,
                                                     uint32_t lt, int lane) {
  uint32_t j = 0;
  for (; j + 1 < minseg; ++j)
    if (!segment<V, true, kResident>(L, rg, pos, lim, j, tD, tV, x, nm1, lt, lane)) return false;
  for (; j < maxseg; ++j)
    if (!segment<V, false, kResident>(L, rg, pos, lim, j, tD, tV, x, nm1, lt, lane)) return false;
  return true;
}

template <typename V>
__global__ void __launch_bounds__(kThreads, 1) spmv_kernel(SpmvArgs<V> a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  {
    const uint4 *src = (const uint4 *)a.tables;
    uint4 *dst = (uint4 *)smem;
    for (int i = threadIdx.x; i < table_bytes<V>() / 16; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  uint32_t *ring_base = (uint32_t *)(smem + table_bytes<V>()) + wid * kRing;
  uint64_t *bars = (uint64_t *)(smem + table_bytes<V>() + kWarpsPerCta * kRing * 4) + wid * kNumChunks;
  if (lane == 0) {
    for (uint32_t c = 0; c < kNumChunks; ++c) mbar_init(smem_addr(bars + c), 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint8_t *tD = smem;
  const uint8_t *tV = smem + kK * 8;

  const int64_t gw = (int64_t)blockIdx.x * kWarpsPerCta + wid;
  const uint32_t s0 = a.warp_slice[gw], s1 = a.warp_slice[gw + 1];
  if (s0 >= s1) return;
  const uint64_t gbeg = a.slice_off[s0], gend = a.slice_off[s1];
  const uint64_t g0 = gbeg & ~3ull;
  const uint64_t span = ((gend + 3) & ~3ull) - g0;
  if (span >= (1ull << 31)) {
    if (lane == 0) atomicExch(a.err, kErrRange);
    return;
  }
  Ring rg;
  rg.src = a.words + g0;
  rg.buf = smem_addr(ring_base);
  rg.bar = smem_addr(bars);
  rg.ring = ring_base;
  rg.total = (uint32_t)span;
  rg.nchunks = (rg.total + kChunk - 1) / kChunk;
  rg.issued = 0;
  rg.ready = 0;
  rg.refill(0, lane);
  const uint32_t lt = lanemask_lt();
  const uint32_t nm1 = a.ncols - 1;
  uint32_t pos = (uint32_t)(gbeg - g0);
  int32_t fail = 0;

  for (uint32_t s = s0; s < s1; ++s) {
    // every slice must start where the previous one ended (a corrupt stream
    // is caught here; reads in between stay inside the ring by masking)
    if (pos != (uint32_t)(a.slice_off[s] - g0)) {
      fail = kErrOverrun;
      break;
    }
    const int64_t u0 = (int64_t)s * kSlice;
    const uint32_t nl = (uint32_t)min((int64_t)kSlice, a.nunits - u0);
    if (!rg.ensure(pos, pos + nl, lane)) {
      fail = kErrOverrun;
      break;
    }
    LaneState<V> L;
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
    L.acc0 = V(0);
    L.acc1 = V(0);
    // A slice whose words all fit in the ring window is made resident once;
    // its segments then read without ring checks.
    const uint32_t se = (uint32_t)(a.slice_off[s + 1] - g0);
    const bool resident = se - (pos & ~(kChunk - 1)) <= kRing && se <= rg.total;
    bool ok;
    if (resident) {
      ok = rg.ensure(pos, se, lane) &&
           decode_unit_segments<V, true>(L, rg, pos, se, minseg, maxseg, tD, tV, a.x, nm1, lt, lane);
    } else {
      ok = decode_unit_segments<V, false>(L, rg, pos, rg.total, minseg, maxseg, tD, tV, a.x, nm1, lt, lane);
    }
    if (!ok) {
      fail = kErrOverrun;
      break;
    }
    if (has) {
      if (L.n > 0 && L.col > nm1) atomicExch(a.err, kErrColumn);
      const V acc = L.acc0 + L.acc1;
      const int64_t u = u0 + lane;
      uint32_t row = (uint32_t)u;
      bool split = false;
      if (a.unit_row) {
        const uint32_t ur = __ldg(a.unit_row + u);
        row = ur & 0x7fffffffu;
        split = (ur >> 31) != 0;
      }
      V *yp = a.y + row;
      if (split)
        atomicAdd(yp, acc);
      else if (a.beta_mode == 0)
        *yp = acc;
      else if (a.beta_mode == 1)
        *yp = acc + *yp;
      else
        *yp = fma(a.beta, *yp, acc);
    }
  }
  if (!fail && pos != (uint32_t)(gend - g0)) fail = kErrOverrun;
  if (fail && lane == 0) atomicExch(a.err, fail);
  rg.drain();
}

dtans_status fail_cuda(cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return set_error(DTANS_ERR_CUDA, m);
}

// Splits the slices into `nwarps` contiguous ranges of about equal word count.
std::vector<uint32_t> warp_ranges(const dtans_handle_s &H, int64_t nwarps) {
  std::vector<uint32_t> r(nwarps + 1);
  const uint64_t total = H.slice_off.empty() ? 0 : H.slice_off.back();
  int64_t s = 0;
  for (int64_t w = 0; w <= nwarps; ++w) {
    const uint64_t target = (uint64_t)((__int128)total * w / nwarps);
    while (s < H.nslices && H.slice_off[s] < target) ++s;
    r[w] = (uint32_t)s;
  }
  r[nwarps] = (uint32_t)H.nslices;
  return r;
}

template <typename V>
dtans_status launch_spmv(dtans_handle_s &H, const void *x, void *y, double beta, cudaStream_t st) {
  cudaError_t e;
  static thread_local int configured = 0;
  const int smem = spmv_smem_bytes<V>();
  if (!configured) {
    if ((e = cudaFuncSetAttribute(spmv_kernel<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return fail_cuda(e, "cudaFuncSetAttribute(spmv)");
    configured = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = H.grid ? H.grid : sms;
  const int64_t nwarps = (int64_t)grid * kWarpsPerCta;
  if (H.d_warp_slice == nullptr || H.warp_slice_n != nwarps) {
    std::vector<uint32_t> r = warp_ranges(H, nwarps);
    cudaFree(H.d_warp_slice);
    H.d_warp_slice = nullptr;
    if ((e = cudaMalloc(&H.d_warp_slice, r.size() * 4)) != cudaSuccess) return fail_cuda(e, "cudaMalloc(ranges)");
    if ((e = cudaMemcpy(H.d_warp_slice, r.data(), r.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail_cuda(e, "cudaMemcpy(ranges)");
    H.warp_slice_n = nwarps;
  }
  SpmvArgs<V> a{};
  a.words = H.d_words;
  a.slice_off = H.d_slice_off;
  a.tables = H.d_tables;
  a.unit_row = H.d_unit_row;
  a.warp_slice = H.d_warp_slice;
  a.nunits = H.nunits;
  a.ncols = (uint32_t)std::max<int64_t>(H.n, 1);
  a.err = H.d_err;
  a.x = (const V *)x;
  a.y = (V *)y;
  a.beta = (V)beta;
  if (H.any_split) {
    a.beta_mode = 1;
  } else {
    a.beta_mode = beta == 0.0 ? 0 : (beta == 1.0 ? 1 : 2);
  }
  spmv_kernel<V><<<grid, kThreads, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "spmv launch");
  return DTANS_OK;
}

}  // namespace

dtans_status spmv_persistent(dtans_handle_s &H, const void *x, void *y, double beta, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  return H.dtype == DTANS_F64 ? launch_spmv<double>(H, x, y, beta, st) : launch_spmv<float>(H, x, y, beta, st);
}

}  // namespace dtans

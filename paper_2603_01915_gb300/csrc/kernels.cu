// CUDA kernels of the CSR-dtANS library for GB300 (sm_103a).
//
// One decoder serves every product: a warp decodes a slice of 32 units (one
// unit per lane, Sec. II "SpMVM"), segment by segment (4 nonzeros, Sec. IV-B),
// with both coding tables resident in shared memory (Sec. IV-F "Tables in
// shared memory").  The word stream is read where the warp's lock-step program
// needs it; offsets of conditional reads come from one ballot and two
// popcounts (Sec. IV-B).  What happens to each decoded nonzero depends on the
// mode: accumulate a * X[col, :] (forward), scatter a * G[row, :] (transpose),
// emit <G[row, :], X[col, :]> (value gradient), add it to the bin of the
// entry's value symbol (codebook gradient) or write (col, a) (decode).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "decode_common.cuh"
#include "dtans_internal.h"
#include "smem_limit.h"

namespace dtans {
namespace {

constexpr unsigned kFull = 0xffffffffu;

enum Mode { kFwd = 0, kTrans = 1, kValsGrad = 2, kDecode = 3, kCodeGrad = 4 };

// Error codes written to the handle's device word.
enum : int32_t { kErrOverrun = 1, kErrColumn = 2 };

template <typename V>
struct VEntry;
template <>
struct VEntry<double> {
  using T = uint4;  // {lo, hi, meta, 0}
  static constexpr int kRaw = 2;
  __device__ static uint32_t meta(const uint4 &e) { return e.z; }
  __device__ static double value(const uint4 &e) { return __hiloint2double((int)e.y, (int)e.x); }
};
template <>
struct VEntry<float> {
  using T = uint2;  // {bits, meta}
  static constexpr int kRaw = 1;
  __device__ static uint32_t meta(const uint2 &e) { return e.y; }
  __device__ static float value(const uint2 &e) { return __uint_as_float(e.x); }
};

struct Args {
  const uint32_t *words;
  const uint64_t *slice_off;
  const uint8_t *tables;
  const uint32_t *unit_row;  // null: unit u is row u
  const uint64_t *unit_pos;
  int64_t nunits, nslices, ncols, nnz;
  int32_t first_rel;  // first delta of a unit relative to its row
  int32_t chain;      // slices per chain: a warp decodes a chain's slices in order, carrying the state
  const uint32_t *esc;         // separate escape stream, or null (raw words in the stream)
  const uint64_t *esc_off;     // its offset per slice
  int32_t *err;
  int32_t ld;    // columns of the dense blocks (k)
  int32_t c0;    // first column of this pass
  const void *A; // X (forward), G (transpose, value gradient)
  const void *B; // X (value gradient)
  void *Y;       // Y, XG, gradient out, or decoded columns
  void *Y2;      // decoded values
  double beta;
  int32_t beta_mode;  // 0: overwrite, 1: accumulate, 2: scale by beta (forward, unsplit rows)
  int32_t accumulate; // value gradient: add to out (later column passes)
  const uint16_t *vrank;  // codebook gradient: bin of each stored value slot
  int32_t nbins;          // codebook gradient: kept value symbols + 1 (escaped values)
  int32_t vecA, vecB;     // rows of A / B at column c0 start on 16-byte (1) or 32-byte (2) boundaries
  int32_t vecY;           // rows of Y start on 16-byte boundaries at column c0
  int32_t aggregate;      // transpose: warp-aggregated atomics (lanes adding to one column merge first)
};

// Loads KT consecutive values from p: 16-byte vector loads when `vec` (p
// 16-byte aligned and KT values fill whole vectors), else one load each.
template <typename V, int KT>
__device__ __forceinline__ void load_row(const V *p, int32_t vec, V (&out)[KT]) {
  constexpr int kVec = 16 / (int)sizeof(V);
  if constexpr ((KT * sizeof(V)) % 32 == 0) {
    if (vec == 2) {  // rows of whole 32-byte sectors on sector boundaries: one sector per load
#pragma unroll
      for (int c = 0; c < KT; c += 32 / (int)sizeof(V)) dev::ldg32(p + c, &out[c]);
      return;
    }
  }
  if constexpr (KT % kVec == 0) {
    if (vec) {
#pragma unroll
      for (int c = 0; c < KT; c += kVec) {
        if constexpr (sizeof(V) == 8) {
          const double2 q = __ldg((const double2 *)(p + c));
          out[c] = q.x;
          out[c + 1] = q.y;
        } else {
          const float4 q = __ldg((const float4 *)(p + c));
          out[c] = q.x;
          out[c + 1] = q.y;
          out[c + 2] = q.z;
          out[c + 3] = q.w;
        }
      }
      return;
    }
  }
#pragma unroll
  for (int c = 0; c < KT; ++c) out[c] = __ldg(p + c);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename V>
__device__ __forceinline__ void atomic_add(V *p, V v) {
  atomicAdd(p, v);
}

// A lane's decoder state between the slices of a chain.
struct ChainState {
  uint32_t w0, w1, w2, d, r;
};

template <typename V, int KT, int MODE>
__device__ __forceinline__ void decode_slice(const Args &a, const uint2 *__restrict__ tD,
                                             const typename VEntry<V>::T *__restrict__ tV, int64_t s, int lane,
                                             V *bins, const uint16_t *vrank, ChainState &cs, bool start) {
  using VE = VEntry<V>;
  const uint64_t base = a.slice_off[s];
  const uint32_t wlen = (uint32_t)(a.slice_off[s + 1] - base);
  const uint32_t *__restrict__ w = a.words + base;
  const int64_t u0 = s * kSlice;
  const int nl = (int)min((int64_t)kSlice, a.nunits - u0);
  const uint32_t lt = lanemask_lt();
  if ((uint32_t)nl > wlen) {
    if (lane == 0) atomicExch(a.err, kErrOverrun);
    return;
  }
  // separate escape stream of this slice (if any)
  const uint32_t *ew = nullptr;
  uint32_t epos = 0, elen = 0;
  if (a.esc) {
    const uint64_t e0 = a.esc_off[s];
    ew = a.esc + e0;
    elen = (uint32_t)(a.esc_off[s + 1] - e0);
  }
  const bool has = lane < nl;
  const uint32_t nword = has ? __ldg(w + lane) : 0u;  // n | continues << 31
  const uint32_t n = nword & 0x7fffffffu;
  const bool cont = (nword >> 31) != 0;
  uint32_t pos = (uint32_t)nl;
  uint32_t w0 = cs.w0, w1 = cs.w1, w2 = cs.w2, d = cs.d, r = cs.r;
  if (start) {  // a chain starts: lanes with entries now or later read their initial words
    const bool act = n > 0 || cont;
    const uint32_t m = __ballot_sync(kFull, act);
    const uint32_t cnt = __popc(m), rk = __popc(m & lt);
    if (pos + 3 * cnt > wlen) {
      if (lane == 0) atomicExch(a.err, kErrOverrun);
      return;
    }
    w0 = w1 = w2 = 0;
    if (act) {
      w0 = __ldg(w + pos + rk);
      w1 = __ldg(w + pos + cnt + rk);
      w2 = __ldg(w + pos + 2 * cnt + rk);
    }
    pos += 3 * cnt;
    d = 0;
    r = 1;
  }
  const uint32_t nseg = (n + 3) >> 2;
  const uint32_t maxseg = __reduce_max_sync(kFull, nseg);

  // unit context
  const int64_t u = u0 + lane;
  uint32_t row = (uint32_t)u;
  bool split = false;
  if (a.unit_row && has) {
    const uint32_t ur = __ldg(a.unit_row + u);
    row = ur & 0x7fffffffu;
    split = (ur >> 31) != 0;
  }
  const int ld = a.ld;
  V acc[KT];
  V gv[KT];
#pragma unroll
  for (int t = 0; t < KT; ++t) acc[t] = V(0), gv[t] = V(0);
  uint64_t opos = 0;
  if (MODE == kTrans || MODE == kValsGrad || MODE == kCodeGrad) {
    if (n > 0) {
      load_row<V, KT>((const V *)a.A + (size_t)row * ld + a.c0, a.vecA, gv);
    }
  }
  if ((MODE == kValsGrad || MODE == kDecode) && has) opos = __ldg(a.unit_pos + u);

  uint32_t col = a.first_rel ? row : 0u;  // the running column starts at 0 or at the row
  for (uint32_t j = 0; j < maxseg; ++j) {
    const bool live = j < nseg;
    const bool more = live && (j + 1 < nseg || cont);  // only the chain's final segment stops
    // unpack: N = w0:w1:w2 (w0 most significant), slot k = bits [12k, 12k + 12)
    uint32_t sl[8];
    sl[0] = w2 & 0xfffu;
    sl[1] = (w2 >> 12) & 0xfffu;
    sl[2] = __funnelshift_r(w2, w1, 24) & 0xfffu;
    sl[3] = (w1 >> 4) & 0xfffu;
    sl[4] = (w1 >> 16) & 0xfffu;
    sl[5] = __funnelshift_r(w1, w0, 28) & 0xfffu;
    sl[6] = (w0 >> 8) & 0xfffu;
    sl[7] = w0 >> 20;
    uint2 eD[4];
    typename VE::T eV[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      eD[t] = tD[sl[2 * t]];
      eV[t] = tV[sl[2 * t + 1]];
    }
    const int nvalid = live ? (int)min(4u, n - 4 * j) : 0;
    // escape point: raw words of this segment, slot order, lanes in order
    uint32_t nraw = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (t < nvalid) {
        nraw += (eD[t].y & kMetaEsc) ? 1u : 0u;
        nraw += (VE::meta(eV[t]) & kMetaEsc) ? (uint32_t)VE::kRaw : 0u;
      }
    if (__any_sync(kFull, nraw != 0)) {
      uint32_t incl = nraw;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
      }
      const uint32_t tot = __shfl_sync(kFull, incl, 31);
      // the raw words: at the escape point of the stream, or in the separate
      // escape stream at the same running position
      const uint32_t *rw = a.esc ? ew : w;
      uint32_t &rpos = a.esc ? epos : pos;
      if (rpos + tot > (a.esc ? elen : wlen)) {
        if (lane == 0) atomicExch(a.err, kErrOverrun);
        return;
      }
      uint32_t p = rpos + incl - nraw;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < nvalid) {
          if (eD[t].y & kMetaEsc) eD[t].x = __ldg(rw + p++);
          if (VE::meta(eV[t]) & kMetaEsc) {
            if constexpr (VE::kRaw == 2) {
              eV[t].x = __ldg(rw + p);
              eV[t].y = __ldg(rw + p + 1);
            } else {
              eV[t].x = __ldg(rw + p);
            }
            p += VE::kRaw;
          }
        }
      rpos += tot;
    }
    // two checks, each after a group of four digits (Sec. IV-D, IV-F)
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      bool need = false;
      if (more) {
        uint32_t wx = 0;
        need = dev::group_step(eD[2 * q].y, VE::meta(eV[2 * q]), eD[2 * q + 1].y, VE::meta(eV[2 * q + 1]), d, r, wx);
        if (!need) {
          if (q == 0) w0 = wx; else w1 = wx;
        }
      }
      const uint32_t m = __ballot_sync(kFull, need);
      if (m) {
        const uint32_t cnt = __popc(m);
        if (pos + cnt > wlen) {
          if (lane == 0) atomicExch(a.err, kErrOverrun);
          return;
        }
        if (need) {
          const uint32_t wx = __ldg(w + pos + __popc(m & lt));
          if (q == 0) w0 = wx; else w1 = wx;
        }
        pos += cnt;
      }
    }
    {
      const uint32_t m = __ballot_sync(kFull, more);
      if (m) {
        const uint32_t cnt = __popc(m);
        if (pos + cnt > wlen) {
          if (lane == 0) atomicExch(a.err, kErrOverrun);
          return;
        }
        if (more) w2 = __ldg(w + pos + __popc(m & lt));
        pos += cnt;
      }
    }
    // the decoded nonzeros
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t >= nvalid) continue;
      col += eD[t].x;
      const V v = VE::value(eV[t]);
      if ((int64_t)col >= a.ncols) {
        atomicExch(a.err, kErrColumn);
        continue;
      }
      if constexpr (MODE == kFwd) {
        V xr[KT];
        load_row<V, KT>((const V *)a.A + (size_t)col * ld + a.c0, a.vecA, xr);
#pragma unroll
        for (int c = 0; c < KT; ++c) acc[c] = fma(v, xr[c], acc[c]);
      } else if constexpr (MODE == kTrans) {
        V *xg = (V *)a.Y + (size_t)col * ld + a.c0;
        if (a.aggregate) {
          // Warp-aggregated atomics: the lanes here that add to the same
          // column (one match) pass their contributions to the lowest of them
          // by shuffles, which then issues one atomic per column of the tile.
          // The lanes taking this branch together are the active mask.
          const uint32_t act = __activemask();
          const uint32_t peers = __match_any_sync(act, col);
          const int gmax = (int)__reduce_max_sync(act, (uint32_t)__popc(peers));
          if (gmax > 1) {
            const int leader = __ffs(peers) - 1;
            V tot[KT];
#pragma unroll
            for (int c = 0; c < KT; ++c) tot[c] = v * gv[c];
            uint32_t others = peers & ~(1u << leader);
            for (int k = 1; k < gmax; ++k) {
              const int src = others ? __ffs(others) - 1 : lane;
              others &= others - 1u;
#pragma unroll
              for (int c = 0; c < KT; ++c) {
                const V o = __shfl_sync(act, v * gv[c], src);
                if (lane == leader && src != lane) tot[c] += o;
              }
            }
            if (lane == leader) {
              if constexpr (sizeof(V) == 4 && KT % 4 == 0) {
                if (a.vecY) {
#pragma unroll
                  for (int c = 0; c < KT; c += 4)
                    atomicAdd((float4 *)(xg + c), make_float4(tot[c], tot[c + 1], tot[c + 2], tot[c + 3]));
                  continue;
                }
              }
#pragma unroll
              for (int c = 0; c < KT; ++c) atomic_add(xg + c, tot[c]);
            }
            continue;
          }
        }
        if constexpr (sizeof(V) == 4 && KT % 4 == 0) {
          if (a.vecY) {  // one 16-byte vector atomic per four columns
#pragma unroll
            for (int c = 0; c < KT; c += 4)
              atomicAdd((float4 *)(xg + c), make_float4(v * gv[c], v * gv[c + 1], v * gv[c + 2], v * gv[c + 3]));
            continue;
          }
        }
#pragma unroll
        for (int c = 0; c < KT; ++c) atomic_add(xg + c, v * gv[c]);
      } else if constexpr (MODE == kValsGrad) {
        if (opos + 4 * j + t >= (uint64_t)a.nnz) {
          atomicExch(a.err, kErrOverrun);
          continue;
        }
        V xr[KT];
        load_row<V, KT>((const V *)a.B + (size_t)col * ld + a.c0, a.vecB, xr);
        V sdot = V(0);
#pragma unroll
        for (int c = 0; c < KT; ++c) sdot = fma(gv[c], xr[c], sdot);
        V *o = (V *)a.Y + opos + 4 * j + t;
        *o = a.accumulate ? *o + sdot : sdot;
      } else if constexpr (MODE == kCodeGrad) {
        // d L / d c_r sums <G[row, :], X[col, :]> over the entries whose value
        // is kept symbol r (the last bin collects escaped values)
        V xr[KT];
        load_row<V, KT>((const V *)a.B + (size_t)col * ld + a.c0, a.vecB, xr);
        V sdot = V(0);
#pragma unroll
        for (int c = 0; c < KT; ++c) sdot = fma(gv[c], xr[c], sdot);
        atomicAdd(bins + vrank[sl[2 * t + 1]], sdot);
      } else {
        if (opos + 4 * j + t >= (uint64_t)a.nnz) {
          atomicExch(a.err, kErrOverrun);
          continue;
        }
        ((uint32_t *)a.Y)[opos + 4 * j + t] = col;
        ((V *)a.Y2)[opos + 4 * j + t] = v;
      }
    }
  }
  cs = ChainState{w0, w1, w2, d, r};
  if constexpr (MODE == kFwd) {
    if (has) {
      V *y = (V *)a.Y + (size_t)row * ld + a.c0;
      if (split) {
#pragma unroll
        for (int c = 0; c < KT; ++c) atomic_add(y + c, acc[c]);
      } else if (a.beta_mode == 0) {
#pragma unroll
        for (int c = 0; c < KT; ++c) y[c] = acc[c];
      } else if (a.beta_mode == 1) {
#pragma unroll
        for (int c = 0; c < KT; ++c) y[c] = acc[c] + y[c];
      } else {
        const V b = (V)a.beta;
#pragma unroll
        for (int c = 0; c < KT; ++c) y[c] = fma(b, y[c], acc[c]);
      }
    }
  }
}

// Shared memory of dtans_kernel: both tables, then (codebook gradient only)
// the value-slot bin map (kK uint16) and the CTA's bins (nbins values).
template <typename V>
constexpr int kernel_table_bytes() {
  return kK * 8 + kK * (int)sizeof(typename VEntry<V>::T);
}
template <typename V>
int kernel_smem_bytes(int mode, int nbins) {
  return kernel_table_bytes<V>() + (mode == kCodeGrad ? kK * 2 + ((nbins * (int)sizeof(V) + 15) & ~15) : 0);
}

template <typename V, int KT, int MODE>
__global__ void __launch_bounds__(512, (KT >= 8 ? 1 : 2)) dtans_kernel(Args a) {
  using VT = typename VEntry<V>::T;
  extern __shared__ __align__(16) uint8_t smem[];
  {
    const int nbytes = kernel_table_bytes<V>();
    const uint4 *src = (const uint4 *)a.tables;
    uint4 *dst = (uint4 *)smem;
    for (int i = threadIdx.x; i < nbytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  uint16_t *vrank = nullptr;
  V *bins = nullptr;
  if constexpr (MODE == kCodeGrad) {
    vrank = (uint16_t *)(smem + kernel_table_bytes<V>());
    bins = (V *)(smem + kernel_table_bytes<V>() + kK * 2);
    for (int i = threadIdx.x; i < kK; i += blockDim.x) vrank[i] = __ldg(a.vrank + i);
    for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) bins[i] = V(0);
  }
  __syncthreads();
  const uint2 *tD = (const uint2 *)smem;
  const VT *tV = (const VT *)(smem + kK * 8);
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t C = a.chain, nchains = (a.nslices + C - 1) / C;
  for (int64_t c = warp; c < nchains; c += nw) {
    ChainState cs{0, 0, 0, 0, 1};
    const int64_t s1 = min((c + 1) * C, a.nslices);
    for (int64_t s = c * C; s < s1; ++s) decode_slice<V, KT, MODE>(a, tD, tV, s, lane, bins, vrank, cs, s == c * C);
  }
  if constexpr (MODE == kCodeGrad) {
    __syncthreads();  // every warp's shared-memory adds are done
    for (int i = threadIdx.x; i < a.nbins; i += blockDim.x)
      if (bins[i] != V(0)) atomicAdd((V *)a.Y + i, bins[i]);
  }
}

template <typename V>
__global__ void scale_kernel(V *y, int64_t count, V beta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = beta == V(0) ? V(0) : y[i] * beta;
}

dtans_status cuda_fail2(cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return set_error(DTANS_ERR_CUDA, m);
}

template <typename V, int KT, int MODE>
dtans_status launch_one(dtans_handle_s &H, const Args &a, cudaStream_t st) {
  const int smem = kernel_smem_bytes<V>(MODE, a.nbins);
  auto kern = dtans_kernel<V, KT, MODE>;
  static std::atomic<uint64_t> configured{0};  // per template instance, one bit per device
  cudaError_t e;
  // the largest this instance can ask for (codebook gradient: kK + 1 bins)
  if ((e = ensure_smem_limit(kern, kernel_smem_bytes<V>(MODE, kK + 1), configured)) != cudaSuccess)
    return cuda_fail2(e, "cudaFuncSetAttribute");
  int block = H.block ? H.block : 512;
  int grid = H.grid;
  if (!grid) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, block, smem)) != cudaSuccess)
      return cuda_fail2(e, "occupancy");
    grid = std::max(1, sms * std::max(per, 1));
    const int64_t need = ((a.nslices + a.chain - 1) / a.chain * 32 + block - 1) / block;  // one warp per chain
    if (need < grid) grid = (int)std::max<int64_t>(1, need);
  }
  kern<<<grid, block, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail2(e, "kernel launch");
  return DTANS_OK;
}

template <typename V, int MODE>
dtans_status launch_tile(dtans_handle_s &H, Args a, int kt, cudaStream_t st) {
  const size_t vb = sizeof(V);
  auto aligned = [&](const void *p, size_t b) {
    return p && (uintptr_t)p % b == 0 && ((size_t)a.ld * vb) % b == 0 && ((size_t)a.c0 * vb) % b == 0;
  };
  // 1: rows start on 16-byte boundaries; 2: on 32-byte boundaries (rows of A
  // and B read with 32-byte loads)
  auto level = [&](const void *p) { return aligned(p, 16) ? (aligned(p, 32) ? 2 : 1) : 0; };
  a.vecA = level(a.A);
  a.vecB = level(a.B);
  a.vecY = aligned(a.Y, 16) ? 1 : 0;
  a.aggregate = H.scatter;
  switch (kt) {
    case 32:
      // per-entry dot products of 32 FP32 columns in one pass
      if constexpr (sizeof(V) == 4 && (MODE == kValsGrad || MODE == kCodeGrad))
        return launch_one<V, 32, MODE>(H, a, st);
      return set_error(DTANS_ERR_UNSUPPORTED, "column tile of 32 not instantiated");
    case 16: return launch_one<V, 16, MODE>(H, a, st);
    case 8: return launch_one<V, 8, MODE>(H, a, st);
    case 4: return launch_one<V, 4, MODE>(H, a, st);
    case 2: return launch_one<V, 2, MODE>(H, a, st);
    default: return launch_one<V, 1, MODE>(H, a, st);
  }
}

int next_tile(int remaining) {
  if (remaining >= 16) return 16;
  if (remaining >= 8) return 8;
  if (remaining >= 4) return 4;
  if (remaining >= 2) return 2;
  return 1;
}

// Column tiles of the per-entry dot products (value and codebook gradients):
// FP32 takes up to 32 columns in one pass.
template <typename V>
int next_dot_tile(int remaining) {
  if (sizeof(V) == 4 && remaining >= 32) return 32;
  return next_tile(remaining);
}

Args base_args(dtans_handle_s &H) {
  Args a{};
  a.words = H.d_words;
  a.slice_off = H.d_slice_off;
  a.tables = H.d_tables;
  a.unit_row = H.d_unit_row;
  a.unit_pos = H.d_unit_pos;
  a.nunits = H.nunits;
  a.nslices = H.nslices;
  a.ncols = H.n;
  a.first_rel = H.opts.first_delta;
  a.chain = std::max(1, H.opts.chain_slices);
  a.esc = H.d_esc_words;
  a.esc_off = H.d_esc_off;
  a.nnz = H.nnz;
  a.err = H.d_err;
  return a;
}

template <typename V>
dtans_status scale(V *y, int64_t count, double beta, cudaStream_t st) {
  if (count <= 0 || beta == 1.0) return DTANS_OK;
  cudaError_t e;
  if (beta == 0.0) {
    if ((e = cudaMemsetAsync(y, 0, count * sizeof(V), st)) != cudaSuccess) return cuda_fail2(e, "memset");
    return DTANS_OK;
  }
  int grid = (int)std::min<int64_t>(4096, (count + 255) / 256);
  scale_kernel<V><<<grid, 256, 0, st>>>(y, count, (V)beta);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail2(e, "scale launch");
  return DTANS_OK;
}

dtans_status check_handle(dtans_handle h) {
  if (!h) return set_error(DTANS_ERR_ARG, "null handle");
  if (!h->uploaded) return set_error(DTANS_ERR_STATE, "handle not uploaded (call dtans_upload)");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return set_error(DTANS_ERR_STATE, "handle was uploaded to another device");
  return DTANS_OK;
}

template <typename V>
dtans_status spmm_t(dtans_handle_s &H, int k, const void *X, void *Y, double beta, cudaStream_t st) {
  if (H.m == 0) return DTANS_OK;
  if (H.nnz == 0) return scale<V>((V *)Y, H.m * (int64_t)k, beta, st);  // y = beta y; x is never read
  Args a = base_args(H);
  a.ld = k;
  a.A = X;
  a.Y = Y;
  a.beta = beta;
  if (H.any_split) {
    dtans_status s = scale<V>((V *)Y, H.m * (int64_t)k, beta, st);
    if (s != DTANS_OK) return s;
    a.beta_mode = 1;
  } else {
    a.beta_mode = beta == 0.0 ? 0 : (beta == 1.0 ? 1 : 2);
  }
  for (int c0 = 0; c0 < k;) {
    // column tiles: the persistent ring kernel takes 32, 16 (FP32), 8, 4,
    // 2 (FP64) or 1 columns when the blocks are 16-byte aligned; other tiles
    // use the one-slice-per-warp kernel with up to 16 columns (see
    // tile_policy)
    int kt = 0;
    // tile policy 1: 16 columns or more left go to one 16-column pass of the
    // one-slice-per-warp kernel instead of two 8-column persistent passes
    if (H.use_persistent && !H.opts.escape_stream && !(H.tile_policy == 1 && k - c0 >= 16))
      for (int cand : {32, 16, 8, 4, 2, 1})
        if (cand <= k - c0 && persistent_tile_ok(H, cand, X, Y, k, c0)) {
          kt = cand;
          break;
        }
    dtans_status s;
    if (kt) {
      s = spmv_persistent(H, kt, X, Y, k, c0, beta, a.beta_mode, st);
    } else {
      kt = next_tile(k - c0);
      a.c0 = c0;
      s = launch_tile<V, kFwd>(H, a, kt, st);
    }
    if (s != DTANS_OK) return s;
    c0 += kt;
  }
  return DTANS_OK;
}

template <typename V>
dtans_status spmm_trans(dtans_handle_s &H, int k, const void *G, void *XG, double beta, cudaStream_t st) {
  dtans_status s = scale<V>((V *)XG, H.n * (int64_t)k, beta, st);
  if (s != DTANS_OK || H.m == 0) return s;
  Args a = base_args(H);
  a.ld = k;
  a.A = G;
  a.Y = XG;
  for (int c0 = 0; c0 < k;) {
    const int kt = next_tile(k - c0);
    a.c0 = c0;
    if ((s = launch_tile<V, kTrans>(H, a, kt, st)) != DTANS_OK) return s;
    c0 += kt;
  }
  return DTANS_OK;
}

template <typename V>
dtans_status vals_grad_t(dtans_handle_s &H, int k, const void *G, const void *X, void *out, cudaStream_t st) {
  if (H.nnz == 0) return DTANS_OK;
  Args a = base_args(H);
  a.ld = k;
  a.A = G;
  a.B = X;
  a.Y = out;
  for (int c0 = 0; c0 < k;) {
    // 32 FP32 columns with 16-byte aligned rows: the persistent ring kernel
    if constexpr (sizeof(V) == 4) {
      const size_t vb = sizeof(V);
      const bool al = (uintptr_t)G % 16 == 0 && (uintptr_t)X % 16 == 0 && ((size_t)k * vb) % 16 == 0 &&
                      ((size_t)c0 * vb) % 16 == 0;
      if (k - c0 >= 32 && al && H.use_persistent && !H.opts.escape_stream) {
        dtans_status s = vals_grad_persistent(H, G, X, out, k, c0, c0 > 0, st);
        if (s != DTANS_OK) return s;
        c0 += 32;
        continue;
      }
    }
    const int kt = next_dot_tile<V>(k - c0);
    a.c0 = c0;
    a.accumulate = c0 > 0;
    dtans_status s = launch_tile<V, kValsGrad>(H, a, kt, st);
    if (s != DTANS_OK) return s;
    c0 += kt;
  }
  return DTANS_OK;
}

// Bin of each stored value slot for the codebook gradient: the rank of the
// kept symbol that owns the slot, or the number of kept symbols for escape
// and unused slots.  Built and uploaded on first use.
dtans_status value_ranks(dtans_handle_s &H, const uint16_t **out) {
  if (!H.d_vrank) {
    const Table &t = H.tab[1];
    const uint16_t T = (uint16_t)t.kept_key.size();
    std::vector<uint16_t> r(kK, T);
    for (uint32_t q = 0; q < (uint32_t)t.kept_first.size(); ++q)
      for (uint32_t s = t.kept_first[q]; s < t.kept_first[q] + t.kept_mult[q]; ++s) r[t.stored(s)] = (uint16_t)q;
    cudaError_t e;
    if ((e = cudaMalloc(&H.d_vrank, kK * 2)) != cudaSuccess) return cuda_fail2(e, "cudaMalloc(value ranks)");
    if ((e = cudaMemcpy(H.d_vrank, r.data(), kK * 2, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail2(e, "cudaMemcpy(value ranks)");
  }
  *out = H.d_vrank;
  return DTANS_OK;
}

template <typename V>
dtans_status codebook_grad_t(dtans_handle_s &H, int k, const void *G, const void *X, void *out, cudaStream_t st) {
  Args a = base_args(H);
  a.nbins = (int32_t)H.tab[1].kept_key.size() + 1;
  cudaError_t e;
  if ((e = cudaMemsetAsync(out, 0, (size_t)a.nbins * sizeof(V), st)) != cudaSuccess)
    return cuda_fail2(e, "memset(codebook gradient)");
  if (H.nnz == 0) return DTANS_OK;
  dtans_status s = value_ranks(H, &a.vrank);
  if (s != DTANS_OK) return s;
  a.ld = k;
  a.A = G;
  a.B = X;
  a.Y = out;
  for (int c0 = 0; c0 < k;) {
    // 32 FP32 columns with 16-byte aligned rows: the persistent ring kernel
    if constexpr (sizeof(V) == 4) {
      const size_t vb = sizeof(V);
      const bool al = (uintptr_t)G % 16 == 0 && (uintptr_t)X % 16 == 0 && ((size_t)k * vb) % 16 == 0 &&
                      ((size_t)c0 * vb) % 16 == 0;
      if (k - c0 >= 32 && al && H.use_persistent && !H.opts.escape_stream) {
        if ((s = codebook_grad_persistent(H, G, X, out, k, c0, a.vrank, a.nbins, st)) != DTANS_OK) return s;
        c0 += 32;
        continue;
      }
    }
    const int kt = next_dot_tile<V>(k - c0);
    a.c0 = c0;
    if ((s = launch_tile<V, kCodeGrad>(H, a, kt, st)) != DTANS_OK) return s;
    c0 += kt;
  }
  return DTANS_OK;
}

template <typename V>
dtans_status decode_t(dtans_handle_s &H, uint32_t *cols, void *vals, cudaStream_t st) {
  if (H.nnz == 0) return DTANS_OK;
  Args a = base_args(H);
  a.ld = 1;
  a.Y = cols;
  a.Y2 = vals;
  return launch_one<V, 1, kDecode>(H, a, st);
}

}  // namespace
}  // namespace dtans

using namespace dtans;

extern "C" {

dtans_status dtans_spmm(dtans_handle h, int32_t k, const void *X, void *Y, double beta, void *stream) {
  dtans_status s = check_handle(h);
  if (s != DTANS_OK) return s;
  if (k < 1) return set_error(DTANS_ERR_ARG, "k must be >= 1");
  if ((h->m > 0 && !Y) || (h->nnz > 0 && !X)) return set_error(DTANS_ERR_ARG, "null vector");
  cudaStream_t st = (cudaStream_t)stream;
  return h->dtype == DTANS_F64 ? spmm_t<double>(*h, k, X, Y, beta, st) : spmm_t<float>(*h, k, X, Y, beta, st);
}

dtans_status dtans_spmv(dtans_handle h, const void *x, void *y, double beta, void *stream) {
  return dtans_spmm(h, 1, x, y, beta, stream);
}

dtans_status dtans_spmv_T(dtans_handle h, int32_t k, const void *G, void *XG, double beta, void *stream) {
  dtans_status s = check_handle(h);
  if (s != DTANS_OK) return s;
  if (k < 1) return set_error(DTANS_ERR_ARG, "k must be >= 1");
  if ((h->n > 0 && !XG) || (h->nnz > 0 && !G)) return set_error(DTANS_ERR_ARG, "null vector");
  cudaStream_t st = (cudaStream_t)stream;
  return h->dtype == DTANS_F64 ? spmm_trans<double>(*h, k, G, XG, beta, st)
                               : spmm_trans<float>(*h, k, G, XG, beta, st);
}

dtans_status dtans_vals_grad(dtans_handle h, int32_t k, const void *G, const void *X, void *out, void *stream) {
  dtans_status s = check_handle(h);
  if (s != DTANS_OK) return s;
  if (k < 1) return set_error(DTANS_ERR_ARG, "k must be >= 1");
  if (h->nnz > 0 && (!G || !X || !out)) return set_error(DTANS_ERR_ARG, "null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  return h->dtype == DTANS_F64 ? vals_grad_t<double>(*h, k, G, X, out, st)
                               : vals_grad_t<float>(*h, k, G, X, out, st);
}

dtans_status dtans_codebook_grad(dtans_handle h, int32_t k, const void *G, const void *X, void *out, void *stream) {
  dtans_status s = check_handle(h);
  if (s != DTANS_OK) return s;
  if (k < 1) return set_error(DTANS_ERR_ARG, "k must be >= 1");
  if (!out || (h->nnz > 0 && (!G || !X))) return set_error(DTANS_ERR_ARG, "null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  return h->dtype == DTANS_F64 ? codebook_grad_t<double>(*h, k, G, X, out, st)
                               : codebook_grad_t<float>(*h, k, G, X, out, st);
}

dtans_status dtans_decode_csr(dtans_handle h, uint32_t *col_idx_out, void *vals_out, void *stream) {
  dtans_status s = check_handle(h);
  if (s != DTANS_OK) return s;
  if (h->nnz > 0 && (!col_idx_out || !vals_out)) return set_error(DTANS_ERR_ARG, "null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  return h->dtype == DTANS_F64 ? decode_t<double>(*h, col_idx_out, vals_out, st)
                               : decode_t<float>(*h, col_idx_out, vals_out, st);
}

}  // extern "C"

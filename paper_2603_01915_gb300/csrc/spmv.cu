// Decode-fused single-vector SpMV of CSR-dtANS for GB300 (sm_103a).
//
// Persistent kernel, one CTA per SM (20 to 32 warps for one right-hand side,
// 16 for column tiles).  Each warp owns a contiguous
// range of slices whose interleaved words form one contiguous range of the
// stream; the warp streams that range into a private 4 KB shared-memory ring
// with 1-D bulk copies (cp.async.bulk, 512 B each, completion on one mbarrier
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
#include <mutex>
#include <vector>

#include "smem_limit.h"
#include "spmv_core.cuh"

namespace dtans {
namespace {

using namespace dev;

using namespace core;

template <typename V>
struct SpmvArgs {
  const uint32_t *words;
  const uint64_t *slice_off;
  const uint8_t *tables;
  const uint32_t *unit_row;    // null: unit u is row u
  const uint32_t *warp_slice;  // [nwarps + 1] first slice of each warp
  int64_t nunits;
  uint32_t ncols;
  int32_t first_rel;  // first delta of a unit relative to its row
  uint32_t chain;     // slices per chain (warp ranges start at chain starts)
  int32_t *err;
  const V *x;
  V *y;
  uint32_t ld, c0;    // dense blocks: leading dimension and first column of this pass
  V beta;
  int32_t beta_mode;  // 0: y = Ax, 1: y += Ax (y pre-scaled), 2: y = Ax + beta y
  const int4 *xfix;   // integer-coefficient products: x as fixed point (else null)
  const int32_t *xexp;  // ... the largest biased exponent of x (the fixed point's anchor)
  int32_t coef_exp;   // ... the common power of two of the value table's coefficients
  int32_t radixw;     // a check group can have radix W (both tables hold a symbol of multiplicity M)
  int32_t x32;        // rows of x (KT > 1) start on 32-byte boundaries at column c0
  const V *g;         // value gradient: G (rows of y's shape), the output is y (nnz values)
  const uint64_t *unit_pos;  // ... sorted-CSR position of each unit's first entry
  int32_t g32, acc_out;      // ... G rows 32-byte aligned; add to the output
  uint64_t nnz;              // ... entries of the matrix
  const uint16_t *vrank;     // codebook gradient: bin of each value-table slot
  int32_t nbins;             // ... bins (kept symbols + 1); the output is y (nbins values, added to)
};

// W warps per CTA, one CTA per SM; KT right-hand-side columns per pass; RW
// ring words per warp; kChain: the stream may chain units over slices; kInt:
// integer-coefficient products (FP64, KT = 1) from the fixed-point x; kGrad:
// instead of a product, the value gradient (1) or the codebook gradient (2)
// of 32 FP32 columns (DotCols32).
template <typename V, int KT, int W, uint32_t RW, bool kChain, bool kInt = false, int kGrad = 0>
__global__ void __launch_bounds__(W * 32, 1) spmv_kernel(SpmvArgs<V> a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  // a CTA whose warps have no slices stages nothing
  if (a.warp_slice[(int64_t)blockIdx.x * W] == a.warp_slice[(int64_t)(blockIdx.x + 1) * W]) return;
  uint32_t *ring_base = (uint32_t *)(smem + table_bytes<V>()) + wid * RW;
  uint64_t *bars = (uint64_t *)(smem + table_bytes<V>() + W * RW * 4) + wid * kNumChunks;
  const uint32_t tbar = smem_addr(smem + table_bytes<V>() + W * RW * 4 + W * kNumChunks * 8);
  if (lane == 0) {
    for (uint32_t c = 0; c < kNumChunks; ++c) mbar_init(smem_addr(bars + c), 1);
    if (wid == 0) mbar_init(tbar, table_chunks<V>());
    fence_mbar_init();
  }
  // codebook gradient: the CTA's bins follow the staging areas (zeroed here,
  // added to global memory once every warp is done)
  V *bins = nullptr;
  if constexpr (kGrad == 2) {
    bins = (V *)(smem + persistent_smem_bytes<V>(W, RW, kStageBytes));
    for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) bins[i] = V(0);
  }
  __syncthreads();
  // the tables arrive by bulk copy while the warps start their rings
  if (wid == 0) stage_tables_bulk<V>(smem, a.tables, tbar, lane);
  const int64_t gw = (int64_t)blockIdx.x * W + wid;
  uint32_t phase_bits = 0;
  Dense<V> Dn{a.x, a.y, a.ld, a.c0, nullptr, 0, 0, a.radixw, a.x32};
  if constexpr (KT == 32 && sizeof(V) == 4)  // the warp's staging area follows the barriers
    Dn.stage = (uint4 *)(smem + persistent_smem_bytes<V>(W, RW)) + wid * (kStageBytes / 16);
  if constexpr (kInt) {
    // x 2^F = the limbs with F = 1115 - E (see x_fixed_kernel); a unit's
    // integer sum times 2^(coef_exp - F) is its product
    Dn.xfix = a.xfix;
    Dn.scale = a.coef_exp - (1115 - max(__ldg(a.xexp), 1));
    Dn.coef_exp = a.coef_exp;
  }
  if constexpr (kGrad != 0) {
    Dn.g = a.g;
    Dn.unit_pos = a.unit_pos;
    Dn.g32 = a.g32;
    Dn.acc_out = a.acc_out;
    Dn.nnz = a.nnz;
    Dn.err = a.err;
    Dn.vrank = a.vrank;
    Dn.bins = bins;
  }
  int32_t fail = warp_spmv_range<V, KT, RW, kChain, kInt, kGrad>(a.words, a.slice_off, a.unit_row, a.nunits, a.ncols,
                                                    a.first_rel != 0, a.chain, a.warp_slice[gw], a.warp_slice[gw + 1],
                                                    smem, smem + kK * 8, ring_base, bars, Dn, a.beta, a.beta_mode,
                                                    a.err, phase_bits, lane, tbar);
  // warp 0 keeps the CTA alive until the table copy has landed (it may have
  // had no slices of its own)
  if (wid == 0 && !mbar_wait_warp(tbar, 0, kSpinLimit) && !fail) fail = kErrTimeout;
  if (fail && lane == 0) atomicExch(a.err, fail);
  if constexpr (kGrad == 2) {
    __syncthreads();  // every warp's shared-memory adds are done
    for (int i = threadIdx.x; i < a.nbins; i += blockDim.x)
      if (bins[i] != V(0)) atomicAdd(a.y + i, bins[i]);
  }
}

// ---------------------------------------------------------------------------
// Integer-coefficient products (FP64 value tables whose kept values are all
// c * 2^e with small integers c, such as the 27-point stencil's 26 and -1).
// GB300 issues two FP64 FMAs per clock per SM, so one FMA per stored entry
// bounds an FP64 SpMV near 0.6 G entries/ms; here x is first turned into exact
// fixed point and each entry costs three 32 x 32 -> 64-bit integer
// multiply-adds instead (IntCols), which run on the integer pipes.  The sums
// are exact, and each unit's result is rounded to FP64 once, so the row
// bound of the FMA chain holds with room to spare.
//
// Fixed point: E = the largest biased exponent of the finite x (at least 1),
// F = 1115 - E, so |x| 2^F < 2^(E - 1022 + F) = 2^93.  x = m 2^(e - 1075)
// (e the biased exponent, at least 1; m < 2^53) gives x 2^F = m 2^s with
// s = e - E + 40, an integer when s >= 0, i.e. for every x within a factor
// 2^40 of the largest.  It is stored as three balanced signed 32-bit limbs
// S0 + S1 2^32 + S2 2^64 (|S0|, |S1| <= 2^31, |S2| <= 2^29 + 1) and a flag
// word 0; x outside the window, infinities and NaNs are stored as their raw
// bits (low word, high word), 0 and the flag 1, and their entries take the
// FMA chain.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t finite_exponent(double v) {
  const uint32_t be = (uint32_t)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ffu;
  return be == 0x7ffu ? 0u : be;
}

// Largest finite biased exponent of x: each CTA reduces its share (16-byte
// loads of pairs), then one atomicMax per CTA.
__global__ void x_exponent_kernel(const double *__restrict__ x, int64_t n, int32_t *emax) {
  __shared__ uint32_t warp_max[32];
  uint32_t e = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n2 = ((uintptr_t)x % 16 == 0) ? n / 2 : 0;  // pairs read as one 16-byte load
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += stride) {
    const double2 v = __ldg((const double2 *)x + i);
    e = max(e, max(finite_exponent(v.x), finite_exponent(v.y)));
  }
  for (int64_t i = 2 * n2 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
    e = max(e, finite_exponent(__ldg(x + i)));
  e = __reduce_max_sync(kFull, e);
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) warp_max[wid] = e;
  __syncthreads();
  if (wid == 0) {
    e = lane < nw ? warp_max[lane] : 0u;
    e = __reduce_max_sync(kFull, e);
    if (lane == 0 && e) atomicMax(emax, (int32_t)e);
  }
}

// One x as fixed-point limbs and flag (see above).
__device__ __forceinline__ int4 fixed_limbs(double v, int32_t E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int32_t be = (int32_t)(b >> 52) & 0x7ff;
  int4 q = make_int4(0, 0, 0, 0);
  const unsigned long long m = (b & ((1ull << 52) - 1)) | (be ? 1ull << 52 : 0ull);
  const int32_t sh = max(be, 1) - E + 40;  // x 2^F = m 2^sh, sh <= 40
  if (be == 0x7ff || (m != 0 && sh < 0)) {
    // infinity, NaN or below the window: the raw bits, for the FMA path
    q = make_int4((int32_t)(uint32_t)b, (int32_t)(uint32_t)(b >> 32), 0, 1);
  } else if (m != 0) {
    __int128 X = (__int128)m << sh;  // m < 2^53, sh <= 40: below 2^93
    if (b >> 63) X = -X;
    q.x = (int32_t)(uint32_t)(unsigned long long)X;  // low 32 bits as a signed limb
    X = (X - q.x) >> 32;                            // exact: X - S0 is a multiple of 2^32
    q.y = (int32_t)(uint32_t)(unsigned long long)X;
    X = (X - q.y) >> 32;
    q.z = (int32_t)X;
  }
  return q;
}

// x as fixed point, one entry per thread and step (a warp's stores are 512
// contiguous bytes).
__global__ void x_fixed_kernel(const double *__restrict__ x, int64_t n, const int32_t *__restrict__ emax,
                               int4 *__restrict__ xf) {
  const int32_t E = max(__ldg(emax), 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    xf[i] = fixed_limbs(__ldg(x + i), E);
}

// Warps per CTA of the single-vector kernel: the handle's choice, else 24.
// On GB300 24 warps (80 registers, no spill; FP64: 96 KB tables + 96 KB rings
// leave 60 KB of L1) measured best on random-column and power-law matrices,
// 28 on the 27-point stencil; dtans_tune_warps picks per matrix.
int single_vector_warps(const dtans_handle_s &H) { return H.warps ? H.warps : 24; }

dtans_status fail_cuda(cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return set_error(DTANS_ERR_CUDA, m);
}

// Splits the slices into `nwarps` contiguous ranges of about equal word
// count, each starting at a chain's first slice.
std::vector<uint32_t> warp_ranges(const dtans_handle_s &H, int64_t nwarps) {
  std::vector<uint32_t> r(nwarps + 1);
  const uint64_t total = H.slice_off.empty() ? 0 : H.slice_off.back();
  const int64_t C = std::max(1, H.opts.chain_slices);
  int64_t s = 0;
  for (int64_t w = 0; w <= nwarps; ++w) {
    const uint64_t target = (uint64_t)((__int128)total * w / nwarps);
    while (s < H.nslices && (H.slice_off[s] < target || s % C)) ++s;
    r[w] = (uint32_t)s;
  }
  r[nwarps] = (uint32_t)H.nslices;
  return r;
}

// Per-warp slice ranges for `nwarps` warps, cached on the device (one entry
// per warps-per-CTA shape).
dtans_status ranges_for(dtans_handle_s &H, int64_t nwarps, int slot, const uint32_t **out) {
  cudaError_t e;
  if (H.d_warp_slice[slot] == nullptr || H.warp_slice_n[slot] != nwarps) {
    std::vector<uint32_t> r = warp_ranges(H, nwarps);
    cudaFree(H.d_warp_slice[slot]);
    H.d_warp_slice[slot] = nullptr;
    if ((e = cudaMalloc(&H.d_warp_slice[slot], r.size() * 4)) != cudaSuccess) return fail_cuda(e, "cudaMalloc(ranges)");
    if ((e = cudaMemcpy(H.d_warp_slice[slot], r.data(), r.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail_cuda(e, "cudaMemcpy(ranges)");
    H.warp_slice_n[slot] = nwarps;
  }
  *out = H.d_warp_slice[slot];
  return DTANS_OK;
}

// The fixed-point copy of x for the integer-coefficient kernels: scratch on
// first use (16 bytes per column, and the exponent word), then two small
// kernels on the product's stream.
dtans_status prepare_fixed_x(dtans_handle_s &H, const double *x, int sms, cudaStream_t st) {
  cudaError_t e;
  if (!H.d_xexp && (e = cudaMalloc(&H.d_xexp, sizeof(int32_t))) != cudaSuccess)
    return fail_cuda(e, "cudaMalloc(exponent word)");
  if (!H.d_xfix || H.xfix_n < H.n) {
    cudaFree(H.d_xfix);
    H.d_xfix = nullptr;
    H.xfix_n = 0;
    if ((e = cudaMalloc(&H.d_xfix, (size_t)H.n * sizeof(int4))) != cudaSuccess)
      return fail_cuda(e, "cudaMalloc(fixed-point x)");
    H.xfix_n = H.n;
  }
  if ((e = cudaMemsetAsync(H.d_xexp, 0, sizeof(int32_t), st)) != cudaSuccess) return fail_cuda(e, "memset");
  // one pass each over x
  const int grid_e = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 4, (H.n + 1023) / 1024));
  const int grid_f = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8, (H.n + 255) / 256));
  x_exponent_kernel<<<grid_e, 512, 0, st>>>(x, H.n, H.d_xexp);
  x_fixed_kernel<<<grid_f, 256, 0, st>>>(x, H.n, H.d_xexp, (int4 *)H.d_xfix);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "fixed-point x launch");
  return DTANS_OK;
}

template <typename V, int KT, int W, uint32_t RW, bool kChain, bool kInt = false, int kGrad = 0>
dtans_status launch_shape(dtans_handle_s &H, const void *x, void *y, uint32_t ld, uint32_t c0, double beta,
                          int32_t beta_mode, cudaStream_t st, const void *g = nullptr, int32_t acc_out = 0,
                          const uint16_t *vrank = nullptr, int32_t nbins = 0) {
  cudaError_t e;
  static std::atomic<uint64_t> configured{0};  // per kernel instance, one bit per device
  const int base = persistent_smem_bytes<V>(W, RW, (KT == 32 && sizeof(V) == 4) ? kStageBytes : 0);
  auto bin_bytes = [](int nb) { return (nb * (int)sizeof(V) + 15) & ~15; };
  const int smem = base + (kGrad == 2 ? bin_bytes(nbins) : 0);
  auto kern = spmv_kernel<V, KT, W, RW, kChain, kInt, kGrad>;
  // the largest this instance can ask for (codebook gradient: kK + 1 bins)
  if ((e = ensure_smem_limit(kern, base + (kGrad == 2 ? bin_bytes(kK + 1) : 0), configured)) != cudaSuccess)
    return fail_cuda(e, "cudaFuncSetAttribute(spmv)");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = H.grid ? H.grid : sms;
  const uint32_t *ranges = nullptr;
  dtans_status s = ranges_for(H, (int64_t)grid * W, KT == 1 ? 0 : 1, &ranges);
  if (s != DTANS_OK) return s;
  if constexpr (kInt) {
    if ((s = prepare_fixed_x(H, (const double *)x, sms, st)) != DTANS_OK) return s;
  }
  SpmvArgs<V> a{};
  a.words = H.d_words;
  a.slice_off = H.d_slice_off;
  a.tables = H.d_tables;
  a.unit_row = H.d_unit_row;
  a.warp_slice = ranges;
  a.nunits = H.nunits;
  a.ncols = (uint32_t)std::max<int64_t>(H.n, 1);
  a.first_rel = H.opts.first_delta;
  a.chain = (uint32_t)std::max(1, H.opts.chain_slices);
  a.err = H.d_err;
  a.x = (const V *)x;
  a.y = (V *)y;
  a.ld = ld;
  a.c0 = c0;
  a.beta = (V)beta;
  a.beta_mode = beta_mode;
  a.radixw = H.radix_w ? 1 : 0;
  a.x32 = KT > 1 && (uintptr_t)x % 32 == 0 && ((size_t)ld * sizeof(V)) % 32 == 0 && ((size_t)c0 * sizeof(V)) % 32 == 0;
  if constexpr (kInt) {
    a.xfix = (const int4 *)H.d_xfix;
    a.xexp = H.d_xexp;
    a.coef_exp = H.int_exp;
  }
  if constexpr (kGrad != 0) {
    a.g = (const V *)g;
    a.vrank = vrank;
    a.nbins = nbins;
    a.unit_pos = H.d_unit_pos;
    a.g32 = (uintptr_t)g % 32 == 0 && ((size_t)ld * sizeof(V)) % 32 == 0 && ((size_t)c0 * sizeof(V)) % 32 == 0;
    a.acc_out = acc_out;
    a.nnz = (uint64_t)H.nnz;
  }
  kern<<<grid, W * 32, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "spmv launch");
  return DTANS_OK;
}

// Single-vector kernels come in a one-slice-chain build (the paper's format,
// fewer live registers) and a chained one; column tiles always take the
// chained build.
template <typename V, int KT, int W, uint32_t RW>
dtans_status launch(dtans_handle_s &H, const void *x, void *y, uint32_t ld, uint32_t c0, double beta,
                    int32_t beta_mode, cudaStream_t st) {
  if constexpr (sizeof(V) == 8 && KT == 1) {
    if (int_products(H)) {
      if (H.opts.chain_slices <= 1) return launch_shape<V, KT, W, RW, false, true>(H, x, y, ld, c0, beta, beta_mode, st);
      return launch_shape<V, KT, W, RW, true, true>(H, x, y, ld, c0, beta, beta_mode, st);
    }
  }
  if (KT == 1 && H.opts.chain_slices <= 1)
    return launch_shape<V, KT, W, RW, false>(H, x, y, ld, c0, beta, beta_mode, st);
  return launch_shape<V, KT, W, RW, true>(H, x, y, ld, c0, beta, beta_mode, st);
}

template <typename V>
dtans_status launch_kt(dtans_handle_s &H, int kt, const void *x, void *y, uint32_t ld, uint32_t c0, double beta,
                       int32_t beta_mode, cudaStream_t st) {
  switch (kt) {
    case 1:
      switch (single_vector_warps(H)) {
        case 20: return launch<V, 1, 20, kRingWords>(H, x, y, ld, c0, beta, beta_mode, st);
        case 28: return launch<V, 1, 28, kRingWords>(H, x, y, ld, c0, beta, beta_mode, st);
        case 32: return launch<V, 1, 32, kRingWords>(H, x, y, ld, c0, beta, beta_mode, st);
        default: return launch<V, 1, 24, kRingWords>(H, x, y, ld, c0, beta, beta_mode, st);
      }
    case 2:
      if constexpr (sizeof(V) == 8) return launch<V, 2, 16, kRingWords>(H, x, y, ld, c0, beta, beta_mode, st);
      break;
    case 4: return launch<V, 4, 16, kRingWords>(H, x, y, ld, c0, beta, beta_mode, st);
    case 8: return launch<V, 8, 16, kRingWords>(H, x, y, ld, c0, beta, beta_mode, st);
    case 16:  // FP32 only: one decode feeds 16 or 32 columns of 64- or 128-byte X rows
      if constexpr (sizeof(V) == 4) return launch<V, 16, 16, kRingWords>(H, x, y, ld, c0, beta, beta_mode, st);
      break;
    case 32:
      if constexpr (sizeof(V) == 4) return launch<V, 32, 16, kRingWords>(H, x, y, ld, c0, beta, beta_mode, st);
      break;
    default: break;
  }
  return set_error(DTANS_ERR_UNSUPPORTED, "column tile not supported by the persistent kernel");
}


}  // namespace

// Whether a single-vector product of the handle uses the integer-coefficient
// kernels: asked for (dtans_set_accumulate mode 1), an FP64 table with
// integer coefficients, units short enough for the 64-bit accumulators (2^16
// entries), and a stream the persistent kernel decodes (no separate escape
// stream).
bool int_products(const dtans_handle_s &H) {
  return H.dtype == DTANS_F64 && H.int_ok && H.accumulate == 1 && H.max_unit_len <= (1 << 16) && H.n > 0 &&
         H.use_persistent && !H.opts.escape_stream;
}

bool persistent_tile_ok(const dtans_handle_s &H, int kt, const void *x, const void *y, int64_t ld, int64_t c0) {
  const int vb = H.dtype == DTANS_F64 ? 8 : 4;
  if (kt == 1) return ld == 1 && c0 == 0;  // the single-column kernel gathers x[col] directly
  if (kt != 2 && kt != 4 && kt != 8 && !(vb == 4 && (kt == 16 || kt == 32))) return false;
  if (kt * vb < 16 || (kt * vb) % 16) return false;
  return ((uintptr_t)x % 16 == 0) && ((uintptr_t)y % 16 == 0) && (ld * vb) % 16 == 0 && (c0 * vb) % 16 == 0;
}

// The value gradient of columns c0 .. c0 + 31 of FP32 G and X (row-major,
// leading dimension ld, rows 16-byte aligned at c0) into out (nnz values,
// sorted-CSR order; added to when acc_out) with the persistent kernel.
dtans_status vals_grad_persistent(dtans_handle_s &H, const void *G, const void *X, void *out, int64_t ld, int64_t c0,
                                  bool acc_out, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (H.dtype != DTANS_F32) return set_error(DTANS_ERR_UNSUPPORTED, "persistent value gradient: FP32 only");
  if (H.opts.chain_slices <= 1)
    return launch_shape<float, 32, 16, kRingWords, false, false, 1>(H, X, out, (uint32_t)ld, (uint32_t)c0, 0.0, 0,
                                                                   st, G, acc_out ? 1 : 0);
  return launch_shape<float, 32, 16, kRingWords, true, false, 1>(H, X, out, (uint32_t)ld, (uint32_t)c0, 0.0, 0, st,
                                                                G, acc_out ? 1 : 0);
}

// The codebook gradient of columns c0 .. c0 + 31 (FP32, as above), added to
// out[bin] for the bin (vrank: rank of the kept symbol owning each value
// slot, nbins - 1 for escape and unused slots) of every entry's value.
dtans_status codebook_grad_persistent(dtans_handle_s &H, const void *G, const void *X, void *out, int64_t ld,
                                      int64_t c0, const uint16_t *vrank, int32_t nbins, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (H.dtype != DTANS_F32) return set_error(DTANS_ERR_UNSUPPORTED, "persistent codebook gradient: FP32 only");
  if (nbins < 1 || nbins > kK + 1) return set_error(DTANS_ERR_ARG, "codebook gradient: bin count");
  if (H.opts.chain_slices <= 1)
    return launch_shape<float, 32, 16, kRingWords, false, false, 2>(H, X, out, (uint32_t)ld, (uint32_t)c0, 0.0, 0,
                                                                   st, G, 0, vrank, nbins);
  return launch_shape<float, 32, 16, kRingWords, true, false, 2>(H, X, out, (uint32_t)ld, (uint32_t)c0, 0.0, 0, st,
                                                                G, 0, vrank, nbins);
}

dtans_status spmv_persistent(dtans_handle_s &H, int kt, const void *x, void *y, int64_t ld, int64_t c0, double beta,
                             int32_t beta_mode, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  return H.dtype == DTANS_F64 ? launch_kt<double>(H, kt, x, y, (uint32_t)ld, (uint32_t)c0, beta, beta_mode, st)
                              : launch_kt<float>(H, kt, x, y, (uint32_t)ld, (uint32_t)c0, beta, beta_mode, st);
}

}  // namespace dtans

// ---------------------------------------------------------------------------
// dtans_spmv_noalloc: the persistent SpMV for callers that cannot allocate
// device memory.  dtans_spmv allocates (once per launch shape) the per-warp
// slice ranges its kernel reads; this variant keeps them in a fixed
// file-scope device array instead and fills it on the device at every call,
// so the call itself allocates nothing and copies nothing from the host.
// ---------------------------------------------------------------------------
namespace dtans {
namespace {

constexpr int kNoallocMaxWarps = 8192;  // e.g. 256 CTAs of 32 warps; 32 KB of device memory

// Per-warp slice ranges of the no-allocation SpMV (shared by every call on a
// device; holds the last call's ranges).
static __device__ __align__(256) uint32_t g_noalloc_ranges[kNoallocMaxWarps + 1];

// Host-side device address of g_noalloc_ranges per device.  In host code the
// array's name is only a stand-in for the symbol, not a device address.
std::mutex g_noalloc_mu;
uint32_t *g_noalloc_addr[64] = {};

dtans_status noalloc_scratch(int dev, uint32_t **out) {
  if (dev < 0 || dev >= 64) return set_error(DTANS_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ranges);  // the current device is `dev`
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_addr[dev] = (uint32_t *)p;
  }
  *out = g_noalloc_addr[dev];
  return DTANS_OK;
}

// ranges[w] = first slice whose word offset is >= total * w / nwarps, moved
// up to the next chain start.
__global__ void noalloc_ranges_kernel(const uint64_t *__restrict__ slice_off, int64_t nslices, int64_t nwarps,
                                      int64_t chain, uint32_t *ranges) {
  const int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (w > nwarps) return;
  if (w == nwarps) {
    ranges[w] = (uint32_t)nslices;
    return;
  }
  const uint64_t total = slice_off[nslices];
  const uint64_t target = (uint64_t)(((unsigned __int128)total * (uint64_t)w) / (uint64_t)nwarps);
  int64_t lo = 0, hi = nslices;  // first s in [0, nslices] with slice_off[s] >= target
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (slice_off[mid] < target)
      lo = mid + 1;
    else
      hi = mid;
  }
  lo = (lo + chain - 1) / chain * chain;  // ranges start at a chain's first slice
  ranges[w] = (uint32_t)(lo < nslices ? lo : nslices);
}

template <typename V>
__global__ void noalloc_scale_kernel(V *y, int64_t count, V beta) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = beta == V(0) ? V(0) : y[i] * beta;
}

template <typename V>
dtans_status noalloc_spmv(dtans_handle_s &H, const void *x, void *y, double beta, cudaStream_t st) {
  cudaError_t e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = H.grid ? H.grid : sms;
  const int W = single_vector_warps(H);
  const int64_t nwarps = (int64_t)grid * W;
  if (nwarps > kNoallocMaxWarps)
    return set_error(DTANS_ERR_ARG, "launch shape exceeds the no-alloc scratch (at most 8192 warps)");
  if (H.m == 0) return DTANS_OK;
  int32_t mode = beta == 0.0 ? 0 : (beta == 1.0 ? 1 : 2);
  if (H.nnz == 0 || H.any_split) {
    if (beta != 1.0) {
      noalloc_scale_kernel<V><<<std::max(1, std::min(sms * 4, (int)((H.m + 255) / 256))), 256, 0, st>>>(
          (V *)y, H.m, (V)beta);
      if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "no-alloc scale launch");
    }
    if (H.nnz == 0) return DTANS_OK;
    mode = 1;
  }
  uint32_t *ranges = nullptr;
  dtans_status s = noalloc_scratch(dev, &ranges);
  if (s != DTANS_OK) return s;
  noalloc_ranges_kernel<<<(int)((nwarps + 1 + 255) / 256), 256, 0, st>>>(
      H.d_slice_off, H.nslices, nwarps, (int64_t)std::max(1, H.opts.chain_slices), ranges);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "no-alloc ranges launch");
  static std::atomic<uint64_t> configured[8];  // per kernel instance, one bit per device
  const bool chained = H.opts.chain_slices > 1;
  const int slot = (W == 20 ? 0 : W == 28 ? 2 : W == 32 ? 3 : 1) + (chained ? 4 : 0);
  const int smem = persistent_smem_bytes<V>(W, kRingWords);
  auto kern = chained ? (W == 20   ? spmv_kernel<V, 1, 20, kRingWords, true>
                         : W == 28 ? spmv_kernel<V, 1, 28, kRingWords, true>
                         : W == 32 ? spmv_kernel<V, 1, 32, kRingWords, true>
                                   : spmv_kernel<V, 1, 24, kRingWords, true>)
                      : (W == 20   ? spmv_kernel<V, 1, 20, kRingWords, false>
                         : W == 28 ? spmv_kernel<V, 1, 28, kRingWords, false>
                         : W == 32 ? spmv_kernel<V, 1, 32, kRingWords, false>
                                   : spmv_kernel<V, 1, 24, kRingWords, false>);
  if ((e = ensure_smem_limit(kern, smem, configured[slot])) != cudaSuccess)
    return fail_cuda(e, "cudaFuncSetAttribute(no-alloc spmv)");
  SpmvArgs<V> a{};
  a.words = H.d_words;
  a.slice_off = H.d_slice_off;
  a.tables = H.d_tables;
  a.unit_row = H.d_unit_row;
  a.warp_slice = ranges;
  a.nunits = H.nunits;
  a.ncols = (uint32_t)std::max<int64_t>(H.n, 1);
  a.first_rel = H.opts.first_delta;
  a.chain = (uint32_t)std::max(1, H.opts.chain_slices);
  a.err = H.d_err;
  a.x = (const V *)x;
  a.y = (V *)y;
  a.ld = 1;
  a.c0 = 0;
  a.beta = (V)beta;
  a.beta_mode = mode;
  a.radixw = H.radix_w ? 1 : 0;
  kern<<<grid, W * 32, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "no-alloc spmv launch");
  return DTANS_OK;
}

}  // namespace
}  // namespace dtans

extern "C" dtans_status dtans_spmv_noalloc(dtans_handle h, const void *x, void *y, double beta, void *stream) {
  using namespace dtans;
  if (!h) return set_error(DTANS_ERR_ARG, "null handle");
  if (!h->uploaded) return set_error(DTANS_ERR_STATE, "handle not uploaded (call dtans_upload)");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return set_error(DTANS_ERR_STATE, "handle was uploaded to another device");
  if ((h->m > 0 && !y) || (h->nnz > 0 && !x)) return set_error(DTANS_ERR_ARG, "null vector");
  if (h->opts.escape_stream)
    return set_error(DTANS_ERR_UNSUPPORTED, "no-allocation SpMV of a handle with a separate escape stream");
  cudaStream_t st = (cudaStream_t)stream;
  return h->dtype == DTANS_F64 ? noalloc_spmv<double>(*h, x, y, beta, st) : noalloc_spmv<float>(*h, x, y, beta, st);
}

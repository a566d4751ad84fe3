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
  int32_t *err;
  const V *x;
  V *y;
  uint32_t ld, c0;    // dense blocks: leading dimension and first column of this pass
  V beta;
  int32_t beta_mode;  // 0: y = Ax, 1: y += Ax (y pre-scaled), 2: y = Ax + beta y
};

// W warps per CTA, one CTA per SM; KT right-hand-side columns per pass.
template <typename V, int KT, int W>
__global__ void __launch_bounds__(W * 32, 1) spmv_kernel(SpmvArgs<V> a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  stage_tables<V>(smem, a.tables);
  uint32_t *ring_base = (uint32_t *)(smem + table_bytes<V>()) + wid * kRing;
  uint64_t *bars = (uint64_t *)(smem + table_bytes<V>() + W * kRing * 4) + wid * kNumChunks;
  if (lane == 0) {
    for (uint32_t c = 0; c < kNumChunks; ++c) mbar_init(smem_addr(bars + c), 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int64_t gw = (int64_t)blockIdx.x * W + wid;
  uint32_t phase_bits = 0;
  const Dense<V> Dn{a.x, a.y, a.ld, a.c0};
  const int32_t fail = warp_spmv_range<V, KT>(a.words, a.slice_off, a.unit_row, a.nunits, a.ncols,
                                              a.warp_slice[gw], a.warp_slice[gw + 1], smem, smem + kK * 8,
                                              ring_base, bars, Dn, a.beta, a.beta_mode, a.err, phase_bits, lane);
  if (fail && lane == 0) atomicExch(a.err, fail);
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

template <typename V, int KT, int W>
dtans_status launch(dtans_handle_s &H, const void *x, void *y, uint32_t ld, uint32_t c0, double beta,
                    int32_t beta_mode, cudaStream_t st) {
  cudaError_t e;
  static thread_local int configured = 0;
  const int smem = persistent_smem_bytes<V>(W);
  auto kern = spmv_kernel<V, KT, W>;
  if (!configured) {
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
      return fail_cuda(e, "cudaFuncSetAttribute(spmv)");
    configured = 1;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = H.grid ? H.grid : sms;
  const uint32_t *ranges = nullptr;
  dtans_status s = ranges_for(H, (int64_t)grid * W, W == 32 ? 0 : 1, &ranges);
  if (s != DTANS_OK) return s;
  SpmvArgs<V> a{};
  a.words = H.d_words;
  a.slice_off = H.d_slice_off;
  a.tables = H.d_tables;
  a.unit_row = H.d_unit_row;
  a.warp_slice = ranges;
  a.nunits = H.nunits;
  a.ncols = (uint32_t)std::max<int64_t>(H.n, 1);
  a.err = H.d_err;
  a.x = (const V *)x;
  a.y = (V *)y;
  a.ld = ld;
  a.c0 = c0;
  a.beta = (V)beta;
  a.beta_mode = beta_mode;
  kern<<<grid, W * 32, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail_cuda(e, "spmv launch");
  return DTANS_OK;
}

template <typename V>
dtans_status launch_kt(dtans_handle_s &H, int kt, const void *x, void *y, uint32_t ld, uint32_t c0, double beta,
                       int32_t beta_mode, cudaStream_t st) {
  switch (kt) {
    case 1: return launch<V, 1, 32>(H, x, y, ld, c0, beta, beta_mode, st);
    case 2:
      if constexpr (sizeof(V) == 8) return launch<V, 2, 16>(H, x, y, ld, c0, beta, beta_mode, st);
      break;
    case 4: return launch<V, 4, 16>(H, x, y, ld, c0, beta, beta_mode, st);
    case 8: return launch<V, 8, 16>(H, x, y, ld, c0, beta, beta_mode, st);
    default: break;
  }
  return set_error(DTANS_ERR_UNSUPPORTED, "column tile not supported by the persistent kernel");
}

}  // namespace

bool persistent_tile_ok(const dtans_handle_s &H, int kt, const void *x, const void *y, int64_t ld, int64_t c0) {
  const int vb = H.dtype == DTANS_F64 ? 8 : 4;
  if (kt == 1) return ld == 1 && c0 == 0;  // the single-column kernel gathers x[col] directly
  if (kt != 2 && kt != 4 && kt != 8) return false;
  if (kt * vb < 16 || (kt * vb) % 16) return false;
  return ((uintptr_t)x % 16 == 0) && ((uintptr_t)y % 16 == 0) && (ld * vb) % 16 == 0 && (c0 * vb) % 16 == 0;
}

dtans_status spmv_persistent(dtans_handle_s &H, int kt, const void *x, void *y, int64_t ld, int64_t c0, double beta,
                             int32_t beta_mode, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  return H.dtype == DTANS_F64 ? launch_kt<double>(H, kt, x, y, (uint32_t)ld, (uint32_t)c0, beta, beta_mode, st)
                              : launch_kt<float>(H, kt, x, y, (uint32_t)ld, (uint32_t)c0, beta, beta_mode, st);
}

}  // namespace dtans

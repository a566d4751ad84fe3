// Batched decode-fused SpMV: many CSR-dtANS matrices of uneven size in one
// persistent launch.
//
// The slices of all members, concatenated in member order, are cut into one
// contiguous piece per CTA with about equal word counts (host side, at batch
// creation).  A CTA walks its pieces in order; when the member changes it
// re-stages that member's coding tables into shared memory, and inside a piece
// its 24 warps split the slices by word count and decode them with the same
// per-warp ring decoder as the single-matrix kernel.  All device pointers of
// the members (streams, tables, x, y) live in a device table, so one launch
// needs no host-device copy and can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <memory>
#include <vector>

#include "smem_limit.h"
#include "spmv_core.cuh"

namespace dtans {
namespace {

using namespace dev;
using namespace core;

// 24 warps per CTA: 80 registers per thread and a 60 KB L1 beside the FP64
// tables and rings (measured faster than 32 on random-column FP64 matrices).
constexpr int kWarpsPerCta = 24;
constexpr int kThreads = kWarpsPerCta * 32;

struct MemberDev {
  const uint32_t *words;
  const uint64_t *slice_off;
  const uint8_t *tables;
  const uint32_t *unit_row;
  const void *x;
  void *y;
  int64_t nunits;
  int64_t m;
  uint32_t ncols;
  int32_t split;      // the layout splits rows: y was pre-scaled, add
  int32_t first_rel;  // first delta of a unit relative to its row
  uint32_t chain;     // slices per chain
  int32_t radixw;     // a check group can have radix W
};

struct PieceDev {
  uint32_t member;
  uint32_t bounds;  // index of its kWarpsPerCta + 1 warp boundaries
};

template <typename V>
struct BatchArgs {
  const MemberDev *members;
  const PieceDev *pieces;
  const uint32_t *piece_start;  // [grid + 1]
  const uint32_t *warp_bounds;
  int32_t *err;
  V beta;
  int32_t beta_mode;  // for members whose rows are not split
};

template <typename V, uint32_t RW>
__global__ void __launch_bounds__(kThreads, 1) batch_spmv_kernel(BatchArgs<V> a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  uint32_t *ring_base = (uint32_t *)(smem + table_bytes<V>()) + wid * RW;
  uint64_t *bars = (uint64_t *)(smem + table_bytes<V>() + kWarpsPerCta * RW * 4) + wid * kNumChunks;
  if (lane == 0) {
    for (uint32_t c = 0; c < kNumChunks; ++c) mbar_init(smem_addr(bars + c), 1);
    fence_mbar_init();
  }
  uint32_t phase_bits = 0;
  int32_t fail = 0;
  uint32_t staged = 0xffffffffu;
  const uint32_t p0 = a.piece_start[blockIdx.x], p1 = a.piece_start[blockIdx.x + 1];
  for (uint32_t p = p0; p < p1; ++p) {
    const PieceDev pc = a.pieces[p];
    const MemberDev mb = a.members[pc.member];
    if (pc.member != staged) {
      __syncthreads();  // every warp is done with the previous member's tables
      stage_tables<V>(smem, mb.tables);
      __syncthreads();
      staged = pc.member;
    }
    if (fail) continue;
    const uint32_t s0 = a.warp_bounds[pc.bounds + wid], s1 = a.warp_bounds[pc.bounds + wid + 1];
    const Dense<V> Dn{(const V *)mb.x, (V *)mb.y, 1u, 0u, nullptr, 0, 0, mb.radixw};
    fail = warp_spmv_range<V, 1, RW>(mb.words, mb.slice_off, mb.unit_row, mb.nunits, mb.ncols, mb.first_rel != 0,
                                     mb.chain, s0, s1, smem, smem + kK * 8, ring_base, bars, Dn, a.beta,
                                     mb.split ? 1 : a.beta_mode, a.err, phase_bits, lane);
  }
  if (fail && lane == 0) atomicExch(a.err, fail);
}

// y_t *= beta for every member t with split rows (before the atomics add in).
template <typename V>
__global__ void batch_scale_kernel(const MemberDev *members, int32_t count, V beta) {
  for (int32_t t = 0; t < count; ++t) {
    if (!members[t].split) continue;
    V *y = (V *)members[t].y;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < members[t].m;
         i += (int64_t)gridDim.x * blockDim.x)
      y[i] = beta == V(0) ? V(0) : y[i] * beta;
  }
}

dtans_status cuda_err(cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return set_error(DTANS_ERR_CUDA, m);
}

}  // namespace
}  // namespace dtans

struct dtans_batch_s {
  std::vector<dtans_handle> hs;
  dtans_dtype dtype = DTANS_F64;
  int device = -1;
  int grid = 0;
  bool any_split = false;
  bool bound = false;
  std::vector<dtans::MemberDev> members;
  dtans::MemberDev *d_members = nullptr;
  dtans::PieceDev *d_pieces = nullptr;
  uint32_t *d_piece_start = nullptr;
  uint32_t *d_warp_bounds = nullptr;
  int32_t *d_err = nullptr;
};

namespace {

void free_batch(dtans_batch_s &b) {
  cudaFree(b.d_members);
  cudaFree(b.d_pieces);
  cudaFree(b.d_piece_start);
  cudaFree(b.d_warp_bounds);
  cudaFree(b.d_err);
  b.d_members = nullptr;
  b.d_pieces = nullptr;
  b.d_piece_start = nullptr;
  b.d_warp_bounds = nullptr;
  b.d_err = nullptr;
}

// First slice s of [lo, hi] with slice_off[s] >= target, moved up to a
// chain start (a multiple of C) and capped at hi.
uint32_t first_at_least(const std::vector<uint64_t> &off, uint32_t lo, uint32_t hi, uint64_t target, uint32_t C = 1) {
  uint32_t s = (uint32_t)(std::lower_bound(off.begin() + lo, off.begin() + hi, target) - off.begin());
  s = (uint32_t)(((uint64_t)s + C - 1) / C * C);
  return std::min(s, hi);
}

}  // namespace

using namespace dtans;
using namespace dtans::core;

namespace {

template <typename V, uint32_t RW>
dtans_status launch_batch(dtans_batch_s &b, double beta, int32_t mode, cudaStream_t st) {
  static std::atomic<uint64_t> configured{0};  // one bit per device
  const int smem = persistent_smem_bytes<V>(kWarpsPerCta, RW);
  const cudaError_t e = ensure_smem_limit(batch_spmv_kernel<V, RW>, smem, configured);
  if (e != cudaSuccess) return cuda_err(e, "cudaFuncSetAttribute(batch)");
  BatchArgs<V> a{b.d_members, b.d_pieces, b.d_piece_start, b.d_warp_bounds, b.d_err, (V)beta, mode};
  batch_spmv_kernel<V, RW><<<b.grid, kThreads, smem, st>>>(a);
  return DTANS_OK;
}

}  // namespace

extern "C" {

dtans_status dtans_batch_create(const dtans_handle *hs, int32_t count, dtans_batch *out) {
  if (!out) return set_error(DTANS_ERR_ARG, "out is null");
  *out = nullptr;
  if (!hs || count < 1) return set_error(DTANS_ERR_ARG, "empty batch");
  std::unique_ptr<dtans_batch_s> b(new dtans_batch_s());
  int dev = 0;
  cudaGetDevice(&dev);
  b->device = dev;
  b->dtype = hs[0] ? hs[0]->dtype : DTANS_F64;
  for (int32_t t = 0; t < count; ++t) {
    dtans_handle h = hs[t];
    if (!h) return set_error(DTANS_ERR_ARG, "null member handle");
    if (!h->uploaded || h->device != dev) return set_error(DTANS_ERR_STATE, "member not uploaded on this device");
    if (h->dtype != b->dtype) return set_error(DTANS_ERR_ARG, "members must share one dtype");
    if (h->opts.escape_stream)
      return set_error(DTANS_ERR_UNSUPPORTED, "batch member with a separate escape stream");
    b->hs.push_back(h);
    MemberDev md{};
    md.words = h->d_words;
    md.slice_off = h->d_slice_off;
    md.tables = h->d_tables;
    md.unit_row = h->d_unit_row;
    md.nunits = h->nunits;
    md.m = h->m;
    md.ncols = (uint32_t)std::max<int64_t>(h->n, 1);
    md.split = h->any_split ? 1 : 0;
    md.first_rel = h->opts.first_delta;
    md.chain = (uint32_t)std::max(1, h->opts.chain_slices);
    md.radixw = h->radix_w ? 1 : 0;
    b->any_split = b->any_split || h->any_split;
    b->members.push_back(md);
  }
  // pieces: the concatenated slices cut into `grid` word-balanced parts
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = std::max(1, sms);
  b->grid = grid;
  std::vector<uint64_t> base(count + 1, 0);
  for (int32_t t = 0; t < count; ++t) base[t + 1] = base[t] + (hs[t]->slice_off.empty() ? 0 : hs[t]->slice_off.back());
  const uint64_t total = base[count];
  std::vector<PieceDev> pieces;
  std::vector<uint32_t> piece_start(grid + 1, 0), bounds;
  // global cut points in word space, snapped to slice starts of the member that contains them
  auto cut = [&](uint64_t w) -> std::pair<int32_t, uint32_t> {  // (member, slice)
    if (w >= total) return {count, 0};
    int32_t t = (int32_t)(std::upper_bound(base.begin(), base.end(), w) - base.begin()) - 1;
    const auto &off = hs[t]->slice_off;
    uint32_t s = first_at_least(off, 0, (uint32_t)hs[t]->nslices, w - base[t], b->members[t].chain);
    if (s >= hs[t]->nslices) return {t + 1, 0};
    return {t, s};
  };
  std::pair<int32_t, uint32_t> prev = {0, 0};
  for (int c = 0; c < grid; ++c) {
    piece_start[c] = (uint32_t)pieces.size();
    std::pair<int32_t, uint32_t> next = c + 1 == grid ? std::make_pair(count, 0u)
                                                      : cut((uint64_t)((__int128)total * (c + 1) / grid));
    if (next < prev) next = prev;
    // members touched by [prev, next)
    for (int32_t t = prev.first; t < count && std::make_pair(t, 0u) < next; ++t) {
      const uint32_t s0 = t == prev.first ? prev.second : 0;
      const uint32_t s1 = t == next.first ? next.second : (uint32_t)hs[t]->nslices;
      if (s1 <= s0) continue;
      PieceDev pd{(uint32_t)t, (uint32_t)bounds.size()};
      const auto &off = hs[t]->slice_off;
      const uint64_t w0 = off[s0], w1 = off[s1];
      for (int w = 0; w <= kWarpsPerCta; ++w) {
        uint32_t s = w == kWarpsPerCta ? s1
                                       : first_at_least(off, s0, s1, w0 + (w1 - w0) * (uint64_t)w / kWarpsPerCta,
                                                        b->members[t].chain);
        bounds.push_back(std::max(s0, std::min(s, s1)));
      }
      pieces.push_back(pd);
    }
    prev = next;
  }
  piece_start[grid] = (uint32_t)pieces.size();
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_members, sizeof(MemberDev) * count)) != cudaSuccess ||
      (e = cudaMalloc(&b->d_pieces, sizeof(PieceDev) * std::max<size_t>(1, pieces.size()))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_piece_start, 4 * piece_start.size())) != cudaSuccess ||
      (e = cudaMalloc(&b->d_warp_bounds, 4 * std::max<size_t>(1, bounds.size()))) != cudaSuccess ||
      (e = cudaMalloc(&b->d_err, 16)) != cudaSuccess) {
    free_batch(*b);
    return set_error(DTANS_ERR_ALLOC, "device allocation failed");
  }
  if ((!pieces.empty() &&
       (e = cudaMemcpy(b->d_pieces, pieces.data(), sizeof(PieceDev) * pieces.size(), cudaMemcpyHostToDevice)) !=
           cudaSuccess) ||
      (e = cudaMemcpy(b->d_piece_start, piece_start.data(), 4 * piece_start.size(), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (!bounds.empty() &&
       (e = cudaMemcpy(b->d_warp_bounds, bounds.data(), 4 * bounds.size(), cudaMemcpyHostToDevice)) != cudaSuccess) ||
      (e = cudaMemset(b->d_err, 0, 16)) != cudaSuccess) {
    free_batch(*b);
    return cuda_err(e, "batch upload");
  }
  *out = b.release();
  return DTANS_OK;
}

dtans_status dtans_batch_bind(dtans_batch b, const void *const *xs, void *const *ys) {
  if (!b || !xs || !ys) return set_error(DTANS_ERR_ARG, "null argument");
  for (size_t t = 0; t < b->members.size(); ++t) {
    if ((b->hs[t]->m > 0 && !ys[t]) || (b->hs[t]->nnz > 0 && !xs[t])) return set_error(DTANS_ERR_ARG, "null vector");
    b->members[t].x = xs[t];
    b->members[t].y = ys[t];
  }
  cudaError_t e = cudaMemcpy(b->d_members, b->members.data(), sizeof(MemberDev) * b->members.size(),
                             cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_err(e, "batch bind");
  b->bound = true;
  return DTANS_OK;
}

dtans_status dtans_batch_spmv(dtans_batch b, double beta, void *stream) {
  if (!b) return set_error(DTANS_ERR_ARG, "null batch");
  if (!b->bound) return set_error(DTANS_ERR_STATE, "batch vectors not bound (dtans_batch_bind)");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != b->device) return set_error(DTANS_ERR_STATE, "batch was created on another device");
  cudaStream_t st = (cudaStream_t)stream;
  const bool f64 = b->dtype == DTANS_F64;
  cudaError_t e;
  if (b->any_split && beta != 1.0) {
    if (f64)
      batch_scale_kernel<double><<<std::max(1, b->grid * 4), 256, 0, st>>>(b->d_members, (int32_t)b->members.size(),
                                                                           beta);
    else
      batch_scale_kernel<float><<<std::max(1, b->grid * 4), 256, 0, st>>>(b->d_members, (int32_t)b->members.size(),
                                                                          (float)beta);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "batch scale launch");
  }
  const int32_t mode = beta == 0.0 ? 0 : (beta == 1.0 ? 1 : 2);
  const dtans_status s = f64 ? launch_batch<double, kRingWords>(*b, beta, mode, st)
                            : launch_batch<float, kRingWords>(*b, beta, mode, st);
  if (s != DTANS_OK) return s;
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_err(e, "batch launch");
  return DTANS_OK;
}

void dtans_batch_destroy(dtans_batch b) {
  if (!b) return;
  free_batch(*b);
  delete b;
}

}  // extern "C"

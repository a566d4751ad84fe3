// Device helpers shared by the CSR-dtANS kernels: table entries, unpack, the
// per-group state update of the dtANS decoder, and thin PTX wrappers for
// mbarriers and 1-D bulk (TMA) copies.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "dtans_internal.h"

namespace dtans {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// Error codes written to a kernel's error word.
enum : int32_t { kErrOverrun = 1, kErrColumn = 2, kErrTimeout = 3, kErrRange = 4 };

// Table entries as stored in the device image (see build_table_image):
//   delta: {delta, meta};  FP32 value: {bits, meta};  FP64 value: {value, meta, coef}
// meta = digit | kMetaEsc | kMetaUnused | base << 16; coef is the integer
// coefficient c of a table whose kept values are all c * 2^e (else 0).
struct __align__(8) DeltaEntry {
  uint32_t delta;
  uint32_t meta;
};
template <typename V>
struct ValueEntry;
template <>
struct __align__(16) ValueEntry<double> {
  double v;
  uint32_t meta;
  int32_t coef;
};
template <>
struct __align__(8) ValueEntry<float> {
  float v;
  uint32_t meta;
};
template <typename V>
struct RawWords {
  static constexpr int kValue = sizeof(V) / 4;  // words of an escaped value
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// 32 bytes at p (eight FP32 or four FP64 values) with one load through the
// read-only path: p 32-byte aligned, the data unchanged while the kernel runs.
__device__ __forceinline__ void ldg32(const float *p, float *r) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
      : "l"(p));
}
__device__ __forceinline__ void ldg32(const double *p, double *r) {
  asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(r[0]), "=d"(r[1]), "=d"(r[2]), "=d"(r[3]) : "l"(p));
}

__device__ __forceinline__ uint32_t digit_of(uint32_t meta) { return meta & 0xffu; }
__device__ __forceinline__ uint32_t base_of(uint32_t meta) { return meta >> 16; }

// Byte offsets of the 8 slots of a segment in tables of entry size `DS`
// (delta, even slots) and `VS` (value, odd slots).  The three words are one
// 96-bit number w0:w1:w2 with w0 most significant; slot k is bits
// [12k, 12k + 12) (Sec. IV-D "Words in v": slot 1 is the least significant).
template <int DS, int VS>
__device__ __forceinline__ void unpack_offsets(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t (&o)[8]) {
  static_assert(DS == 8, "delta entries are 8 bytes");
  constexpr int vs = VS == 16 ? 4 : 3;  // log2 of the value entry size
  o[0] = (w2 << 3) & (0xfffu << 3);
  o[1] = (w2 >> (12 - vs)) & (0xfffu << vs);
  o[2] = (__funnelshift_r(w2, w1, 24) << 3) & (0xfffu << 3);
  o[3] = (w1 >> (4 - vs)) & (0xfffu << vs);  // vs <= 4
  o[4] = (w1 >> (16 - 3)) & (0xfffu << 3);
  o[5] = (__funnelshift_r(w1, w0, 28) << vs) & (0xfffu << vs);
  o[6] = (w0 >> (8 - 3)) & (0xfffu << 3);
  o[7] = (w0 >> (20 - vs)) & (0xfffu << vs);
}

// One check group of four slots (Sec. IV-D; four digits per word-sized
// digit/base pair, Sec. IV-F "Positioning of checks"): appends the digits to
// the state, d = d * R + D and r = r * R with R = b0 b1 b2 b3 <= 2^32, then
// either extracts a word (r >= W = 2^32) or asks for one to be read.
// D < R fits 32 bits; R - 1 is computed modulo 2^32, which is exact because
// 0 <= R - 1 < 2^32 (the decremented radix of Sec. IV-F).  d, r < 2^32 on
// entry and exit; returns true when a read is needed.
__device__ __forceinline__ bool group_step(uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3, uint32_t &d,
                                           uint32_t &r, uint32_t &wout) {
  const uint32_t b0 = base_of(m0), b1 = base_of(m1), b2 = base_of(m2), b3 = base_of(m3);
  const uint32_t D = ((digit_of(m0) * b1 + digit_of(m1)) * b2 + digit_of(m2)) * b3 + digit_of(m3);
  const uint32_t Rm = b0 * b1 * b2 * b3 - 1u;
  const uint64_t dd = (uint64_t)d * Rm + ((uint64_t)d + D);  // d * R + D
  const uint64_t rr = (uint64_t)r * Rm + r;                  // r * R
  const uint32_t rhi = (uint32_t)(rr >> 32);
  const bool ext = rhi != 0;  // r * R >= W: a whole word can be extracted
  wout = ext ? (uint32_t)dd : wout;
  d = ext ? (uint32_t)(dd >> 32) : (uint32_t)dd;
  r = ext ? rhi : (uint32_t)rr;
  return !ext;
}

// A group whose four symbols all have multiplicity M = 256 has radix
// R = 256^4 = 2^32 = W: its check always extracts, d and r come out unchanged
// (d * W + D has high word d, r * W has high word r) and the extracted word is
// D = d0 d1 d2 d3 in base 256, i.e. the four digits packed as bytes.
__device__ __forceinline__ bool all_base_w(uint32_t m) { return (m & (1u << 24)) != 0; }  // base == 256

__device__ __forceinline__ uint32_t pack_digits(uint32_t m0, uint32_t m1, uint32_t m2, uint32_t m3) {
  const uint32_t hi = __byte_perm(m1, m0, 0x0040);  // (d0 << 8) | d1
  const uint32_t lo = __byte_perm(m3, m2, 0x0040);  // (d2 << 8) | d3
  return __byte_perm(lo, hi, 0x5410);               // d0 d1 d2 d3, d0 most significant
}

// Exclusive prefix sum over the warp of per-lane counts c < 8 and the warp
// total, from one ballot per bit of c (no shuffles, no dependent chain).
__device__ __forceinline__ uint32_t warp_prefix8(uint32_t c, uint32_t lt, uint32_t &total) {
  const uint32_t b0 = __ballot_sync(kFull, c & 1u), b1 = __ballot_sync(kFull, c & 2u);
  const uint32_t b2 = __ballot_sync(kFull, c & 4u);
  total = __popc(b0) + 2u * __popc(b1) + 4u * __popc(b2);
  return __popc(b0 & lt) + 2u * __popc(b1 & lt) + 4u * __popc(b2 & lt);
}

// The same for counts c < 16.
__device__ __forceinline__ uint32_t warp_prefix16(uint32_t c, uint32_t lt, uint32_t &total) {
  const uint32_t b0 = __ballot_sync(kFull, c & 1u), b1 = __ballot_sync(kFull, c & 2u);
  const uint32_t b2 = __ballot_sync(kFull, c & 4u), b3 = __ballot_sync(kFull, c & 8u);
  total = __popc(b0) + 2u * __popc(b1) + 4u * __popc(b2) + 8u * __popc(b3);
  return __popc(b0 & lt) + 2u * __popc(b1 & lt) + 4u * __popc(b2 & lt) + 8u * __popc(b3 & lt);
}

// ---------------------------------------------------------------------------
// mbarrier and bulk-copy wrappers (sm_90+ PTX)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// If `issue` is non-zero: arms the barrier for `bytes` of transaction and
// issues one bulk copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned) into shared memory.  Predicated, so a warp can call it without
// branching (only the lane with issue != 0 acts).
__device__ __forceinline__ void bulk_load(uint32_t issue, uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %0, 0;\n\t"
      "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%4], %3;\n\t"
      "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%1], [%2], %3, [%4];\n\t}" ::"r"(issue),
      "r"(dst), "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Warp-collective wait for the phase with the given parity: every lane polls
// and the loop ends when all lanes have seen the phase complete, so the
// result is warp-uniform.  Gives up after `limit` polls and returns false
// (the caller records an error).
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (__all_sync(kFull, done)) return true;
  }
  return false;
}

}  // namespace dev
}  // namespace dtans

// Microbenchmarks of the secondary ceilings of the decode-fused SpMV on the
// current GPU (measurement infrastructure for the benchmark, not part of the
// CSR-dtANS library): the FP64 FMA pipe (one DFMA per stored entry bounds the
// FP64 products), the 32-bit integer multiply-add rate (the dtANS state
// update and unpacking), and shared-memory loads at random and at
// conflict-free addresses (the table lookups).  Every kernel runs a fixed
// number of iterations on in-bounds addresses and waits on nothing.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

namespace {

thread_local std::string g_err;

constexpr int kThreads = 256;
constexpr int kChains = 8;  // independent accumulators per thread

__global__ void __launch_bounds__(kThreads) dfma_kernel(double *sink, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) imad_kernel(uint32_t *sink, int iters, uint32_t b, uint32_t c) {
  uint32_t a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = threadIdx.x * 7u + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = a[i] * b + c;
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s ^= a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 32 x 32 -> 64-bit multiply-adds (mad.wide), signed or unsigned, and the
// high half of a 32 x 32 product (mad.hi): their rates decide whether wide
// integer arithmetic can stand in for FP64 FMAs.
template <int kOp>
__global__ void __launch_bounds__(kThreads) imad_wide_kernel(long long *sink, int iters, int b, int c) {
  long long a[kChains];
  int bb[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    a[i] = threadIdx.x + i;
    bb[i] = b + i;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      if constexpr (kOp == 0) {
        asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(a[i]) : "r"(bb[i]), "r"(c));
      } else if constexpr (kOp == 1) {
        asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(a[i]) : "r"(bb[i]), "r"(c));
      } else {
        uint32_t lo = (uint32_t)a[i];
        asm("mad.hi.u32 %0, %1, %2, %0;" : "+r"(lo) : "r"(bb[i]), "r"(c));
        a[i] = lo;
      }
    }
  }
  long long s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s ^= a[i];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int kSmemWords = 4096;  // 16 KB (bank statistics do not depend on the size)

// Each thread reads kChains shared-memory words per iteration.  random != 0:
// word addresses from a per-thread 32-bit LCG (independent of the loaded
// values, so the loads pipeline), masked into the array; random == 0: lane
// and iteration give consecutive words (no bank conflicts).
__global__ void __launch_bounds__(kThreads) lds_kernel(uint32_t *sink, int iters, int random) {
  __shared__ uint32_t tab[kSmemWords];
  for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x) tab[i] = i * 2654435761u;
  __syncthreads();
  uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 747796405u + 2891336453u;
  uint32_t acc = 0;
  const uint32_t lin = threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      uint32_t idx;
      if (random) {
        x = x * 1664525u + 1013904223u;
        idx = x >> 20;  // 12 bits: [0, kSmemWords)
      } else {
        idx = (lin + (uint32_t)(it * kChains + i) * 32u) & (kSmemWords - 1);
      }
      acc += tab[idx];
    }
  }
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

}  // namespace

extern "C" {

const char *dtc_last_error(void) { return g_err.c_str(); }

// out[0] DFMA TFLOP/s (2 flop per FMA), out[1] FP64 FMAs per clock per SM,
// out[2] 32-bit IMADs per clock per SM, out[3] random shared-memory 32-bit
// loads (lanes) per clock per SM, out[4] conflict-free ones, out[5] the SM
// clock (MHz) the per-clock figures use (the device's maximum clock), out[6]
// SMs, out[7] signed 32 x 32 -> 64-bit multiply-adds (mad.wide.s32) per
// clock per SM, out[8] unsigned ones (mad.wide.u32), out[9] high-half
// multiply-adds (mad.hi.u32).  Each figure is the best of `reps` timed
// launches.  Returns 0, or -1 with dtc_last_error() set.
int dtc_ceilings(double *out, int reps) {
  int dev = 0, sms = 0, khz = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess) {
    g_err = "device query failed";
    return -1;
  }
  if (reps < 1) reps = 3;
  const int blocks = sms * 4;  // 32 warps per SM, all resident in one wave
  void *sink = nullptr;
  if (cudaMalloc(&sink, (size_t)blocks * kThreads * 8) != cudaSuccess) {
    g_err = "cudaMalloc failed";
    return -1;
  }
  Timer t;
  const double hz = khz * 1e3;
  auto best_ms = [&](auto launch) {
    float best = 1e30f;
    launch();  // warm-up
    for (int r = 0; r < reps; ++r) {
      cudaEventRecord(t.a);
      launch();
      cudaEventRecord(t.b);
      cudaEventSynchronize(t.b);
      float ms = 0;
      cudaEventElapsedTime(&ms, t.a, t.b);
      if (ms < best) best = ms;
    }
    return (double)best;
  };
  const int it_fma = 4096, it_lds = 2048;
  const double n_fma = (double)blocks * kThreads * kChains * it_fma;
  const double n_lds = (double)blocks * kThreads * kChains * it_lds;
  const double t_dfma = best_ms([&] { dfma_kernel<<<blocks, kThreads>>>((double *)sink, it_fma, 0.999, 1e-3); });
  const double t_imad = best_ms([&] { imad_kernel<<<blocks, kThreads>>>((uint32_t *)sink, it_fma, 1664525u, 7u); });
  const double t_iw0 = best_ms([&] { imad_wide_kernel<0><<<blocks, kThreads>>>((long long *)sink, it_fma, 1664525, 7); });
  const double t_iw1 = best_ms([&] { imad_wide_kernel<1><<<blocks, kThreads>>>((long long *)sink, it_fma, 1664525, 7); });
  const double t_ihi = best_ms([&] { imad_wide_kernel<2><<<blocks, kThreads>>>((long long *)sink, it_fma, 1664525, 7); });
  const double t_ldr = best_ms([&] { lds_kernel<<<blocks, kThreads>>>((uint32_t *)sink, it_lds, 1); });
  const double t_ldl = best_ms([&] { lds_kernel<<<blocks, kThreads>>>((uint32_t *)sink, it_lds, 0); });
  cudaFree(sink);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_err = std::string("ceilings: ") + cudaGetErrorString(e);
    return -1;
  }
  const double per_sm_clk = (double)sms * hz;
  out[0] = 2.0 * n_fma / (t_dfma * 1e-3) / 1e12;
  out[1] = n_fma / (t_dfma * 1e-3) / per_sm_clk;
  out[2] = n_fma / (t_imad * 1e-3) / per_sm_clk;
  out[3] = n_lds / (t_ldr * 1e-3) / per_sm_clk;
  out[4] = n_lds / (t_ldl * 1e-3) / per_sm_clk;
  out[5] = hz / 1e6;
  out[6] = sms;
  out[7] = n_fma / (t_iw0 * 1e-3) / per_sm_clk;
  out[8] = n_fma / (t_iw1 * 1e-3) / per_sm_clk;
  out[9] = n_fma / (t_ihi * 1e-3) / per_sm_clk;
  return 0;
}

}  // extern "C"

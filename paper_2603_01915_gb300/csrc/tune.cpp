// Measurement-driven choice of the CSR-dtANS layout: encode the matrix with
// each candidate (rows split into units of at most U entries, optional
// ordering by unit length), upload it, time the product with CUDA events on
// the device (L2 flushed between repetitions) and keep the fastest handle.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "dtans_internal.h"

using namespace dtans;

namespace {

dtans_status tune_cuda(cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return set_error(DTANS_ERR_CUDA, m);
}

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

}  // namespace

extern "C" {

dtans_status dtans_tune(int64_t m, int64_t n, const int64_t *row_ptr, const uint32_t *col_idx, const void *vals,
                        dtans_dtype dtype, const dtans_tune_opts *opts, dtans_handle *out, dtans_tune_report *rep,
                        void *stream) {
  if (!out) return set_error(DTANS_ERR_ARG, "out is null");
  *out = nullptr;
  dtans_tune_opts o{};
  if (opts) o = *opts;
  const int k = o.k > 0 ? o.k : 1;
  const int reps = o.reps > 0 ? std::min(o.reps, 50) : 5;
  struct Cand {
    int32_t U, order, first;
  };
  std::vector<Cand> cand;
  if (o.n_candidates > 0) {
    if (o.n_candidates > DTANS_TUNE_MAX) return set_error(DTANS_ERR_ARG, "too many candidates");
    for (int i = 0; i < o.n_candidates; ++i) cand.push_back({o.unit_max_nnz[i], o.row_order[i], o.first_delta[i]});
  } else {
    if (o.first_delta_default < 0 || o.first_delta_default > 2) return set_error(DTANS_ERR_ARG, "bad first_delta");
    int64_t maxlen = 0;
    for (int64_t i = 0; i < m; ++i) maxlen = std::max<int64_t>(maxlen, row_ptr[i + 1] - row_ptr[i]);
    std::vector<std::pair<int32_t, int32_t>> lay{{0, 0}, {0, 1}};
    for (int32_t U : {16, 32, 64, 128})
      if (U < maxlen) {
        lay.push_back({U, 1});
        lay.push_back({U, 0});
      }
    for (const auto &l : lay)
      for (int32_t fd = 0; fd < 2; ++fd)
        if (o.first_delta_default == 2 || o.first_delta_default == fd) cand.push_back({l.first, l.second, fd});
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t vb = dtype == DTANS_F64 ? 8 : 4;
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  DevBuf X, Y, F;
  cudaError_t e;
  const size_t xbytes = std::max<size_t>(16, (size_t)n * k * vb), ybytes = std::max<size_t>(16, (size_t)m * k * vb);
  const size_t fbytes = std::max<size_t>(1 << 20, 2 * (size_t)l2);
  if ((e = cudaMalloc(&X.p, xbytes)) != cudaSuccess || (e = cudaMalloc(&Y.p, ybytes)) != cudaSuccess ||
      (e = cudaMalloc(&F.p, fbytes)) != cudaSuccess)
    return tune_cuda(e, "tuner buffers");
  // x = small positive values (any finite input gives the same timings)
  if ((e = cudaMemsetAsync(X.p, 0x3c, xbytes, st)) != cudaSuccess) return tune_cuda(e, "tuner x");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best_ms = 1e300;
  dtans_handle best = nullptr;
  int best_i = -1;
  dtans_tune_report r{};
  dtans_status status = DTANS_OK;
  for (size_t i = 0; i < cand.size() && status == DTANS_OK; ++i) {
    dtans_encode_opts eo{};
    eo.unit_max_nnz = cand[i].U;
    eo.row_order = cand[i].order;
    eo.first_delta = cand[i].first;
    eo.num_threads = o.num_threads;
    dtans_handle h = nullptr;
    status = dtans_encode(m, n, row_ptr, col_idx, vals, dtype, &eo, &h);
    if (status != DTANS_OK) break;
    if ((status = dtans_upload(h, stream)) != DTANS_OK) {
      dtans_destroy(h);
      break;
    }
    std::vector<float> t;
    for (int it = 0; it < reps + 2 && status == DTANS_OK; ++it) {
      cudaMemsetAsync(F.p, it & 0xff, fbytes, st);
      cudaEventRecord(e0, st);
      status = dtans_spmm(h, k, X.p, Y.p, 0.0, stream);
      cudaEventRecord(e1, st);
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) status = tune_cuda(e, "tuner timing");
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (it >= 2) t.push_back(ms);
    }
    if (status == DTANS_OK) status = dtans_check(h, stream);
    if (status != DTANS_OK) {
      dtans_destroy(h);
      break;
    }
    std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
    const double med = t[t.size() / 2];
    r.unit_max_nnz[i] = cand[i].U;
    r.row_order[i] = cand[i].order;
    r.first_delta[i] = cand[i].first;
    r.ms[i] = med;
    r.n = (int32_t)i + 1;
    if (med < best_ms) {
      best_ms = med;
      dtans_destroy(best);
      best = h;
      best_i = (int)i;
    } else {
      dtans_destroy(h);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != DTANS_OK) {
    dtans_destroy(best);
    return status;
  }
  r.best = best_i;
  if (rep) *rep = r;
  *out = best;
  return DTANS_OK;
}

}  // extern "C"

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

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  Events() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Events() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// Median time (ms) of dtans_spmm(h, k, X, Y) over `reps` runs after two
// warm-up runs, the flush buffer F rewritten before each run.
dtans_status time_product(dtans_handle h, int k, void *X, void *Y, void *F, size_t fbytes, int reps,
                          cudaStream_t st, double *med) {
  Events ev;
  std::vector<float> t;
  dtans_status status = DTANS_OK;
  cudaError_t e;
  for (int it = 0; it < reps + 2 && status == DTANS_OK; ++it) {
    cudaMemsetAsync(F, it & 0xff, fbytes, st);
    cudaEventRecord(ev.a, st);
    status = dtans_spmm(h, k, X, Y, 0.0, st);
    cudaEventRecord(ev.b, st);
    if ((e = cudaEventSynchronize(ev.b)) != cudaSuccess) status = tune_cuda(e, "tuner timing");
    float ms = 0;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    if (it >= 2) t.push_back(ms);
  }
  if (status != DTANS_OK) return status;
  std::nth_element(t.begin(), t.begin() + t.size() / 2, t.end());
  *med = t[t.size() / 2];
  return DTANS_OK;
}

// Scratch x (small positive values: any finite input gives the same
// timings), y and a 2 x L2 flush buffer for timing products of h with k columns.
struct Scratch {
  DevBuf X, Y, F;
  size_t fbytes = 0;
  dtans_status init(int64_t m, int64_t n, int k, dtans_dtype dtype, cudaStream_t st) {
    const size_t vb = dtype == DTANS_F64 ? 8 : 4;
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    const size_t xbytes = std::max<size_t>(16, (size_t)n * k * vb), ybytes = std::max<size_t>(16, (size_t)m * k * vb);
    fbytes = std::max<size_t>(1 << 20, 2 * (size_t)l2);
    cudaError_t e;
    if ((e = cudaMalloc(&X.p, xbytes)) != cudaSuccess || (e = cudaMalloc(&Y.p, ybytes)) != cudaSuccess ||
        (e = cudaMalloc(&F.p, fbytes)) != cudaSuccess)
      return tune_cuda(e, "tuner buffers");
    if ((e = cudaMemsetAsync(X.p, 0x3c, xbytes, st)) != cudaSuccess) return tune_cuda(e, "tuner x");
    return DTANS_OK;
  }
};

constexpr int32_t kWarpChoices[4] = {20, 24, 28, 32};

// Times the single-vector product for every warp count and keeps the fastest.
dtans_status pick_warps(dtans_handle h, Scratch &S, int reps, cudaStream_t st, int32_t *best, double *ms) {
  double best_ms = 1e300;
  int32_t best_w = 0;
  for (int i = 0; i < 4; ++i) {
    dtans_status s = dtans_set_warps(h, kWarpChoices[i]);
    double t = 0;
    if (s == DTANS_OK) s = time_product(h, 1, S.X.p, S.Y.p, S.F.p, S.fbytes, reps, st, &t);
    if (s != DTANS_OK) return s;
    if (ms) ms[i] = t;
    if (t < best_ms) best_ms = t, best_w = kWarpChoices[i];
  }
  dtans_set_warps(h, best_w);
  if (best) *best = best_w;
  return dtans_check(h, st);
}

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
    int32_t U, order, first, window;
  };
  std::vector<Cand> cand;
  if (o.n_candidates > 0) {
    if (o.n_candidates > DTANS_TUNE_MAX) return set_error(DTANS_ERR_ARG, "too many candidates");
    for (int i = 0; i < o.n_candidates; ++i)
      cand.push_back({o.unit_max_nnz[i], o.row_order[i], o.first_delta[i], o.order_window[i]});
  } else {
    if (o.first_delta_default < 0 || o.first_delta_default > 2) return set_error(DTANS_ERR_ARG, "bad first_delta");
    int64_t maxlen = 0;
    for (int64_t i = 0; i < m; ++i) maxlen = std::max<int64_t>(maxlen, row_ptr[i + 1] - row_ptr[i]);
    // (U, row_order, order_window); the windowed order only differs from the
    // global one when there is more than one window.  Windows of 2048 rows
    // measured best on GB300 for the 4 M-row power-law matrix (0.346 ms;
    // 1024: 0.349, 4096: 0.355, 16384: 0.378).
    constexpr int32_t kWindow = 2048;
    std::vector<Cand> lay;
    for (int32_t U : {0, 16, 32, 64, 128})
      if (U == 0 || U < maxlen) {
        if (U == 0) lay.push_back({0, 0, 0, 0});
        lay.push_back({U, 1, 0, 0});
        if (m > kWindow) lay.push_back({U, 1, 0, kWindow});
        if (U > 0) lay.push_back({U, 0, 0, 0});
      }
    for (const auto &l : lay)
      for (int32_t fd = 0; fd < 2; ++fd)
        if (o.first_delta_default == 2 || o.first_delta_default == fd) cand.push_back({l.U, l.order, fd, l.window});
    if (cand.size() > DTANS_TUNE_MAX) return set_error(DTANS_ERR_UNSUPPORTED, "default candidate list too long");
  }
  cudaStream_t st = (cudaStream_t)stream;
  Scratch S;
  dtans_status status = S.init(m, n, k, dtype, st);
  if (status != DTANS_OK) return status;
  double best_ms = 1e300;
  dtans_handle best = nullptr;
  int best_i = -1;
  dtans_tune_report r{};
  for (size_t i = 0; i < cand.size() && status == DTANS_OK; ++i) {
    dtans_encode_opts eo{};
    eo.unit_max_nnz = cand[i].U;
    eo.row_order = cand[i].order;
    eo.first_delta = cand[i].first;
    eo.order_window = cand[i].window;
    eo.num_threads = o.num_threads;
    dtans_handle h = nullptr;
    status = dtans_encode(m, n, row_ptr, col_idx, vals, dtype, &eo, &h);
    if (status != DTANS_OK) break;
    if ((status = dtans_upload(h, stream)) != DTANS_OK) {
      dtans_destroy(h);
      break;
    }
    double med = 0;
    status = time_product(h, k, S.X.p, S.Y.p, S.F.p, S.fbytes, reps, st, &med);
    if (status == DTANS_OK) status = dtans_check(h, stream);
    if (status != DTANS_OK) {
      dtans_destroy(h);
      break;
    }
    r.unit_max_nnz[i] = cand[i].U;
    r.row_order[i] = cand[i].order;
    r.first_delta[i] = cand[i].first;
    r.order_window[i] = cand[i].window;
    r.warps[i] = 24;
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
  // single vector: the winning layout's warps per CTA
  if (status == DTANS_OK && best && k == 1) {
    double wms[4];
    int32_t w = 0;
    status = pick_warps(best, S, reps, st, &w, wms);
    const int lay = best_i;
    for (int i = 0; i < 4 && status == DTANS_OK; ++i) {
      int j = lay;  // the winning layout's row holds its (re-timed) 24-warp time
      if (kWarpChoices[i] != 24) {
        if (r.n >= DTANS_TUNE_MAX) continue;
        j = r.n++;
        r.unit_max_nnz[j] = r.unit_max_nnz[lay];
        r.row_order[j] = r.row_order[lay];
        r.first_delta[j] = r.first_delta[lay];
        r.order_window[j] = r.order_window[lay];
        r.warps[j] = kWarpChoices[i];
      }
      r.ms[j] = wms[i];
      if (kWarpChoices[i] == w) best_i = j;
    }
  }
  // 16 or more columns: the winning layout with one-pass 16-column tiles
  if (status == DTANS_OK && best && k >= 16 && r.n < DTANS_TUNE_MAX) {
    double t1 = 0;
    status = dtans_set_tile_policy(best, 1);
    if (status == DTANS_OK) status = time_product(best, k, S.X.p, S.Y.p, S.F.p, S.fbytes, reps, st, &t1);
    if (status == DTANS_OK) {
      const int j = r.n++;
      r.unit_max_nnz[j] = r.unit_max_nnz[best_i];
      r.row_order[j] = r.row_order[best_i];
      r.first_delta[j] = r.first_delta[best_i];
      r.order_window[j] = r.order_window[best_i];
      r.warps[j] = r.warps[best_i];
      r.tile_policy[j] = 1;
      r.ms[j] = t1;
      if (t1 < r.ms[best_i])
        best_i = j;
      else
        status = dtans_set_tile_policy(best, 0);
    }
  }
  if (status != DTANS_OK) {
    dtans_destroy(best);
    return status;
  }
  r.best = best_i;
  if (rep) *rep = r;
  *out = best;
  return DTANS_OK;
}

dtans_status dtans_tune_warps(dtans_handle h, int32_t reps, int32_t *best, double *ms, void *stream) {
  if (!h) return set_error(DTANS_ERR_ARG, "null handle");
  if (!h->uploaded) return set_error(DTANS_ERR_STATE, "handle not uploaded (call dtans_upload)");
  cudaStream_t st = (cudaStream_t)stream;
  Scratch S;
  dtans_status s = S.init(h->m, h->n, 1, h->dtype, st);
  if (s != DTANS_OK) return s;
  return pick_warps(h, S, reps > 0 ? std::min(reps, 50) : 5, st, best, ms);
}

}  // extern "C"

// cuSPARSE SpMV baselines for the benchmark (not part of the CSR-dtANS
// library): the same matrix in CSR (SpMV algorithms 1 and 2), COO (1 and 2)
// and sliced ELLPACK (slice 32), each timed with CUDA events after an L2
// flush, as the paper compares against the fastest and the smallest of
// cuSPARSE's CSR, COO and SELL (Sec. V).
#include <cuda_runtime.h>
#include <cusparse.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

namespace {
thread_local std::string g_msg;

struct Dev {
  void *p = nullptr;
  ~Dev() { cudaFree(p); }
  bool alloc(size_t b) { return cudaMalloc(&p, std::max<size_t>(b, 16)) == cudaSuccess; }
};

int fail(const std::string &m) {
  g_msg = m;
  return -1;
}
}  // namespace

constexpr int kWarmBatch = 10;  // back-to-back calls per warm-cache timing

extern "C" {

const char *csb_last_error(void) { return g_msg.c_str(); }

// Times y = A x for each format; results in ms[6] (CSR alg1, CSR alg2, COO
// alg1, COO alg2, SELL alg1, unused) with -1 for a format that failed, and the
// storage bytes of each format in bytes[6] (CSR = 4(m+1) + nnz(4+V), COO =
// nnz(8+V), SELL = padded slices).  row_ptr, cols, vals, x are host arrays.
// flush != 0: a 2 x L2 buffer is written before each timed run (cold cache);
// flush == 0: each timed run is kWarmBatch calls back to back between the two
// events, divided by kWarmBatch (warm cache, Sec. V reports both; the batch
// keeps host launch time out of the figure).
int csb_benchmark_mode(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *cols,
                       const void *vals, int32_t f64, const void *x, int32_t reps, int32_t flush, double *ms,
                       int64_t *bytes) {
  const size_t V = f64 ? 8 : 4;
  const cudaDataType vt = f64 ? CUDA_R_64F : CUDA_R_32F;
  for (int i = 0; i < 6; ++i) ms[i] = -1.0, bytes[i] = 0;
  cusparseHandle_t hs = nullptr;
  if (cusparseCreate(&hs) != CUSPARSE_STATUS_SUCCESS) return fail("cusparseCreate failed");
  struct Guard {
    cusparseHandle_t h;
    ~Guard() { cusparseDestroy(h); }
  } guard{hs};
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  Dev d_rp, d_ci, d_ri, d_v, d_x, d_y, d_flush;
  std::vector<int32_t> rows(nnz);
  for (int64_t i = 0; i < m; ++i)
    for (int32_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) rows[q] = (int32_t)i;
  if (!d_rp.alloc(4 * (m + 1)) || !d_ci.alloc(4 * nnz) || !d_ri.alloc(4 * nnz) || !d_v.alloc(V * nnz) ||
      !d_x.alloc(V * n) || !d_y.alloc(V * m) || !d_flush.alloc(2 * (size_t)l2))
    return fail("device allocation failed");
  cudaMemcpy(d_rp.p, row_ptr, 4 * (m + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(d_ci.p, cols, 4 * nnz, cudaMemcpyHostToDevice);
  cudaMemcpy(d_ri.p, rows.data(), 4 * nnz, cudaMemcpyHostToDevice);
  cudaMemcpy(d_v.p, vals, V * nnz, cudaMemcpyHostToDevice);
  cudaMemcpy(d_x.p, x, V * n, cudaMemcpyHostToDevice);
  bytes[0] = bytes[1] = 4 * (m + 1) + nnz * (int64_t)(4 + V);
  bytes[2] = bytes[3] = nnz * (int64_t)(8 + V);

  // SELL-32: per slice, rows padded to the slice's longest row, column-major
  const int64_t S = 32, nsl = (m + S - 1) / S;
  std::vector<int32_t> sl_off(nsl + 1, 0);
  for (int64_t s = 0; s < nsl; ++s) {
    int32_t L = 0;
    for (int64_t r = s * S; r < std::min(m, (s + 1) * S); ++r) L = std::max(L, row_ptr[r + 1] - row_ptr[r]);
    sl_off[s + 1] = sl_off[s] + L * (int32_t)S;
  }
  const int64_t sell_n = sl_off[nsl];
  std::vector<int32_t> sell_c(sell_n, -1);
  std::vector<uint8_t> sell_v(sell_n * V, 0);
  for (int64_t s = 0; s < nsl; ++s)
    for (int64_t r = s * S; r < std::min(m, (s + 1) * S); ++r)
      for (int32_t k = 0; k < row_ptr[r + 1] - row_ptr[r]; ++k) {
        const int64_t at = sl_off[s] + (int64_t)k * S + (r - s * S);
        sell_c[at] = cols[row_ptr[r] + k];
        std::memcpy(&sell_v[at * V], (const uint8_t *)vals + (row_ptr[r] + k) * V, V);
      }
  bytes[4] = sell_n * (int64_t)(4 + V) + 4 * (nsl + 1);
  Dev d_so, d_sc, d_sv;
  if (!d_so.alloc(4 * (nsl + 1)) || !d_sc.alloc(4 * sell_n) || !d_sv.alloc(V * sell_n))
    return fail("device allocation failed (SELL)");
  cudaMemcpy(d_so.p, sl_off.data(), 4 * (nsl + 1), cudaMemcpyHostToDevice);
  cudaMemcpy(d_sc.p, sell_c.data(), 4 * sell_n, cudaMemcpyHostToDevice);
  cudaMemcpy(d_sv.p, sell_v.data(), V * sell_n, cudaMemcpyHostToDevice);

  cusparseDnVecDescr_t vx = nullptr, vy = nullptr;
  cusparseCreateDnVec(&vx, n, d_x.p, vt);
  cusparseCreateDnVec(&vy, m, d_y.p, vt);
  double one = 1.0, zero = 0.0;
  float onef = 1.0f, zerof = 0.0f;
  const void *alpha = f64 ? (const void *)&one : (const void *)&onef;
  const void *beta = f64 ? (const void *)&zero : (const void *)&zerof;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int fmt = 0; fmt < 5; ++fmt) {
    cusparseSpMatDescr_t A = nullptr;
    cusparseStatus_t st;
    cusparseSpMVAlg_t alg;
    if (fmt < 2) {
      st = cusparseCreateCsr(&A, m, n, nnz, d_rp.p, d_ci.p, d_v.p, CUSPARSE_INDEX_32I, CUSPARSE_INDEX_32I,
                             CUSPARSE_INDEX_BASE_ZERO, vt);
      alg = fmt == 0 ? CUSPARSE_SPMV_CSR_ALG1 : CUSPARSE_SPMV_CSR_ALG2;
    } else if (fmt < 4) {
      st = cusparseCreateCoo(&A, m, n, nnz, d_ri.p, d_ci.p, d_v.p, CUSPARSE_INDEX_32I, CUSPARSE_INDEX_BASE_ZERO, vt);
      alg = fmt == 2 ? CUSPARSE_SPMV_COO_ALG1 : CUSPARSE_SPMV_COO_ALG2;
    } else {
      st = cusparseCreateSlicedEll(&A, m, n, nnz, sell_n, S, d_so.p, d_sc.p, d_sv.p, CUSPARSE_INDEX_32I,
                                   CUSPARSE_INDEX_32I, CUSPARSE_INDEX_BASE_ZERO, vt);
      alg = CUSPARSE_SPMV_SELL_ALG1;
    }
    if (st != CUSPARSE_STATUS_SUCCESS) continue;
    size_t wb = 0;
    Dev work;
    bool ok = cusparseSpMV_bufferSize(hs, CUSPARSE_OPERATION_NON_TRANSPOSE, alpha, A, vx, beta, vy, vt, alg, &wb) ==
                  CUSPARSE_STATUS_SUCCESS &&
              work.alloc(wb);
    std::vector<float> t;
    const int batch = flush ? 1 : kWarmBatch;
    for (int it = 0; ok && it < reps + 2; ++it) {
      if (flush) cudaMemsetAsync(d_flush.p, it & 0xff, 2 * (size_t)l2);
      cudaEventRecord(e0);
      for (int b = 0; ok && b < batch; ++b)
        ok = cusparseSpMV(hs, CUSPARSE_OPERATION_NON_TRANSPOSE, alpha, A, vx, beta, vy, vt, alg, work.p) ==
             CUSPARSE_STATUS_SUCCESS;
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float f = 0;
      cudaEventElapsedTime(&f, e0, e1);
      if (it >= 2) t.push_back(f / batch);
    }
    cusparseDestroySpMat(A);
    if (ok && !t.empty()) {
      std::sort(t.begin(), t.end());
      ms[fmt] = t[t.size() / 2];
    }
    cudaGetLastError();
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cusparseDestroyDnVec(vx);
  cusparseDestroyDnVec(vy);
  return 0;
}

int csb_benchmark(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *cols, const void *vals,
                  int32_t f64, const void *x, int32_t reps, double *ms, int64_t *bytes) {
  return csb_benchmark_mode(m, n, nnz, row_ptr, cols, vals, f64, x, reps, 1, ms, bytes);
}

}  // extern "C"

// Handle management of the CSR-dtANS C ABI: encoding entry point, device
// upload, summaries, host views, error reporting and the file format.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>

#include "dtans_internal.h"

namespace {
thread_local std::string g_err;
}

namespace dtans {
dtans_status set_error(dtans_status st, const std::string &msg) {
  g_err = msg;
  return st;
}

dtans_status cuda_fail(cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return set_error(DTANS_ERR_CUDA, m);
}

void free_device(dtans_handle_s &H) {
  if (!H.uploaded) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (H.device >= 0 && cur != H.device) cudaSetDevice(H.device);
  free_host_io(H);
  cudaFree(H.d_words);
  cudaFree(H.d_slice_off);
  cudaFree(H.d_tables);
  cudaFree(H.d_unit_row);
  cudaFree(H.d_unit_pos);
  cudaFree(H.d_esc_words);
  cudaFree(H.d_esc_off);
  H.d_esc_words = nullptr;
  H.d_esc_off = nullptr;
  cudaFree(H.d_err);
  cudaFree(H.d_vrank);
  H.d_vrank = nullptr;
  cudaFree(H.d_xfix);
  cudaFree(H.d_xexp);
  H.d_xfix = nullptr;
  H.d_xexp = nullptr;
  H.xfix_n = 0;
  for (int i = 0; i < 2; ++i) {
    cudaFree(H.d_warp_slice[i]);
    H.d_warp_slice[i] = nullptr;
    H.warp_slice_n[i] = 0;
  }
  if (H.device >= 0 && cur >= 0 && cur != H.device) cudaSetDevice(cur);
  H.d_words = nullptr;
  H.d_slice_off = nullptr;
  H.d_tables = nullptr;
  H.d_unit_row = nullptr;
  H.d_unit_pos = nullptr;
  H.d_err = nullptr;
  H.uploaded = false;
}
}  // namespace dtans

using namespace dtans;

extern "C" {

const char *dtans_last_error(void) { return g_err.c_str(); }

dtans_status dtans_encode(int64_t m, int64_t n, const int64_t *row_ptr, const uint32_t *col_idx, const void *vals,
                          dtans_dtype dtype, const dtans_encode_opts *opts, dtans_handle *out) {
  if (!out) return set_error(DTANS_ERR_ARG, "out is null");
  *out = nullptr;
  dtans_encode_opts o{};
  if (opts) o = *opts;
  std::unique_ptr<dtans_handle_s> H(new (std::nothrow) dtans_handle_s());
  if (!H) return set_error(DTANS_ERR_ALLOC, "out of host memory");
  try {
    dtans_status st = encode_matrix(m, n, row_ptr, col_idx, vals, dtype, o, *H);
    if (st != DTANS_OK) return st;
  } catch (const std::bad_alloc &) {
    return set_error(DTANS_ERR_ALLOC, "out of host memory while encoding");
  }
  *out = H.release();
  return DTANS_OK;
}

dtans_status dtans_upload(dtans_handle h, void *stream) {
  if (!h) return set_error(DTANS_ERR_ARG, "null handle");
  if (h->uploaded) return DTANS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  h->device = dev;
  h->uploaded = true;  // so that free_device releases partial allocations
  auto alloc = [&](void **p, size_t bytes) -> cudaError_t { return cudaMalloc(p, bytes ? bytes : 16); };
  // The stream is padded by 16 words so that vector loads near the end stay in bounds.
  const size_t wbytes = (h->words.size() + 16) * 4;
  if ((e = alloc((void **)&h->d_words, wbytes)) != cudaSuccess ||
      (e = alloc((void **)&h->d_slice_off, h->slice_off.size() * 8)) != cudaSuccess ||
      (e = alloc((void **)&h->d_tables, h->table_image.size())) != cudaSuccess ||
      (e = alloc((void **)&h->d_unit_pos, h->unit_pos.size() * 8)) != cudaSuccess ||
      (e = alloc((void **)&h->d_err, 16)) != cudaSuccess) {
    free_device(*h);
    return e == cudaErrorMemoryAllocation ? set_error(DTANS_ERR_ALLOC, "device allocation failed")
                                          : cuda_fail(e, "cudaMalloc");
  }
  if (!h->esc_off.empty()) {
    if ((e = alloc((void **)&h->d_esc_words, (h->esc_words.size() + 16) * 4)) != cudaSuccess ||
        (e = alloc((void **)&h->d_esc_off, h->esc_off.size() * 8)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h->d_esc_words, h->esc_words.data(), h->esc_words.size() * 4, cudaMemcpyHostToDevice,
                             s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(h->d_esc_off, h->esc_off.data(), h->esc_off.size() * 8, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess) {
      free_device(*h);
      return e == cudaErrorMemoryAllocation ? set_error(DTANS_ERR_ALLOC, "device allocation failed")
                                            : cuda_fail(e, "upload(escape stream)");
    }
  }
  std::vector<uint32_t> urow;
  if (!h->identity_layout) {
    if ((e = alloc((void **)&h->d_unit_row, h->unit_row.size() * 4)) != cudaSuccess) {
      free_device(*h);
      return set_error(DTANS_ERR_ALLOC, "device allocation failed");
    }
    urow.resize(h->unit_row.size());
    for (size_t u = 0; u < urow.size(); ++u)
      urow[u] = h->unit_row[u] | (h->row_split[h->unit_row[u]] ? 0x80000000u : 0u);
  }
  if ((e = cudaMemsetAsync(h->d_words, 0, wbytes, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->d_words, h->words.data(), h->words.size() * 4, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(h->d_slice_off, h->slice_off.data(), h->slice_off.size() * 8, cudaMemcpyHostToDevice,
                           s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h->d_tables, h->table_image.data(), h->table_image.size(), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(h->d_unit_pos, h->unit_pos.data(), h->unit_pos.size() * 8, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess ||
      (e = cudaMemsetAsync(h->d_err, 0, 16, s)) != cudaSuccess ||
      (!urow.empty() &&
       (e = cudaMemcpyAsync(h->d_unit_row, urow.data(), urow.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    free_device(*h);
    return cuda_fail(e, "upload");
  }
  return DTANS_OK;
}

dtans_status dtans_codebook(dtans_handle h, void *values) {
  if (!h || !values) return set_error(DTANS_ERR_ARG, "null argument");
  const Table &t = h->tab[1];
  for (size_t r = 0; r < t.kept_key.size(); ++r) {
    if (h->dtype == DTANS_F64) {
      std::memcpy((uint64_t *)values + r, &t.kept_key[r], 8);
    } else {
      const uint32_t b = (uint32_t)t.kept_key[r];
      std::memcpy((uint32_t *)values + r, &b, 4);
    }
  }
  return DTANS_OK;
}

dtans_status dtans_set_codebook(dtans_handle h, const void *values, void *stream) {
  if (!h || !values) return set_error(DTANS_ERR_ARG, "null argument");
  if (h->uploaded) {
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != h->device) return set_error(DTANS_ERR_STATE, "handle was uploaded to another device");
  }
  Table &t = h->tab[1];
  for (size_t r = 0; r < t.kept_key.size(); ++r) {
    uint64_t key;
    if (h->dtype == DTANS_F64) {
      std::memcpy(&key, (const uint64_t *)values + r, 8);
    } else {
      uint32_t b;
      std::memcpy(&b, (const uint32_t *)values + r, 4);
      key = b;
    }
    t.kept_key[r] = key;
    for (uint32_t s = t.kept_first[r]; s < t.kept_first[r] + t.kept_mult[r]; ++s) t.slot_key[s] = key;
  }
  build_table_image(*h);
  if (h->uploaded) {
    cudaStream_t st = (cudaStream_t)stream;
    const size_t off = (size_t)kK * 8;  // the value table follows the delta table
    cudaError_t e = cudaMemcpyAsync(h->d_tables + off, h->table_image.data() + off, h->table_image.size() - off,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host image may change on the next call
    if (e != cudaSuccess) return cuda_fail(e, "codebook upload");
  }
  return DTANS_OK;
}

void dtans_destroy(dtans_handle h) {
  if (!h) return;
  free_device(*h);
  delete h;
}

dtans_status dtans_info(dtans_handle h, dtans_info_t *o) {
  if (!h || !o) return set_error(DTANS_ERR_ARG, "null argument");
  std::memset(o, 0, sizeof(*o));
  o->m = h->m, o->n = h->n, o->nnz = h->nnz;
  o->nunits = h->nunits, o->nslices = h->nslices, o->nwords = h->nwords;
  o->bytes_words = 4 * h->nwords;
  o->bytes_slice_off = 8 * (h->nslices + 1);
  o->bytes_tables = (int64_t)h->table_image.size();
  o->bytes_unit_meta = h->identity_layout ? 0 : 4 * h->nunits;
  o->bytes_compressed = o->bytes_words + o->bytes_slice_off + o->bytes_tables + o->bytes_unit_meta;
  o->kept_delta = (int64_t)h->tab[0].kept_key.size();
  o->kept_value = (int64_t)h->tab[1].kept_key.size();
  o->esc_delta = h->tab[0].has_esc, o->esc_value = h->tab[1].has_esc;
  o->dtype = h->dtype;
  o->uploaded = h->uploaded;
  o->cost_bits_delta = h->tab[0].cost_bits, o->cost_bits_value = h->tab[1].cost_bits;
  o->unit_max_nnz = h->opts.unit_max_nnz, o->row_order = h->opts.row_order;
  o->first_delta = h->opts.first_delta;
  o->warps = h->warps ? h->warps : 24;
  o->chain_slices = std::max(1, h->opts.chain_slices);
  o->escape_stream = h->opts.escape_stream;
  o->tile_policy = h->tile_policy;
  o->order_window = h->opts.order_window;
  o->nesc = (int64_t)h->esc_words.size();
  o->bytes_esc = h->esc_off.empty() ? 0 : (int64_t)(4 * h->esc_words.size() + 8 * h->esc_off.size());
  o->bytes_compressed += o->bytes_esc;
  o->grid = h->grid, o->block = h->block;
  o->int_coefficients = h->int_ok ? 1 : 0;
  o->int_exp = h->int_exp;
  o->accumulate = h->accumulate;
  o->int_products = int_products(*h) ? 1 : 0;
  o->scatter = h->scatter;
  return DTANS_OK;
}

dtans_status dtans_view(dtans_handle h, dtans_view_t *o) {
  if (!h || !o) return set_error(DTANS_ERR_ARG, "null argument");
  std::memset(o, 0, sizeof(*o));
  o->words = h->words.data();
  o->slice_off = h->slice_off.data();
  o->unit_row = h->unit_row.data();
  o->unit_len = h->unit_len.data();
  o->unit_pos = h->unit_pos.data();
  for (int d = 0; d < 2; ++d) {
    o->slot_key[d] = h->tab[d].slot_key.data();
    o->slot_digit[d] = h->tab[d].slot_digit.data();
    o->slot_base[d] = h->tab[d].slot_base.data();
    o->slot_kind[d] = h->tab[d].slot_kind.data();
    o->perm[d] = h->tab[d].perm.empty() ? nullptr : h->tab[d].perm.data();
  }
  o->esc_words = h->esc_off.empty() ? nullptr : h->esc_words.data();
  o->esc_off = h->esc_off.empty() ? nullptr : h->esc_off.data();
  return DTANS_OK;
}

dtans_status dtans_check(dtans_handle h, void *stream) {
  if (!h) return set_error(DTANS_ERR_ARG, "null handle");
  if (!h->uploaded) return set_error(DTANS_ERR_STATE, "handle not uploaded");
  int32_t v = 0;
  cudaError_t e;
  cudaStream_t s = (cudaStream_t)stream;
  if ((e = cudaMemcpyAsync(&v, h->d_err, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "dtans_check");
  if (v) {
    cudaMemsetAsync(h->d_err, 0, 4, s);
    cudaStreamSynchronize(s);
    return set_error(DTANS_ERR_CORRUPT, "a kernel met a corrupt stream (code " + std::to_string(v) + ")");
  }
  return DTANS_OK;
}

dtans_status dtans_set_launch(dtans_handle h, int32_t grid, int32_t block) {
  if (!h || grid < 0 || block < 0 || (block && (block % 32 || block > 1024)))
    return set_error(DTANS_ERR_ARG, "bad launch shape");
  h->grid = grid;
  h->block = block;
  return DTANS_OK;
}

dtans_status dtans_set_tile_policy(dtans_handle h, int32_t policy) {
  if (!h || policy < 0 || policy > 1) return set_error(DTANS_ERR_ARG, "tile policy must be 0 or 1");
  h->tile_policy = policy;
  return DTANS_OK;
}

dtans_status dtans_set_scatter(dtans_handle h, int32_t mode) {
  if (!h || mode < 0 || mode > 1) return set_error(DTANS_ERR_ARG, "scatter mode must be 0 or 1");
  h->scatter = mode;
  return DTANS_OK;
}

dtans_status dtans_set_accumulate(dtans_handle h, int32_t mode) {
  if (!h || mode < 0 || mode > 1) return set_error(DTANS_ERR_ARG, "accumulate mode must be 0 or 1");
  h->accumulate = mode;
  return DTANS_OK;
}

dtans_status dtans_set_warps(dtans_handle h, int32_t warps) {
  if (!h || (warps != 0 && warps != 20 && warps != 24 && warps != 28 && warps != 32))
    return set_error(DTANS_ERR_ARG, "warps must be 0, 20, 24, 28 or 32");
  h->warps = warps;
  return DTANS_OK;
}

// ---------------------------------------------------------------------------
// File format: "DTANSv3\0", then int64 header fields, then arrays.
// Versions 1 and 2 (shorter headers) still load.
// ---------------------------------------------------------------------------
namespace {
const char kMagic[8] = {'D', 'T', 'A', 'N', 'S', 'v', '3', 0};
const char kMagicV2[8] = {'D', 'T', 'A', 'N', 'S', 'v', '2', 0};
const char kMagicV1[8] = {'D', 'T', 'A', 'N', 'S', 'v', '1', 0};

struct FileHeader {
  int64_t m, n, nnz, nunits, nslices, nwords;
  int64_t dtype, unit_max_nnz, row_order, has_perm[2];
  uint64_t perm_seed[2];
};
// Version 2 appends this after the version-1 header.
struct FileHeaderV2 {
  int64_t first_delta;
  int64_t chain_slices;
  int64_t escape_stream, nesc;  // nesc words follow the unit metadata, then nslices + 1 offsets
};
// Version 3 appends this after the version-2 header.
struct FileHeaderV3 {
  int64_t order_window;
  int64_t reserved[3];
};

bool wr(FILE *f, const void *p, size_t b) { return b == 0 || fwrite(p, 1, b, f) == b; }
bool rd(FILE *f, void *p, size_t b) { return b == 0 || fread(p, 1, b, f) == b; }
}  // namespace

dtans_status dtans_save(dtans_handle h, const char *path) {
  if (!h || !path) return set_error(DTANS_ERR_ARG, "null argument");
  FILE *f = fopen(path, "wb");
  if (!f) return set_error(DTANS_ERR_IO, std::string("cannot open ") + path);
  FileHeader hd{h->m, h->n, h->nnz, h->nunits, h->nslices, h->nwords, (int64_t)h->dtype,
                h->opts.unit_max_nnz, h->opts.row_order, {!h->tab[0].perm.empty(), !h->tab[1].perm.empty()},
                {h->opts.perm_seed_delta, h->opts.perm_seed_value}};
  const FileHeaderV2 h2{h->opts.first_delta, std::max(1, h->opts.chain_slices), h->opts.escape_stream,
                        (int64_t)h->esc_words.size()};
  const FileHeaderV3 h3{h->opts.order_window, {0, 0, 0}};
  bool ok = wr(f, kMagic, 8) && wr(f, &hd, sizeof(hd)) && wr(f, &h2, sizeof(h2)) && wr(f, &h3, sizeof(h3));
  for (int d = 0; d < 2 && ok; ++d) {
    const Table &t = h->tab[d];
    int64_t nk = (int64_t)t.kept_key.size();
    int64_t esc[3] = {t.has_esc, t.esc_first, t.esc_mult};
    ok = wr(f, &nk, 8) && wr(f, esc, sizeof(esc)) && wr(f, &t.cost_bits, 8) && wr(f, t.kept_key.data(), 8 * nk) &&
         wr(f, t.kept_first.data(), 4 * nk) && wr(f, t.kept_mult.data(), 4 * nk) &&
         wr(f, t.slot_key.data(), 8 * kK) && wr(f, t.slot_digit.data(), 2 * kK) &&
         wr(f, t.slot_base.data(), 2 * kK) && wr(f, t.slot_kind.data(), kK) &&
         (t.perm.empty() || wr(f, t.perm.data(), 4 * kK));
  }
  ok = ok && wr(f, h->words.data(), 4 * h->words.size()) && wr(f, h->slice_off.data(), 8 * h->slice_off.size()) &&
       wr(f, h->unit_row.data(), 4 * h->unit_row.size()) && wr(f, h->unit_len.data(), 4 * h->unit_len.size()) &&
       wr(f, h->unit_pos.data(), 8 * h->unit_pos.size());
  if (ok && h->opts.escape_stream)
    ok = wr(f, h->esc_words.data(), 4 * h->esc_words.size()) && wr(f, h->esc_off.data(), 8 * h->esc_off.size());
  ok = (fclose(f) == 0) && ok;
  return ok ? DTANS_OK : set_error(DTANS_ERR_IO, std::string("write failed: ") + path);
}

dtans_status dtans_load(const char *path, dtans_handle *out) {
  if (!path || !out) return set_error(DTANS_ERR_ARG, "null argument");
  *out = nullptr;
  FILE *f = fopen(path, "rb");
  if (!f) return set_error(DTANS_ERR_IO, std::string("cannot open ") + path);
  std::unique_ptr<FILE, int (*)(FILE *)> guard(f, fclose);
  // the file's length bounds every array the header declares
  int64_t fsize = -1;
  if (std::fseek(f, 0, SEEK_END) == 0) fsize = (int64_t)std::ftell(f);
  if (fsize < 0 || std::fseek(f, 0, SEEK_SET) != 0) return set_error(DTANS_ERR_IO, std::string("cannot read ") + path);
  char mg[8];
  FileHeader hd;
  FileHeaderV2 h2{0, 1, 0, 0};
  FileHeaderV3 h3{0, {0, 0, 0}};
  if (!rd(f, mg, 8)) return set_error(DTANS_ERR_CORRUPT, "bad header");
  const int version = !std::memcmp(mg, kMagic, 8) ? 3 : !std::memcmp(mg, kMagicV2, 8) ? 2
                      : !std::memcmp(mg, kMagicV1, 8) ? 1 : 0;
  if (version == 0 || !rd(f, &hd, sizeof(hd))) return set_error(DTANS_ERR_CORRUPT, "bad header");
  if (version >= 2 && (!rd(f, &h2, sizeof(h2)) || h2.first_delta < 0 || h2.first_delta > 1 || h2.chain_slices < 1 ||
                       h2.chain_slices > 64 || h2.escape_stream < 0 || h2.escape_stream > 1 || h2.nesc < 0 ||
                       h2.nesc > (1ll << 40)))
    return set_error(DTANS_ERR_CORRUPT, "bad header");
  if (version >= 3 && (!rd(f, &h3, sizeof(h3)) || h3.order_window < 0 || h3.order_window >= (1ll << 31)))
    return set_error(DTANS_ERR_CORRUPT, "bad header");
  if (hd.m < 0 || hd.n < 0 || hd.m >= (1ll << 31) || hd.n >= (1ll << 31) || hd.nnz < 0 || hd.nnz > (1ll << 40) ||
      hd.nunits < hd.m || hd.nunits > hd.m + hd.nnz || hd.nslices != (hd.nunits + kSlice - 1) / kSlice ||
      hd.nwords < hd.nunits || hd.nwords > (1ll << 40) || (hd.dtype != DTANS_F32 && hd.dtype != DTANS_F64))
    return set_error(DTANS_ERR_CORRUPT, "inconsistent header");
  {
    // stream, slice offsets, unit metadata and escape arrays must fit in
    // what is left of the file (the tables come on top), checked before
    // anything of that size is allocated
    const int64_t at = (int64_t)std::ftell(f);
    const int64_t need = 4 * hd.nwords + 8 * (hd.nslices + 1) + 16 * hd.nunits +
                         (h2.escape_stream ? 4 * h2.nesc + 8 * (hd.nslices + 1) : 0);
    if (at < 0 || need > fsize - at) return set_error(DTANS_ERR_CORRUPT, "declared sizes exceed the file");
  }
  std::unique_ptr<dtans_handle_s> H(new (std::nothrow) dtans_handle_s());
  if (!H) return set_error(DTANS_ERR_ALLOC, "out of host memory");
  H->m = hd.m, H->n = hd.n, H->nnz = hd.nnz, H->nunits = hd.nunits, H->nslices = hd.nslices, H->nwords = hd.nwords;
  H->dtype = (dtans_dtype)hd.dtype;
  H->opts.unit_max_nnz = (int32_t)hd.unit_max_nnz;
  H->opts.row_order = (int32_t)hd.row_order;
  H->opts.perm_seed_delta = hd.perm_seed[0];
  H->opts.perm_seed_value = hd.perm_seed[1];
  H->opts.first_delta = (int32_t)h2.first_delta;
  H->opts.chain_slices = (int32_t)h2.chain_slices;
  H->opts.escape_stream = (int32_t)h2.escape_stream;
  H->opts.order_window = (int32_t)h3.order_window;
  try {
    for (int d = 0; d < 2; ++d) {
      Table &t = H->tab[d];
      int64_t nk, esc[3];
      if (!rd(f, &nk, 8) || nk < 0 || nk > kK || !rd(f, esc, sizeof(esc)) || !rd(f, &t.cost_bits, 8))
        return set_error(DTANS_ERR_CORRUPT, "bad table header");
      t.kept_key.resize(nk), t.kept_first.resize(nk), t.kept_mult.resize(nk);
      t.slot_key.resize(kK), t.slot_digit.resize(kK), t.slot_base.resize(kK), t.slot_kind.resize(kK);
      t.has_esc = esc[0] != 0, t.esc_first = (uint32_t)esc[1], t.esc_mult = (uint32_t)esc[2];
      if (!rd(f, t.kept_key.data(), 8 * nk) || !rd(f, t.kept_first.data(), 4 * nk) ||
          !rd(f, t.kept_mult.data(), 4 * nk) || !rd(f, t.slot_key.data(), 8 * kK) ||
          !rd(f, t.slot_digit.data(), 2 * kK) || !rd(f, t.slot_base.data(), 2 * kK) ||
          !rd(f, t.slot_kind.data(), kK))
        return set_error(DTANS_ERR_CORRUPT, "truncated table");
      for (int s = 0; s < kK; ++s)
        if (t.slot_kind[s] > 2 || (t.slot_kind[s] && (t.slot_base[s] < 1 || t.slot_base[s] > kM ||
                                                      t.slot_digit[s] >= t.slot_base[s])))
          return set_error(DTANS_ERR_CORRUPT, "bad table slot");
      if (hd.has_perm[d]) {
        t.perm.resize(kK);
        if (!rd(f, t.perm.data(), 4 * kK)) return set_error(DTANS_ERR_CORRUPT, "truncated permutation");
        std::vector<uint8_t> seen(kK, 0);
        for (int s = 0; s < kK; ++s) {
          if (t.perm[s] >= (uint32_t)kK || seen[t.perm[s]]) return set_error(DTANS_ERR_CORRUPT, "bad permutation");
          seen[t.perm[s]] = 1;
        }
      }
    }
    H->words.resize(hd.nwords), H->slice_off.resize(hd.nslices + 1);
    H->unit_row.resize(hd.nunits), H->unit_len.resize(hd.nunits), H->unit_pos.resize(hd.nunits);
  } catch (const std::bad_alloc &) {
    return set_error(DTANS_ERR_ALLOC, "out of host memory");
  }
  if (!rd(f, H->words.data(), 4 * hd.nwords) || !rd(f, H->slice_off.data(), 8 * (hd.nslices + 1)) ||
      !rd(f, H->unit_row.data(), 4 * hd.nunits) || !rd(f, H->unit_len.data(), 4 * hd.nunits) ||
      !rd(f, H->unit_pos.data(), 8 * hd.nunits))
    return set_error(DTANS_ERR_CORRUPT, "truncated stream");
  if (H->slice_off[0] != 0 || H->slice_off[hd.nslices] != (uint64_t)hd.nwords)
    return set_error(DTANS_ERR_CORRUPT, "bad slice offsets");
  if (h2.escape_stream) {
    try {
      H->esc_words.resize(h2.nesc);
      H->esc_off.resize(hd.nslices + 1);
    } catch (const std::bad_alloc &) {
      return set_error(DTANS_ERR_ALLOC, "out of host memory");
    }
    if (!rd(f, H->esc_words.data(), 4 * h2.nesc) || !rd(f, H->esc_off.data(), 8 * (hd.nslices + 1)))
      return set_error(DTANS_ERR_CORRUPT, "truncated escape stream");
    if (H->esc_off[0] != 0 || H->esc_off[hd.nslices] != (uint64_t)h2.nesc)
      return set_error(DTANS_ERR_CORRUPT, "bad escape offsets");
    for (int64_t sl = 0; sl < hd.nslices; ++sl)
      if (H->esc_off[sl + 1] < H->esc_off[sl]) return set_error(DTANS_ERR_CORRUPT, "bad escape offsets");
  }
  for (int64_t s = 0; s < hd.nslices; ++s)
    if (H->slice_off[s + 1] < H->slice_off[s]) return set_error(DTANS_ERR_CORRUPT, "bad slice offsets");
  H->row_split.assign(hd.m, 0);
  std::vector<int64_t> units_of(hd.m, 0);
  int64_t total = 0;
  for (int64_t u = 0; u < hd.nunits; ++u) {
    if ((int64_t)H->unit_row[u] >= hd.m || H->unit_pos[u] + H->unit_len[u] > (uint64_t)hd.nnz)
      return set_error(DTANS_ERR_CORRUPT, "bad unit metadata");
    units_of[H->unit_row[u]] += 1;
    total += H->unit_len[u];
  }
  if (total != hd.nnz) return set_error(DTANS_ERR_CORRUPT, "unit lengths do not add up");
  H->identity_layout = hd.nunits == hd.m;
  for (int64_t r = 0; r < hd.m; ++r) {
    if (units_of[r] == 0) return set_error(DTANS_ERR_CORRUPT, "row without unit");
    if (units_of[r] > 1) H->row_split[r] = 1;
  }
  for (int64_t u = 0; u < hd.nunits && H->identity_layout; ++u)
    if (H->unit_row[u] != (uint32_t)u) H->identity_layout = false;
  H->any_split = hd.nunits != hd.m;
  build_table_image(*H);
  *out = H.release();
  return DTANS_OK;
}

}  // extern "C"

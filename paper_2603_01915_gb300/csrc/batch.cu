// Batched multiply of many CSR-dtANS matrices in one launch (placeholder
// until the persistent kernel lands).
#include "dtans_internal.h"

struct dtans_batch_s {
  int dummy;
};

extern "C" {
dtans_status dtans_batch_create(const dtans_handle *, int32_t, dtans_batch *out) {
  if (out) *out = nullptr;
  return dtans::set_error(DTANS_ERR_UNSUPPORTED, "batched multiply not built yet");
}
dtans_status dtans_batch_bind(dtans_batch, const void *const *, void *const *) {
  return dtans::set_error(DTANS_ERR_UNSUPPORTED, "batched multiply not built yet");
}
dtans_status dtans_batch_spmv(dtans_batch, double, void *) {
  return dtans::set_error(DTANS_ERR_UNSUPPORTED, "batched multiply not built yet");
}
void dtans_batch_destroy(dtans_batch) {}
}

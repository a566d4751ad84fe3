// dtans_spmv_host: y = A x + beta y with x and y in host memory.
//
// The handle keeps kSets sets of device buffers (x and y) and three streams
// of its own: copies in, products, copies out.  Call i uses buffer set
// i % kSets.  Each buffer waits only for its own last user: the copy of x in
// waits for the product that last read that x buffer, and the product (or,
// with beta != 0, the copy of y in) waits for the copy out that last read
// that y buffer.  So with pinned host buffers the copies in and out of
// neighbouring calls overlap the product of call i, and a step costs the
// longest of the three instead of their sum.  Events order the three
// streams; the caller's stream waits for the copy out, so work put on it
// after the call runs once y has reached host memory.  The copies in do not
// wait for work already on the caller's stream (that stream waits for every
// earlier call's copy out, so such a wait would serialize consecutive calls):
// the host buffers must hold the call's inputs when it is made.
#include <cuda_runtime.h>

#include <cstdint>

#include "dtans_internal.h"

namespace dtans {

constexpr int kSets = 3;  // buffer sets in turn

struct HostIO {
  int device = -1;
  size_t xbytes = 0, ybytes = 0;
  void *d_x[kSets] = {};
  void *d_y[kSets] = {};
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  cudaEvent_t ev_in[kSets] = {}, ev_comp[kSets] = {}, ev_out[kSets] = {};
  uint64_t calls = 0;
};

namespace {

dtans_status io_fail(cudaError_t e, const char *what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return set_error(DTANS_ERR_CUDA, m);
}

void release(HostIO *io) {
  if (!io) return;
  for (int b = 0; b < kSets; ++b) {
    cudaFree(io->d_x[b]);
    cudaFree(io->d_y[b]);
    if (io->ev_in[b]) cudaEventDestroy(io->ev_in[b]);
    if (io->ev_comp[b]) cudaEventDestroy(io->ev_comp[b]);
    if (io->ev_out[b]) cudaEventDestroy(io->ev_out[b]);
  }
  if (io->s_in) cudaStreamDestroy(io->s_in);
  if (io->s_comp) cudaStreamDestroy(io->s_comp);
  if (io->s_out) cudaStreamDestroy(io->s_out);
  delete io;
}

// Creates the buffers, streams and events on the handle's device.
dtans_status setup(dtans_handle_s &H) {
  HostIO *io = new (std::nothrow) HostIO();
  if (!io) return set_error(DTANS_ERR_ALLOC, "host I/O state");
  const size_t vb = H.dtype == DTANS_F64 ? 8 : 4;
  io->device = H.device;
  io->xbytes = (size_t)H.n * vb;
  io->ybytes = (size_t)H.m * vb;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < kSets && e == cudaSuccess; ++b) {
    if (io->xbytes) e = cudaMalloc(&io->d_x[b], io->xbytes);
    if (e == cudaSuccess && io->ybytes) e = cudaMalloc(&io->d_y[b], io->ybytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->ev_in[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->ev_comp[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->ev_out[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io->s_out, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    release(io);
    return io_fail(e, e == cudaErrorMemoryAllocation ? "cudaMalloc(host I/O buffers)" : "host I/O streams");
  }
  H.host_io = io;
  return DTANS_OK;
}

}  // namespace

void free_host_io(dtans_handle_s &H) {
  if (!H.host_io) return;
  cudaStreamSynchronize(H.host_io->s_out);  // no copy may still target a buffer being freed
  release(H.host_io);
  H.host_io = nullptr;
}

}  // namespace dtans

using namespace dtans;

extern "C" dtans_status dtans_spmv_host(dtans_handle h, const void *x_host, void *y_host, double beta,
                                        void *stream) {
  if (!h) return set_error(DTANS_ERR_ARG, "null handle");
  if (!h->uploaded) return set_error(DTANS_ERR_STATE, "handle not uploaded (call dtans_upload)");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device) return set_error(DTANS_ERR_STATE, "handle was uploaded to another device");
  if ((h->m > 0 && !y_host) || (h->n > 0 && h->nnz > 0 && !x_host)) return set_error(DTANS_ERR_ARG, "null vector");
  if (h->m == 0) return DTANS_OK;
  if (!h->host_io) {
    const dtans_status s = setup(*h);
    if (s != DTANS_OK) return s;
  }
  HostIO &io = *h->host_io;
  cudaStream_t user = (cudaStream_t)stream;
  const int b = (int)(io.calls % kSets);
  const bool reuse = io.calls >= (uint64_t)kSets;  // this set served an earlier call
  cudaError_t e;
  // copy of x in: once the product that last read this x buffer is done
  if (reuse && (e = cudaStreamWaitEvent(io.s_in, io.ev_comp[b], 0)) != cudaSuccess) return io_fail(e, "stream wait");
  if (io.xbytes && x_host &&
      (e = cudaMemcpyAsync(io.d_x[b], x_host, io.xbytes, cudaMemcpyHostToDevice, io.s_in)) != cudaSuccess)
    return io_fail(e, "copy of x to the device");
  // copy of y in (beta != 0): once the copy out that last read this y buffer is done
  if (beta != 0.0) {
    if (reuse && (e = cudaStreamWaitEvent(io.s_in, io.ev_out[b], 0)) != cudaSuccess) return io_fail(e, "stream wait");
    if ((e = cudaMemcpyAsync(io.d_y[b], y_host, io.ybytes, cudaMemcpyHostToDevice, io.s_in)) != cudaSuccess)
      return io_fail(e, "copy of y to the device");
  }
  if ((e = cudaEventRecord(io.ev_in[b], io.s_in)) != cudaSuccess) return io_fail(e, "event record");
  // product: once the inputs are in and the y buffer's last copy out is done
  if ((e = cudaStreamWaitEvent(io.s_comp, io.ev_in[b], 0)) != cudaSuccess) return io_fail(e, "stream wait");
  if (reuse && (e = cudaStreamWaitEvent(io.s_comp, io.ev_out[b], 0)) != cudaSuccess) return io_fail(e, "stream wait");
  const dtans_status s = dtans_spmv(h, io.d_x[b], io.d_y[b], beta, io.s_comp);
  if (s != DTANS_OK) return s;
  if ((e = cudaEventRecord(io.ev_comp[b], io.s_comp)) != cudaSuccess) return io_fail(e, "event record");
  // copy out, then the caller's stream waits for it
  if ((e = cudaStreamWaitEvent(io.s_out, io.ev_comp[b], 0)) != cudaSuccess) return io_fail(e, "stream wait");
  if ((e = cudaMemcpyAsync(y_host, io.d_y[b], io.ybytes, cudaMemcpyDeviceToHost, io.s_out)) != cudaSuccess)
    return io_fail(e, "copy of y to the host");
  if ((e = cudaEventRecord(io.ev_out[b], io.s_out)) != cudaSuccess) return io_fail(e, "event record");
  if ((e = cudaStreamWaitEvent(user, io.ev_out[b], 0)) != cudaSuccess) return io_fail(e, "stream wait");
  ++io.calls;
  return DTANS_OK;
}

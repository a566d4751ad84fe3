/*
 * dtans.h -- C ABI of the CSR-dtANS sparse matrix library for GB300 (sm_103a).
 *
 * CSR-dtANS (arXiv 2603.01915, Sec. II and IV) stores a CSR matrix whose
 * per-row column deltas and values are entropy coded with dtANS: two coding
 * tables of K = 4096 slots (one for deltas, one for values) and one stream of
 * 32-bit words in which the streams of the 32 units of a slice are interleaved
 * in the order a warp consumes them.  The multiply decodes the stream on the
 * fly, so only compressed bytes cross HBM.
 *
 * Conventions (all entry points):
 *   - Every call returns a dtans_status; nothing throws across the ABI.  On an
 *     error, dtans_last_error() gives a message (thread-local, valid until the
 *     next call on the same thread).
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the current device, owned by the caller unless stated.
 *   - Dense vectors and blocks are of the handle's value type (float for
 *     DTANS_F32, double for DTANS_F64).  Blocks of k right-hand sides are
 *     row-major: X is n x k (X[j*k + b]), Y is m x k (Y[i*k + b]).
 *   - Calls that take a `stream` (a cudaStream_t, NULL for the legacy default
 *     stream) are asynchronous with respect to the host; the handle's device
 *     buffers must not be destroyed while work that uses them is in flight.
 *   - A handle may be used from several host threads only if the calls do not
 *     overlap in time.
 *   - A kernel that meets a corrupt stream (a read past its slice, a column
 *     outside [0, n)) skips the offending work and records the fact in a
 *     device word owned by the handle; dtans_check() reports it.
 */
#ifndef DTANS_H
#define DTANS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dtans_handle_s *dtans_handle;
typedef struct dtans_batch_s *dtans_batch;

typedef enum {
  DTANS_OK = 0,
  DTANS_ERR_ARG = -1,         /* invalid argument (null pointer, size out of range, wrong dtype) */
  DTANS_ERR_ALLOC = -2,       /* host or device allocation failed */
  DTANS_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  DTANS_ERR_CORRUPT = -4,     /* a stream or file failed validation */
  DTANS_ERR_UNSUPPORTED = -5, /* option or shape not supported */
  DTANS_ERR_IO = -6,          /* file could not be read or written */
  DTANS_ERR_STATE = -7        /* handle not in the required state (e.g. not uploaded) */
} dtans_status;

typedef enum { DTANS_F32 = 1, DTANS_F64 = 2 } dtans_dtype;

/* Encoder options; a zero-initialised struct gives the paper's canonical
 * format (one unit per row, rows in natural order, canonical slot layout). */
typedef struct {
  /* unit_max_nnz U: 0 = one unit per row (Sec. II: a slice is 32 consecutive
   * rows).  U > 0 splits a row of length L > U into ceil(L/U) units of
   * near-equal length (the first L mod k one longer), each an independent
   * dtANS sequence with its own first delta (see first_delta) -- the "several
   * threads per row" load-balancing remedy of Sec. V/VI. */
  int32_t unit_max_nnz;
  /* row_order: 0 = natural order; 1 = rows ordered by their longest unit
   * (with U = 0: by their length), descending, ties by row index, so slices
   * hold units of similar length (within order_window blocks, see below). */
  int32_t row_order;
  /* Slot permutation seeds for the delta and value tables (Sec. IV-F "Tables
   * in shared memory"): 0 keeps the canonical consecutive layout; non-zero
   * applies a seeded Fisher-Yates shuffle (splitmix64) of the used slots. */
  uint64_t perm_seed_delta;
  uint64_t perm_seed_value;
  /* Host threads for encoding; 0 = all hardware threads. */
  int32_t num_threads;
  /* first_delta: 0 = a unit's first delta is its absolute column (the
   * paper's convention, Sec. IV-A); 1 = the column minus the unit's row,
   * modulo 2^32 (decoding starts the running column at the row).  Option 1 is
   * not in the paper: for banded and stencil matrices it turns the first
   * delta of every row into a few frequent symbols instead of an escape. */
  int32_t first_delta;
  /* chain_slices C (0 or 1 = the paper's one dtANS sequence per unit, up to
   * 64): each lane's units in C consecutive slices form one dtANS sequence,
   * so the decoder state runs on from a unit into the lane's unit of the next
   * slice and only the chain's final segment drops its trailing words (the
   * "several rows per thread" the paper names as future work).  A unit's
   * length word then carries, in bit 31, whether the lane's chain goes on
   * after it.  Saves about 3 words per unit on short rows. */
  int32_t chain_slices;
  /* escape_stream: 0 = escaped raw symbols sit in the stream at each
   * segment's escape point (the paper's choice); 1 = they go, in the same
   * order, to a separate array with per-slice offsets (the alternative the
   * paper describes in Sec. IV-F "Escaping rare values").  Handles with a
   * separate escape stream multiply with the one-slice-per-warp kernels
   * (direct loads); the persistent, batched and no-allocation entry points
   * return DTANS_ERR_UNSUPPORTED for them. */
  int32_t escape_stream;
  /* order_window: with row_order = 1, 0 orders all rows together; w > 0
   * orders each block of w consecutive rows on its own (blocks stay in
   * natural order).  Not in the paper: a slice's rows then stay within w rows
   * of each other, so on banded and near-diagonal matrices the lanes' x
   * gathers share cache lines while slices still hold units of similar
   * length. */
  int32_t order_window;
  int32_t reserved[3];
} dtans_encode_opts;

/* Summary of an encoded matrix. */
typedef struct {
  int64_t m, n, nnz;         /* shape and stored entries                        */
  int64_t nunits, nslices;   /* dtANS sequences and 32-unit slices             */
  int64_t nwords;            /* 32-bit words in the interleaved stream          */
  int64_t bytes_words;       /* 4 * nwords                                      */
  int64_t bytes_slice_off;   /* 8 * (nslices + 1)                               */
  int64_t bytes_tables;      /* device image of both coding tables              */
  int64_t bytes_unit_meta;   /* unit -> row map (0 for the one-unit-per-row layout) */
  int64_t bytes_compressed;  /* words + slice offsets + tables + unit map       */
  int64_t kept_delta, kept_value; /* kept symbols per table (T)                 */
  int32_t esc_delta, esc_value;   /* escape symbol present                      */
  int32_t dtype;                  /* dtans_dtype                                */
  int32_t uploaded;               /* 1 once device buffers exist                */
  double cost_bits_delta, cost_bits_value; /* coded + raw bits chosen per table */
  int32_t unit_max_nnz, row_order;
  int32_t grid, block;            /* launch shape used by the multiply kernels  */
  int32_t first_delta;            /* dtans_encode_opts.first_delta              */
  int32_t warps;                  /* warps per CTA of the single-vector kernel  */
  int32_t chain_slices;           /* dtans_encode_opts.chain_slices (1 = none)  */
  int32_t escape_stream;          /* dtans_encode_opts.escape_stream            */
  int64_t nesc;                   /* words in the separate escape stream        */
  int64_t bytes_esc;              /* 4 * nesc + 8 * (nslices + 1), or 0         */
  int32_t tile_policy;            /* dtans_set_tile_policy                      */
  int32_t order_window;           /* dtans_encode_opts.order_window             */
  int32_t int_coefficients;       /* 1: FP64 value table with integer coefficients
                                     (every kept value c * 2^e, |c| < 2^15, one e) */
  int32_t int_exp;                /* that e                                      */
  int32_t accumulate;             /* dtans_set_accumulate                        */
  int32_t scatter;                /* dtans_set_scatter                           */
  int32_t int_products;           /* 1: single-vector products use the integer-
                                     coefficient kernels (dtans_set_accumulate mode 1
                                     and a table that allows them) */
} dtans_info_t;

/* Read-only host view of the encoded matrix (owned by the handle; valid until
 * dtans_destroy).  Tables are given in canonical slot order per domain
 * (0 = deltas, 1 = values): key (delta, or value bit pattern zero-extended),
 * digit, base (= multiplicity) and kind (0 unused, 1 kept symbol, 2 escape). */
typedef struct {
  const uint32_t *words;      /* [nwords] interleaved stream                    */
  const uint64_t *slice_off;  /* [nslices + 1] word offset of each slice        */
  const uint32_t *unit_row;   /* [nunits] row of each unit                      */
  const uint32_t *unit_len;   /* [nunits] entries of each unit                  */
  const uint64_t *unit_pos;   /* [nunits] CSR position of each unit's first entry */
  const uint64_t *slot_key[2];
  const uint16_t *slot_digit[2];
  const uint16_t *slot_base[2];
  const uint8_t *slot_kind[2];
  const uint32_t *perm[2];    /* canonical slot -> stored slot, or NULL         */
  const uint32_t *esc_words;  /* [nesc] separate escape stream, or NULL         */
  const uint64_t *esc_off;    /* [nslices + 1] its offset per slice, or NULL    */
} dtans_view_t;

/*
 * dtans_encode -- host-side encoding (Sec. II "Encoding", Sec. IV-A..E).
 * Steps: per row, sort entries by column (stable: duplicates keep their input
 * order; a duplicate gives delta 0) and delta-encode (first delta of a unit is
 * its absolute column, Sec. IV-A, or relative to its row, opts->first_delta);
 * histogram both domains; build both coding tables (Sec. III-D, IV-C, IV-F
 * escapes); encode every unit with a forward base pass and a backward digit
 * pass (Sec. IV-E); interleave 32 units per slice (Sec. II "Interleaving for
 * warps").
 *   m, n      rows and columns (0 <= m, n < 2^31)
 *   row_ptr   host, m + 1 int64, non-decreasing, row_ptr[0] = 0
 *   col_idx   host, row_ptr[m] uint32 in [0, n)
 *   vals      host, row_ptr[m] floats or doubles (bit patterns preserved:
 *             -0.0, NaN payloads and infinities round-trip)
 *   opts      may be NULL (canonical)
 *   out       receives a new handle (host data only; see dtans_upload)
 * No CUDA call is made.  Errors: DTANS_ERR_ARG for bad shapes or column
 * indices, DTANS_ERR_ALLOC.
 */
dtans_status dtans_encode(int64_t m, int64_t n, const int64_t *row_ptr, const uint32_t *col_idx, const void *vals,
                          dtans_dtype dtype, const dtans_encode_opts *opts, dtans_handle *out);

/* Allocates the handle's device buffers on the current device and copies the
 * tables, stream and metadata (synchronous).  Idempotent. */
dtans_status dtans_upload(dtans_handle h, void *stream);

/*
 * dtans_spmv -- y = A x + beta y (Sec. III-A; the paper's y = Ax + y is
 * beta = 1, the plain product y = A x is beta = 0).  Decodes A on the fly
 * (Sec. II "Decoding and SpMVM", Algorithm 3).  x: device, n values;
 * y: device, m values.  With beta == 0, y is not read (NaNs in y are not
 * propagated).  Each y_i is a sum in FP of the handle's type, in an order
 * that may differ from CSR order.
 */
dtans_status dtans_spmv(dtans_handle h, const void *x, void *y, double beta, void *stream);

/*
 * dtans_spmv_host -- y = A x + beta y as dtans_spmv, with x (n values) and y
 * (m values) in HOST memory: the end-to-end call for a caller whose vectors
 * live on the host.  The problem is the one of Sec. III-A; moving the vectors
 * is not part of the paper.
 *   x_host, y_host  host buffers, pinned (cudaHostAlloc / cudaHostRegister) or
 *                   pageable; with beta == 0 y_host is only written.
 *   stream          the caller's stream: work put on it after the call runs
 *                   once y_host holds the result.  The call's copies do not
 *                   wait for work already on `stream` (so that consecutive
 *                   calls overlap): x_host (and y_host when beta != 0) must
 *                   hold the inputs when the call is made.  The call returns
 *                   once everything is enqueued: synchronize `stream` before
 *                   reading y_host, and keep both buffers unchanged and alive
 *                   until then.
 * The handle keeps three sets of device x/y buffers and three internal
 * streams (copy in, product, copy out), created by the first call
 * (cudaMalloc of 3 * (n + m) values) and released by dtans_destroy.
 * Consecutive calls use the sets in turn, and each buffer waits only for its
 * own last user (an x buffer for the product that read it, a y buffer for
 * the copy out that read it), so with pinned buffers the copies of
 * neighbouring calls overlap a call's product and a step costs the longest
 * of copy in, product and copy out; pageable buffers make the CUDA runtime
 * stage the copies and the overlap is lost.  One cudaMemcpyAsync per
 * copy: x in, y in (only when beta != 0), y out.  Calls on one handle must
 * come from one host thread at a time.
 * Errors: DTANS_ERR_ARG (null handle or vector), DTANS_ERR_STATE (not
 * uploaded, or uploaded to another device than the current one),
 * DTANS_ERR_CUDA (allocation, copy or launch failure).
 */
dtans_status dtans_spmv_host(dtans_handle h, const void *x_host, void *y_host, double beta, void *stream);

/* dtans_spmm -- Y = A X + beta Y for k >= 1 right-hand sides (row-major
 * X: n x k, Y: m x k, device).  One decode pass feeds up to 32 columns (FP32)
 * or 16 (FP64); larger k is processed in column tiles (dtans_set_tile_policy). */
dtans_status dtans_spmm(dtans_handle h, int32_t k, const void *X, void *Y, double beta, void *stream);

/* dtans_spmv_T -- XG = A^T G + beta XG (G: m x k, XG: n x k, device,
 * row-major).  Decodes A in row order and scatters each product into XG with
 * atomic adds (order of the adds is not fixed). */
dtans_status dtans_spmv_T(dtans_handle h, int32_t k, const void *G, void *XG, double beta, void *stream);

/* dtans_vals_grad -- out[q] = sum_b G[i, b] * X[j, b] for every stored entry
 * q = (i, j) in sorted-CSR order (rows in order, columns ascending within a
 * row): the gradient of sum(G .* (A X)) with respect to the stored values.
 * G: m x k, X: n x k, out: nnz values, all device. */
dtans_status dtans_vals_grad(dtans_handle h, int32_t k, const void *G, const void *X, void *out, void *stream);

/*
 * Codebook of the value domain.  The kept value symbols of the value table,
 * in its rank order (count descending, then bit pattern ascending, fixed at
 * encode time), form a codebook c_0 .. c_{T-1} with T = info.kept_value; every
 * stored value is either one of them or an escaped raw value.  The stream
 * encodes table slots, not values, so replacing the codebook changes the
 * matrix without re-encoding it -- the trainable form of a weight-shared
 * (quantised) sparse layer.  Not in the paper; the decode is its Sec. IV-F
 * table lookup.
 *
 * dtans_codebook     -- copies c_0 .. c_{T-1} to `values` (host, T values of
 *                       the handle's type).
 * dtans_set_codebook -- replaces them with `values` (host, T values): the host
 *                       tables and, if the handle is uploaded, its device value
 *                       table (copied on `stream`, which is synchronised).
 *                       Products issued afterwards use the new values; escaped
 *                       values are unchanged.  dtans_save writes the new values.
 * dtans_codebook_grad -- out[r] = sum over stored entries q = (i, j) whose value
 *                       is c_r of sum_b G[i, b] * X[j, b] (r < T), i.e. the
 *                       gradient of sum(G .* (A X)) with respect to c_r;
 *                       out[T] = the same sum over escaped entries.  G: m x k,
 *                       X: n x k, out: T + 1 values, all device.  Partial sums
 *                       go through shared-memory and global atomic adds, so the
 *                       summation order is not fixed.  Allocates a 8 KB device
 *                       table (slot -> rank) on first use.
 */
dtans_status dtans_codebook(dtans_handle h, void *values);
dtans_status dtans_set_codebook(dtans_handle h, const void *values, void *stream);
dtans_status dtans_codebook_grad(dtans_handle h, int32_t k, const void *G, const void *X, void *out, void *stream);

/* dtans_decode_csr -- decodes the stream back to sorted CSR: col_idx_out
 * (nnz uint32) and vals_out (nnz values), both device, in sorted-CSR order. */
dtans_status dtans_decode_csr(dtans_handle h, uint32_t *col_idx_out, void *vals_out, void *stream);

/* Summary and host view. */
dtans_status dtans_info(dtans_handle h, dtans_info_t *out);
dtans_status dtans_view(dtans_handle h, dtans_view_t *out);

/* Reads the handle's device error word (synchronises the stream).  Returns
 * DTANS_ERR_CORRUPT if a kernel met a corrupt stream since the last check
 * (and clears the word), DTANS_OK otherwise. */
dtans_status dtans_check(dtans_handle h, void *stream);

/* Serialised form (Sec. II: "saved in a file for repeated decoding"):
 * versioned header, tables, stream, slice offsets and unit metadata
 * (version 2 adds first_delta, chain_slices, escape_stream and the escape
 * arrays, version 3 order_window; version-1 files load with the paper's
 * format, version-2 files with order_window 0).
 * dtans_load validates sizes and offsets and returns DTANS_ERR_CORRUPT for
 * an inconsistent file. */
dtans_status dtans_save(dtans_handle h, const char *path);
dtans_status dtans_load(const char *path, dtans_handle *out);

/*
 * dtans_tune -- measurement-driven layout choice (the autotuner).  Encodes
 * the matrix once per candidate layout (unit_max_nnz U, row_order,
 * order_window, first_delta), uploads it to the current device, times
 * dtans_spmm with k columns (CUDA events on `stream`, L2 flushed between
 * repetitions, median of `reps`) and returns the fastest handle (uploaded) in
 * *out.  With n_candidates = 0 the layouts are (U = 0, row_order 0) and,
 * for U = 0 and every U in {16, 32, 64, 128} shorter than the longest row,
 * (U, row_order 1), (U, row_order 1, order_window 4096) when m > 4096, and,
 * for U > 0, (U, row_order 0); each
 * layout is tried with first_delta = first_delta_default, or with both 0 and 1
 * when first_delta_default = 2.  With k = 1 the winner is then timed with
 * every warp count of dtans_set_warps (one report row each) and keeps the
 * fastest; with k >= 16 it is timed with both column-tile policies
 * (dtans_set_tile_policy) and keeps the faster.  The report (optional) lists
 * each candidate's median time and the index of the winner.  Allocates scratch device buffers
 * for x, y and an L2 flush (2 x L2) for the duration of the call.  Errors as
 * dtans_encode / dtans_upload / dtans_spmm.
 */
#define DTANS_TUNE_MAX 64
typedef struct {
  int32_t k;            /* right-hand sides to tune for (0 or 1 = single vector) */
  int32_t reps;         /* timed repetitions per candidate (0 = 5)                */
  int32_t num_threads;  /* host encoder threads (0 = all)                         */
  int32_t n_candidates; /* 0 = the default list                                    */
  int32_t unit_max_nnz[DTANS_TUNE_MAX];
  int32_t row_order[DTANS_TUNE_MAX];
  int32_t first_delta[DTANS_TUNE_MAX];
  int32_t first_delta_default; /* default list: 0, 1, or 2 = both             */
  int32_t order_window[DTANS_TUNE_MAX];
} dtans_tune_opts;

typedef struct {
  int32_t n;    /* candidates timed */
  int32_t best; /* index of the fastest */
  int32_t unit_max_nnz[DTANS_TUNE_MAX];
  int32_t row_order[DTANS_TUNE_MAX];
  int32_t first_delta[DTANS_TUNE_MAX];
  int32_t warps[DTANS_TUNE_MAX];  /* warps per CTA the candidate was timed with */
  int32_t tile_policy[DTANS_TUNE_MAX]; /* column-tile policy it was timed with  */
  double ms[DTANS_TUNE_MAX];
  int32_t order_window[DTANS_TUNE_MAX];
} dtans_tune_report;

dtans_status dtans_tune(int64_t m, int64_t n, const int64_t *row_ptr, const uint32_t *col_idx, const void *vals,
                        dtans_dtype dtype, const dtans_tune_opts *opts, dtans_handle *out, dtans_tune_report *report,
                        void *stream);

/*
 * dtans_spmv_noalloc -- y = A x + beta y exactly like dtans_spmv, for callers
 * that must not allocate device memory at call time: code that runs while
 * allocation is forbidden or too costly (a real-time loop, an allocator-free
 * runtime, a host callback, a pool that has handed out all its memory).
 * dtans_spmv allocates, on its first call for a launch shape, a small device
 * table of per-warp slice ranges; this call keeps those ranges in a fixed
 * device array compiled into the library instead (at most 8192 warps, i.e.
 * grid x warps per CTA <= 8192, such as 256 CTAs of 32 warps: 32 KB, held on
 * every device that loads the library until the process exits) and fills it with a small device kernel, so it
 * performs no cudaMalloc/cudaFree and no host-to-device copy.  The paper has
 * no counterpart; this is a deployment variant.
 *   h         uploaded handle (its device buffers are the inputs)
 *   x, y      device vectors as in dtans_spmv
 *   stream    as in dtans_spmv
 * The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call on a device shares the array, which
 * keeps the last call's ranges: calls that overlap on the GPU (different
 * streams, no ordering between them) race on it and must not be issued.
 * Errors: DTANS_ERR_ARG for a launch shape (dtans_set_launch, dtans_set_warps)
 * above 8192 warps or null vectors, DTANS_ERR_STATE if not uploaded or
 * uploaded to another device, DTANS_ERR_UNSUPPORTED for a handle encoded with
 * escape_stream = 1 (only the one-slice-per-warp kernel decodes a separate
 * escape stream) or a current device with ordinal 64 or more, DTANS_ERR_CUDA.
 */
dtans_status dtans_spmv_noalloc(dtans_handle h, const void *x, void *y, double beta, void *stream);

/* Sets the launch shape of the multiply kernels (0 = automatic): grid = CTAs
 * of every kernel, block = threads per CTA of the one-slice-per-warp kernels
 * (multiple of 32, at most 1024). */
dtans_status dtans_set_launch(dtans_handle h, int32_t grid, int32_t block);

/* Warps per CTA of the persistent single-vector kernel (dtans_spmv, and
 * dtans_spmm with one column): 20, 24, 28 or 32, or 0 for the default (24).
 * Fewer warps leave more registers per thread and more of the SM's 256 KB of
 * L1/shared memory to L1; which count is fastest depends on the matrix
 * (dtans_tune_warps measures it).  Errors: DTANS_ERR_ARG for other counts. */
dtans_status dtans_set_warps(dtans_handle h, int32_t warps);

/* How dtans_spmv_T adds its products into XG.  Mode 0 (default): one atomic
 * add per decoded entry and column (16-byte vector atomics for FP32 tiles of
 * four columns).  Mode 1: warp-aggregated atomics: in each step the lanes of a
 * warp whose entries fall in the same column merge their products by warp
 * shuffles (one match per step) and one lane adds the sum; it pays when rows
 * decoded together share columns (hub columns) and costs a match per step
 * otherwise.  The result is the same sum in another order, within the column
 * bound either way.  Errors: DTANS_ERR_ARG for other modes. */
dtans_status dtans_set_scatter(dtans_handle h, int32_t mode);

/* How single-vector FP64 products (dtans_spmv, dtans_spmm with k = 1,
 * dtans_spmv_host) sum their entries.  Mode 0 (default): one FP64 fused
 * multiply-add per entry.  Mode 1, integer coefficients: when every kept value
 * of the value table is c * 2^e with one e and integers |c| < 2^15 (the
 * 27-point stencil's 26 and -1, graph Laplacians, 0/1 patterns) and no unit
 * has more than 2^16 entries, x is first converted to exact 96-bit fixed point
 * (two small kernels; scratch of 16 bytes per column allocated on first use)
 * and each unit's sum of c x is accumulated exactly in integers, then rounded
 * to FP64 once, so a row whose x all lie within 2^40 of the largest |x| is the
 * correctly rounded product; entries with an escaped value or an x outside
 * that window (and infinities, NaNs) take FP64 fused multiply-adds.  Tables
 * without integer coefficients stay on mode 0's kernel.  Both modes satisfy
 * the row bound |y - A x| <= 8 len u sum |a x|; the results may differ in the
 * last bits.  On GB300 mode 1 measured slower than mode 0 on the 27-point
 * stencil (0.149 ms including its fixed-point pass over x, against 0.121 ms at
 * 24 warps per CTA): it trades one FMA per entry on the narrow FP64 pipe for
 * more integer instructions and wider gathers than that saves.
 * Errors: DTANS_ERR_ARG for other modes. */
dtans_status dtans_set_accumulate(dtans_handle h, int32_t mode);

/* Column tiles of dtans_spmm: policy 0 (default) takes columns with the
 * persistent kernel, 32 or 16 at a time for FP32 and 8 at a time for FP64
 * (then 4, 2, 1); policy 1 takes 16 at a time with the one-slice-per-warp
 * kernel whenever 16 or more columns are left (one decode pass for 16
 * columns).  Which is faster depends on the matrix (measured on GB300:
 * policy 1 is 34 % faster on the escape-heavy FP32 power-law with k = 16 than
 * two 8-column passes, and half as fast on the pruned layer with k = 32 as
 * one 32-column pass); dtans_tune picks it for k >= 16.  Errors:
 * DTANS_ERR_ARG for other values. */
dtans_status dtans_set_tile_policy(dtans_handle h, int32_t policy);

/* dtans_tune_warps -- times dtans_spmv on the current device for each warp
 * count of dtans_set_warps (CUDA events on `stream`, L2 flushed between
 * repetitions, median of `reps`, 0 = 5), keeps the fastest on the handle and
 * writes it to *best (optional) and the medians to ms[4] (optional, in the
 * order 20, 24, 28, 32).  Allocates scratch x, y and a flush buffer for the
 * duration of the call.  The handle must be uploaded. */
dtans_status dtans_tune_warps(dtans_handle h, int32_t reps, int32_t *best, double *ms, void *stream);

void dtans_destroy(dtans_handle h);
const char *dtans_last_error(void);

/*
 * Batched multiply of many matrices of uneven size in one persistent launch.
 * A batch keeps its member handles (which must be uploaded, share one dtype
 * and outlive the batch) and a device task table of (matrix, slice range)
 * items balanced over the SMs.  dtans_batch_bind stores the device pointers
 * of every member's x and y (host arrays of `count` device pointers, copied
 * to the device synchronously); dtans_batch_spmv then computes
 * y_t = A_t x_t + beta y_t for every member t in one kernel launch, with no
 * host-device copy, so the call can be captured in a CUDA graph.
 */
dtans_status dtans_batch_create(const dtans_handle *hs, int32_t count, dtans_batch *out);
dtans_status dtans_batch_bind(dtans_batch b, const void *const *xs, void *const *ys);
dtans_status dtans_batch_spmv(dtans_batch b, double beta, void *stream);
void dtans_batch_destroy(dtans_batch b);

#ifdef __cplusplus
}
#endif
#endif /* DTANS_H */

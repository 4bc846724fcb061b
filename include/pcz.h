/*
 * pcz.h -- C ABI of libpcz: GPU multi-component progressive-precision
 * compression and retrieval of floating-point fields, after Magri & Lindstrom,
 * "A General Framework for Progressive Data Compression and Retrieval".
 *
 * A field x is stored as n components.  Component i is an error-bounded lossy
 * compression y_i = C(e, tau_i) of the residual e = x - x~_{i-1} left by the
 * components before it, and x~_i = x~_{i-1} + D(y_i) (Algorithm 1, Sec. 4.1).
 * Reading the first k components back and summing them left to right gives x~_k
 * (Algorithm 2, Sec. 4.2), with ||x - x~_k||_inf <= tau_k (Eq. 1, Sec. 4.3).
 * The compressor C/D is a zfp-style coder of 4^d-value blocks ("bricks") with
 * one exponent per block and component (Sec. 4.4) and group-tested bit planes
 * (Sec. 2).
 *
 * Conventions shared by every call:
 *  - Fields are dense, x fastest: element (ix, iy, iz) sits at
 *    ix + dims[0] * (iy + dims[1] * iz).  ndims is 1, 2 or 3; extents need not
 *    be multiples of 4.
 *  - Device pointers are CUDA global memory on the current device.  Host
 *    pointers are accepted where stated: pinned (page-locked) host memory is
 *    read or written in place by the kernels through its device mapping (on
 *    a Grace-Blackwell node over the C2C link, overlapped with the
 *    computation), except that a retrieval output of 32 MiB or more in
 *    pinned memory is decoded into device staging slabs of whole brick
 *    layers that the copy engines move to the host while the next slab
 *    decodes.  Results in pinned host memory are complete in stream order,
 *    as after a cudaMemcpyAsync: synchronise cuda_stream before reading them.
 *    Pageable host memory is copied through the same stream, and such calls
 *    return with the data in place.
 *  - cuda_stream is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    are asynchronous on it except where they must read a result back.
 *  - The caller owns its input and output buffers.  The library owns the
 *    component streams (device memory) until pc_streams_free.  Device memory
 *    the library frees (streams, scratch) stays in a stream-ordered pool of
 *    its own for later calls, so that steady-state calls map no new memory;
 *    pc_release_cached_memory hands it back to the driver.
 *  - No C++ exception crosses this interface.  Every call returns a pc_status;
 *    pc_last_error() gives a message for the last failure on this thread.
 *  - Not thread-safe on one pc_streams object; different objects may be used
 *    from different threads.
 */
#ifndef PCZ_H
#define PCZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PC_MAX_COMPONENTS 64

typedef enum { PC_F32 = 1, PC_F64 = 2 } pc_dtype;

typedef enum {
  PC_OK = 0,
  PC_ERR_ARG = 1,              /* a pointer, size, extent or index is invalid */
  PC_ERR_TAU_ORDER = 2,        /* tolerances not finite, positive and strictly decreasing */
  PC_ERR_NONFINITE = 3,        /* the field holds a NaN or an infinity */
  PC_ERR_OOM = 4,              /* a device allocation failed */
  PC_ERR_CUDA = 5,             /* a CUDA call failed; see pc_last_error() */
  PC_ERR_CORRUPT_STREAM = 6,   /* a component stream does not parse */
  PC_ERR_TOL_UNREACHABLE = 7,  /* tolerance finer than the last component's */
  PC_ERR_VERSION = 8           /* serialized data of another format or version */
} pc_status;

typedef struct pc_streams pc_streams; /* opaque */

/* Half-open box [lo, hi) in element units, lo[a] < hi[a] <= dims[a]; entries
 * beyond ndims are ignored.  A NULL box means the whole field. */
typedef struct {
  int64_t lo[3], hi[3];
} pc_box;

/*
 * Algorithm 1 (Sec. 4.1): compresses the field into n components with
 * tolerances tau[0] > tau[1] > ... > tau[n-1] > 0 (absolute, max-norm).
 *   field   device or host pointer to prod(dims) values of dtype.
 *   dims    ndims extents, dims[0] fastest.
 *   tau     host array of n doubles; n in 1..PC_MAX_COMPONENTS.
 *   out     receives a new pc_streams (free with pc_streams_free).
 * The field must be finite (Sec. 6.1: NaN, infinities and signed zeros are not
 * handled); otherwise PC_ERR_NONFINITE and *out is left NULL.  Synchronises
 * once on cuda_stream to read the component sizes back.
 */
pc_status pc_compress(const void *field, const int64_t *dims, int ndims, pc_dtype dtype, const double *tau,
                      int n, void *cuda_stream, pc_streams **out);

/*
 * Tolerance query (Sec. 6.2, "Benefits"): the number of components k that a
 * request at tolerance tau needs, k = min{i : tau_i <= tau} (1-based); a tau at
 * or above tau_1 gives 1.  PC_ERR_TOL_UNREACHABLE when tau < tau_n.
 */
pc_status pc_query_k(const pc_streams *s, double tau, int *k_out);

/*
 * Computed tolerances (Sec. 4.3: tau_i <- ||x - x~_i||_inf kept as metadata, a
 * tighter bound than the prescribed tau_i).  pc_compress records, per
 * component, the largest |fl_T(x - x~_i)| over the field (evaluated in the
 * field's type; 0 once x~_i reproduces x, the lossless limit of Sec. 5.1.3).
 * pc_stream_measured_error returns it for component i (0-based, double,
 * exact).  pc_query_k_measured is pc_query_k on these values: the smallest k
 * with measured_k <= tau, never more components than pc_query_k needs;
 * PC_ERR_TOL_UNREACHABLE when tau is below every measured error.
 */
pc_status pc_stream_measured_error(const pc_streams *s, int i, double *err);
pc_status pc_query_k_measured(const pc_streams *s, double tau, int *k_out);

/*
 * Algorithm 2 (Sec. 4.2): x~_k = fl(...fl(fl(0 + D(y_1)) + D(y_2))... + D(y_k)),
 * written for the box into out (device or host pointer to the box's values,
 * x fastest, dtype of the field).  If tau >= 0, k is taken from pc_query_k(tau)
 * and the k argument is ignored; if tau < 0, k (0..n) is used as given (k = 0
 * writes zeros).  Only bricks that meet the box are decoded (Sec. 6.1: single
 * 4^d blocks can be decoded on their own).
 */
pc_status pc_retrieve(const pc_streams *s, double tau, int k, const pc_box *box, void *out, void *cuda_stream);

/*
 * Incremental refinement (Sec. 4.2: the reconstruction is refined by further
 * loop iterations of Algorithm 2): inout holds x~_k0 on the box (as written by
 * pc_retrieve or pc_refine with k0 components) and receives x~_k, 0 <= k0 <= k
 * <= n.  The result is bit-identical to pc_retrieve with k components.
 * inout is a device or host pointer.
 */
pc_status pc_refine(const pc_streams *s, int k0, int k, const pc_box *box, void *inout, void *cuda_stream);

/*
 * Per-component metadata (the tolerance stored as metadata, Sec. 6.2) and size:
 * component i (0-based) has tolerance *tau_i, a payload of *bits bits (chunk
 * padding included) and an index of *index_bytes bytes.  Any output may be NULL.
 */
pc_status pc_stream_info(const pc_streams *s, int i, double *tau_i, uint64_t *bits, uint64_t *index_bytes);

/*
 * Field shape and component count of a pc_streams.  dims receives 3 extents
 * (1 beyond ndims).  Any output may be NULL.
 */
pc_status pc_streams_shape(const pc_streams *s, int *ndims, int64_t *dims, pc_dtype *dtype, int *n);

/*
 * Block-mode counters of component i (0-based) from pc_compress: counts[0] =
 * bricks coded ZERO, [1] = CODED, [2] = RAW, [3] = total escalation steps,
 * [4] = field values where Eq. 1 failed in floating point (Sec. 4.3).
 */
pc_status pc_stream_counts(const pc_streams *s, int i, uint64_t counts[5]);

/*
 * Serialization (checkpoint/restart use, Sec. 5.1.1): writes the header, the
 * tolerances and every component's index and payload into h_buf (host memory,
 * *len bytes).  With h_buf NULL only *len is set to the size needed.
 * Synchronises cuda_stream.
 */
pc_status pc_streams_serialize(const pc_streams *s, void *h_buf, size_t *len, void *cuda_stream);

/* Inverse of pc_streams_serialize: the data (host memory) is checked and copied
 * to the device.  PC_ERR_VERSION for another format, PC_ERR_CORRUPT_STREAM for
 * inconsistent sizes. */
pc_status pc_streams_deserialize(const void *h_buf, size_t len, void *cuda_stream, pc_streams **out);

/* Device pointers of component i's data (for users that move components
 * between memories themselves, Sec. 6.2): payload (u64 words), chunk word
 * offsets (u64 per 32 bricks) and brick bit lengths (u16 per brick).  They
 * stay valid until pc_streams_free, which does not wait for the caller's own
 * work on them. */
pc_status pc_stream_device_ptrs(const pc_streams *s, int i, const uint64_t **payload, const uint64_t **chunk_word,
                                const uint16_t **brick_len, uint64_t *payload_words, uint64_t *nchunks,
                                uint64_t *nbricks);

/* Copies component i's index to host memory: h_chunk_word receives nchunks
 * u64 (each chunk's first payload word), h_brick_len nbricks u16 (each brick's
 * bit length); either may be NULL.  Synchronises cuda_stream.  Together with
 * pc_stream_read this gives any single brick's bits (Sec. 6.1: blocks are
 * decodable one at a time). */
pc_status pc_stream_read_index(const pc_streams *s, int i, uint64_t *h_chunk_word, uint16_t *h_brick_len,
                               void *cuda_stream);

/* Copies nwords payload words of component i, starting at word word_off, to
 * host memory h_out.  PC_ERR_ARG if the range leaves the payload.
 * Synchronises cuda_stream. */
pc_status pc_stream_read(const pc_streams *s, int i, uint64_t word_off, uint64_t nwords, uint64_t *h_out,
                         void *cuda_stream);

/* Releases the streams and their device memory.  Waits for the library's
 * launches that read them (retrievals and refinements on any stream), not for
 * the rest of the device; work the caller launched on the arrays of
 * pc_stream_device_ptrs must have finished.  NULL is a no-op. */
void pc_streams_free(pc_streams *s);

/*
 * Returns the device memory the library keeps for later calls -- freed
 * streams and scratch in its pools, and the bit pool of the construction
 * kernel -- to the driver, on every device the library has used.  Waits for
 * each such device first.  Live pc_streams are untouched.  Not to be called
 * while another thread is inside a library call.
 */
pc_status pc_release_cached_memory(void);

/*
 * The range min/max of a field in device or pinned host memory (Sec. 5.1:
 * tau_0 is the range of the field values), reduced on cuda_stream; *vmin and
 * *vmax receive the extreme values as doubles.  Synchronises.
 * PC_ERR_NONFINITE if a value is not finite; PC_ERR_ARG for pageable memory.
 */
pc_status pc_field_range(const void *d_field, int64_t count, pc_dtype dtype, void *cuda_stream, double *vmin,
                         double *vmax);

/*
 * Tolerance schedules (Sec. 5.1: tolerances are relative to tau_0, the range
 * of the field values, and fall geometrically, tau_i = 2^(-Delta i) tau_0).
 *   PC_TAU_BINARY: tau_i = tau_0 * 2^(-param * i), i = 1..n, param = Delta >= 1
 *     (param * n <= 4096).  One rounding: exact unless the value is subnormal,
 *     and 0 once it falls below the smallest subnormal.
 *   PC_TAU_DECADE: tau_i = c_i * tau_0 rounded once, i = 1..n, with c_i the
 *     double nearest 10^-(param + i - 1), param >= 0 (param + n - 1 <= 400).
 * pc_tau_schedule writes tau[0..n-1] (host, n in 1..PC_MAX_COMPONENTS) from a
 * given tau_0 (positive, finite); pure host arithmetic, no GPU work.
 * pc_field_tau_schedule first reduces the field's range on the device (as
 * pc_field_range; device or pinned host memory, count values of dtype) and
 * takes tau_0 = max - min rounded once in double; PC_ERR_ARG for a constant
 * field (range 0) or a range that overflows.  It synchronises cuda_stream.
 * A schedule that underflows to 0 is returned as computed; pc_compress
 * rejects it with PC_ERR_TAU_ORDER.
 */
typedef enum { PC_TAU_BINARY = 1, PC_TAU_DECADE = 2 } pc_tau_kind;
pc_status pc_tau_schedule(pc_tau_kind kind, double tau0, int param, int n, double *tau);
pc_status pc_field_tau_schedule(const void *field, int64_t count, pc_dtype dtype, pc_tau_kind kind, int param, int n,
                                void *cuda_stream, double *tau);

/*
 * Lossless sweep (Sec. 5.1.3: components are added until x~ reproduces x).
 * Compresses the field (as pc_compress) with the binary schedule tau_i =
 * 2^(-delta i) tau_0, i = 1..n_max (1 <= delta <= 64, n_max <= 64), stopping
 * the schedule where it would underflow to 0; tau_0 is the field's range, or
 * max(|value|, 1) for a constant field.  *out receives the streams (free with
 * pc_streams_free), *k the first component whose computed tolerance
 * (pc_stream_measured_error) is 0, i.e. whose x~_k equals x value for value
 * (0 when none of them does), and *bits_per_value the stream bits of
 * components 1..k, payload and index, per field value (0 when *k is 0).
 * Errors as pc_compress.  Synchronises cuda_stream.
 */
pc_status pc_lossless_sweep(const void *field, const int64_t *dims, int ndims, pc_dtype dtype, int delta, int n_max,
                            void *cuda_stream, pc_streams **out, int *k, double *bits_per_value);

/*
 * Derivatives of (reconstructed) fields on a regular grid of spacing h: the
 * operators of the progressive use case (Sec. 5.3), where the vorticity
 * component v_x - u_y and the second derivative w_zz of a velocity field
 * magnify the reconstruction error like h^-1 and h^-2.  Second-order
 * differences at every point: central inside; at the two ends of the axis
 * ((4 f1 - 3 f0) - f2) / (2h) and ((3 f[n-1] - 4 f[n-2]) + f[n-3]) / (2h) for a
 * first derivative, (((2 f0 - 5 f1) + 4 f2) - f3) / h^2 and its mirror image
 * for a second.  Arithmetic in dtype, one rounding per operation in that
 * order, with h rounded to dtype first.
 *   pc_fd_vorticity_z: out = v_x - u_y.  u, v, out: device pointers to
 *     prod(dims) values of dtype, dims[0] = nx fastest; ndims 2 or 3; nx >= 3
 *     and ny >= 3.
 *   pc_fd_second: out = d2w/da2 along axis a (0 = x, 1 = y, 2 = z; a < ndims,
 *     ndims 1..3), at least 4 points along it.
 * out must not overlap an input.  h > 0 and finite.  Extents below 2^31 (ny
 * at most 524280).  PC_ERR_ARG otherwise.
 * Asynchronous on cuda_stream.
 */
pc_status pc_fd_vorticity_z(const void *u, const void *v, const int64_t *dims, int ndims, pc_dtype dtype, double h,
                            void *out, void *cuda_stream);
pc_status pc_fd_second(const void *w, const int64_t *dims, int ndims, pc_dtype dtype, int axis, double h, void *out,
                       void *cuda_stream);

/*
 * Kernel timing (instrumentation, off by default).  While enabled, every
 * kernel the library launches is bracketed by CUDA events recorded on the
 * stream it is launched on.  pc_timing_read synchronises the device and
 * returns, per kernel kind, the summed device time in milliseconds and the
 * number of launches since the last pc_timing_enable; kinds are indexed by
 * pc_kernel_kind.  ms and launches hold PC_KERNEL_KINDS entries each.
 */
typedef enum {
  PC_KERNEL_COMPRESS = 0, /* fused construction, Algorithm 1 */
  PC_KERNEL_SCAN = 1,     /* chunk offsets per component */
  PC_KERNEL_PACK = 2,     /* chunk copy into the streams */
  PC_KERNEL_RETRIEVE = 3, /* fused reconstruction, Algorithm 2 */
  PC_KERNEL_RANGE = 4,    /* field min/max */
  PC_KERNEL_FD = 5,       /* finite-difference derivatives */
  PC_KERNEL_KINDS = 6
} pc_kernel_kind;
pc_status pc_timing_enable(int on);
pc_status pc_timing_read(double *ms, uint64_t *launches);

/*
 * pc_compress without device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while
 * they run -- a host whose own allocator has already reserved the free device
 * memory (a framework's caching allocator, an application memory pool), or a
 * latency-critical loop that must avoid cudaMalloc/cudaFree, which can
 * synchronise the device.  It computes exactly what pc_compress computes
 * (the same streams as pc_compress, bit for bit) but takes all its temporary
 * memory from one fixed 64 MiB device array inside the library, held on every
 * GPU that loads the library until the process exits, and writes the streams
 * into buffers the caller provides:
 *   d_field     device pointer, 3D field of dtype (ndims must be 3).
 *   d_payload   device, payload_capacity_words u64 words; receives the
 *               components' payloads back to back (component i starts at word
 *               h_words[0] + ... + h_words[i-1]).
 *   d_chunk_word device, n * ceil(bricks / 32) u64: per component, each
 *               chunk's first word within that component's payload.
 *   d_brick_len device, n * bricks u16: each brick's bit length.
 *   h_words     host, n: payload words per component.
 *   h_counts    host, 5 * n: the counters of pc_stream_counts per component.
 * Limit: n * ceil(bricks / 32) must not exceed the bound given in the
 * PC_ERR_ARG message (2026 for one float64 component, 4042 for one float32
 * component, a little less for more components; e.g. a 64^3 field with up to
 * 15 float64 components); larger inputs are rejected before any GPU work, and
 * so is a too small payload buffer (its message gives the words needed).  The
 * four buffers must be device memory (PC_ERR_ARG otherwise); the index
 * buffers must hold the sizes stated above.  The library-internal array is shared by all
 * calls: calls whose work overlaps on the GPU (other streams or threads) race
 * on it, so the caller must serialise them.  The first call on a device looks
 * up the array's device address; make that first call before any stream
 * capture.  Synchronises cuda_stream.  Errors are reported by pc_last_error().
 */
pc_status pc_compress_noalloc(const void *d_field, const int64_t *dims, int ndims, pc_dtype dtype,
                              const double *tau, int n, uint64_t *d_payload, uint64_t payload_capacity_words,
                              uint64_t *d_chunk_word, uint16_t *d_brick_len, uint64_t *h_words,
                              uint64_t *h_counts, void *cuda_stream);

/*
 * Progressive-query server.  Serves queries (field, box, tolerance or k)
 * against component streams resident on the device, the way Sec. 6.1 and 6.2
 * describe progressive access: the components stay compressed, the blocks a
 * query needs are decoded on demand and added into x~, and more precision is
 * more components added to the current approximation.
 *
 * Per field the server keeps a cache of partial sums x~ and, per brick, the k
 * it holds.  A query at k starts a brick from the cache when the cached k is
 * at most k and decodes only the components above it; other bricks decode
 * from their first component.  The result is the same either way, bit for
 * bit: x~_k of pc_retrieve on the same box.  Bricks a query produced in full
 * at a k above their cached one are written back into the cache.
 *
 * Queries are batched continuously by a dispatcher thread of the server:
 * queries are admitted in submission order while their output boxes fit in
 * the arena (the part of hbm_budget_bytes left after the fields' streams,
 * their caches and the server's own buffers), and the admitted queries of one
 * dtype are launched as one batch -- one launch of the retrieval kernel over
 * all their boxes -- into a free slot.  Up to 4 slots (1 in PC_SERVE_SERIAL
 * mode) each have their own CUDA stream, so a batch admitted while others
 * run executes concurrently with them on the device.  A batch whose brick
 * region of a field overlaps that of an in-flight batch waits for it (the
 * cache reads and write-backs of a brick stay ordered); other batches do not
 * wait.  A host function queued behind every batch signals its completion:
 * no thread polls the GPU.
 *
 * The server reads the pc_streams objects given to it, which must stay alive
 * and unchanged until pc_server_free.  The first query (submit or replay)
 * starts the dispatcher; its batches run after the work queued on the
 * cuda_stream given at creation.  Only 3D fields are served.
 */
typedef struct pc_server pc_server; /* opaque */

#define PC_SERVE_NO_CACHE 1 /* decode every query from its first component, keep no cache */
#define PC_SERVE_SERIAL 2   /* one query per batch and one batch in flight: the unbatched pipeline */

typedef struct {
  int field;    /* index returned by pc_server_add_field */
  int k;        /* components to sum, 1..n; 0: the smallest k with tau_k <= tau */
  double tau;   /* absolute tolerance, used when k == 0 */
  pc_box box;   /* the box of the field to return (element units, half-open) */
} pc_query;

typedef struct {
  double wall_s;               /* from the start of the replay to the last completion */
  uint64_t batches;            /* retrieval launches */
  uint64_t queries;            /* queries served */
  uint64_t bytes_out;          /* result bytes produced */
  uint64_t max_batch;          /* most queries in one batch */
  uint64_t peak_device_bytes;  /* fields, caches, buffers and the arena's largest use */
  uint64_t arena_bytes;        /* size of the result arena */
  uint64_t max_inflight;       /* most batches in flight at once */
} pc_serve_stats;

/* Creates a server.  max_batch (1..65535) bounds the queries of one batch;
 * flags is a combination of PC_SERVE_*.  PC_ERR_OOM if the budget cannot hold
 * the server's own buffers. */
pc_status pc_server_create(uint64_t hbm_budget_bytes, int max_batch, int flags, void *cuda_stream,
                           pc_server **out);

/* Registers a 3D stream set; *field receives its index.  Allocates its cache
 * (one value per field element and 5 bytes per brick) unless
 * PC_SERVE_NO_CACHE.  PC_ERR_OOM if the streams and the cache exceed the
 * budget.  Fields are added before the first replay. */
pc_status pc_server_add_field(pc_server *srv, const pc_streams *s, int *field);

/* Runs nq queries as a recorded request stream through the same dispatcher:
 * query j is submitted arrival_s[j] seconds (non-decreasing) after the call
 * starts (the call sleeps between arrivals), and the call returns when all
 * are served.  latency_s[j] (host, nq doubles) receives the time from its arrival
 * to its batch's completion on the device (signalled to the host).  d_out, if not NULL, holds nq device
 * pointers (NULL entries allowed) that receive a copy of each result box (x
 * fastest, dtype of the field).  stats may be NULL.  Every query is checked
 * before any GPU work (PC_ERR_ARG, PC_ERR_TOL_UNREACHABLE, or PC_ERR_OOM for
 * a box larger than the arena).  Blocks the calling thread. */
pc_status pc_server_replay(pc_server *srv, const pc_query *queries, const double *arrival_s, int nq,
                           void *const *d_out, double *latency_s, pc_serve_stats *stats);

/* Online serving.  pc_server_submit queues one query (checked at once:
 * PC_ERR_ARG, PC_ERR_TOL_UNREACHABLE, or PC_ERR_OOM for a box larger than the
 * arena) and returns without waiting; *ticket identifies it.  d_out, if not
 * NULL, is a device buffer that receives a copy of the result box (x fastest,
 * dtype of the field) before the query counts as done.  Its arrival time is
 * the moment of the call.  pc_server_poll reports without blocking whether
 * the query is done (*done 1) and then its latency, from submission to the
 * moment its batch completed on the device (*latency_s, seconds, may be
 * NULL).  pc_server_wait blocks until the query is done or timeout_s seconds
 * have passed (timeout_s < 0: no limit) and reports the same.  A CUDA failure
 * of a batch is reported by the calls that ask about it.  Thread-safe: any
 * thread may submit, poll and wait. */
pc_status pc_server_submit(pc_server *srv, const pc_query *query, void *d_out, uint64_t *ticket);
pc_status pc_server_poll(pc_server *srv, uint64_t ticket, int *done, double *latency_s);
pc_status pc_server_wait(pc_server *srv, uint64_t ticket, double timeout_s, int *done, double *latency_s);

/* Counters since the server was created (wall_s: since the first query). */
pc_status pc_server_stats(pc_server *srv, pc_serve_stats *stats);

/* Forgets every cached partial sum (waits until no batch is queued or running). */
pc_status pc_server_reset_cache(pc_server *srv);

/* Releases the server and its device memory (not the streams).  NULL is a no-op. */
pc_status pc_server_free(pc_server *srv);

/*
 * Batched construction (Algorithm 1 over many fields at once).  A plan fixes
 * the fields' shapes, the type and the number of components; each
 * pc_batch_compress call then codes one set of fields of those shapes (new
 * values and tolerances) in one persistent kernel launch over all the
 * fields' chunks -- 3D chunks by whole CTAs of 16 warps in one kernel and,
 * on a parallel branch, 1D/2D chunks by single warps in a second one, or
 * both in one kernel --
 * followed by one segmented scan (per field and component) and one packing
 * launch.  The launches up to the scan are captured in CUDA graphs when the
 * plan is created (one per kernel shape) and replayed on every call.  On the
 * plan's first call an autotuner times a fixed set of 16 schedules on that
 * batch and keeps the fastest (pc_batch_info): CTAs of 16 warps per SM for
 * the 3D kernel (1 at up to 128 registers per thread, or 2 at 64), warps per
 * CTA of the 1D/2D kernel (2 to 16), chunks per warp in a 1D/2D work item
 * (1 or 2), items per claim (1 or 2), or instead one kernel of 16-warp CTAs
 * that takes the items of both parts from one queue.  For float64 the
 * schedules with 16-warp 1D/2D CTAs and the single kernel are left out (their
 * 128 registers per thread are too few for a 2D float64 brick).  The result
 * of every call is exactly what pc_compress gives for each field on its own,
 * bit for bit.
 *
 *   pc_batch_create: nfields >= 1; dims: 3 extents per field (x first,
 *     entries beyond the field's ndims ignored); ndims: 1..3 per field; n
 *     components for every field.  The plan runs on a stream of its own and
 *     each call first waits for the work queued on cuda_stream.
 *   pc_batch_compress: d_fields: nfields device pointers (dense, x fastest);
 *     tau: n tolerances per field, field after field; out: nfields
 *     pc_streams* (freed one by one with pc_streams_free; the batch's
 *     device arrays are released with the last of them).  Errors as
 *     pc_compress (PC_ERR_TAU_ORDER, PC_ERR_NONFINITE, ...).  Synchronises
 *     the plan's stream.
 */
typedef struct pc_batch pc_batch; /* opaque */

typedef struct {
  int schedule;          /* index of the chosen schedule, -1 before the first call */
  int order;             /* 0: fields in the given order, 1: largest first */
  int chunks_per_item;   /* chunks of a 1D/2D field per work item */
  int items_per_claim;   /* work items a CTA claims per atomic */
  int candidates;        /* schedules timed by the autotuner */
  int grid;              /* persistent CTAs of the 3D kernel */
  int graph;             /* 1 when the launches run as a CUDA graph */
  int ctas_per_sm;       /* CTAs of 16 warps per SM of the 3D kernel variant (1 or 2) */
  int warps_small;       /* warps per CTA of the 1D/2D kernel (2, 4, 8 or 16) */
  int mixed;             /* 1 when one kernel codes both parts from one queue */
  uint64_t calls;        /* pc_batch_compress calls so far */
  double candidate_ms[16]; /* the autotuner's timings (ms); -1: not a schedule of this type */
} pc_batch_info_t;

pc_status pc_batch_create(int nfields, const int64_t *dims, const int *ndims, pc_dtype dtype, int n,
                          void *cuda_stream, pc_batch **out);
pc_status pc_batch_compress(pc_batch *b, const void *const *d_fields, const double *tau, pc_streams **out);
pc_status pc_batch_info(const pc_batch *b, pc_batch_info_t *info);
pc_status pc_batch_free(pc_batch *b);

/*
 * Batched retrieval (Algorithm 2 over many boxes at once): query q returns
 * x~_{k[q]} of streams s[q] on boxes[q] (NULL boxes: whole fields) into the
 * device buffer d_out[q] (box values, x fastest).  The queries of each type
 * and dimensionality run in one launch of the retrieval kernel over a list
 * of box jobs.  Same results as pc_retrieve per query.  Asynchronous on
 * cuda_stream.
 */
pc_status pc_retrieve_batch(int nq, const pc_streams *const *s, const int *k, const pc_box *boxes,
                            void *const *d_out, void *cuda_stream);

/*
 * Debug builds (libpcz_debug.so, compiled with PCZ_DEBUG) check every
 * shared-memory bit write of the coders and every plane slot and spill index
 * of the retrieval against its buffer; a failed check skips the access and
 * sets a bit of a check word instead of faulting.  *word receives the check
 * bits seen since the last reset (bit 0: 3D chunk buffer, 1: 3D plane tables,
 * 2: 1D/2D chunk buffer, 3: retrieval plane slots), *enabled (may be NULL) 1
 * in a debug build and 0 in a release build, where *word is always 0 and no
 * device call is made.  reset != 0 clears the word.
 */
pc_status pc_debug_status(uint32_t *word, int *enabled, int reset);

/* Message for the last failed call on this thread ("" if none). */
const char *pc_last_error(void);

/* Library format version (of serialized streams) and build information. */
int pc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PCZ_H */

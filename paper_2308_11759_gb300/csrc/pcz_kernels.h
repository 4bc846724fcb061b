// pcz_kernels.h -- parameter blocks and launchers shared between the C-ABI
// host code (pcz_api.cu) and the kernels.  Internal to libpcz.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pcz {

constexpr int kMaxComponents = 64;
constexpr int kChunk = 32;  // bricks per index chunk (R15)

// Launch parameters of the fused construction kernel (Algorithm 1 over every
// brick of a field, all components in one pass).
struct CompressParams {
  const void* field;             // device, prod(dims) values of T
  int64_t dims[3];               // extents, x fastest (1 beyond ndims)
  int64_t nb[3];                 // bricks per axis
  int64_t nbricks, nchunks;
  int n;                         // components
  uint64_t tau_bits[kMaxComponents];  // bit pattern of the largest T not above tau_i
  int L[kMaxComponents];              // floor(log2(tau_i))
  uint64_t* pool;                // scratch for the chunks' bits, pool_words u64 words
  uint64_t pool_words;
  unsigned long long* pool_used; // bump counter (words)
  uint32_t* chunk_nwords;        // [n][nchunks] u64 words of each chunk
  uint64_t* chunk_pool;          // [n][nchunks] word offset of each chunk in the pool
  uint16_t* brick_len;           // [n][nbricks] bits of each brick
  uint32_t* brick_off;           // [n][nbricks] first bit of each brick within its chunk (may be null)
  uint32_t* chunk_counts;        // [n][nchunks][5] ZERO, CODED, RAW, escalations, Eq. 1 failures
  uint64_t* chunk_maxerr;        // [n][nchunks] bits of max |fl(x - x~_i)| over the chunk (may be null)
  unsigned int* flags;           // bit 0 non-finite input, bit 1 pool too small
};

// One component's stream as the retrieval kernel sees it.
struct CompDesc {
  const uint64_t* payload;
  uint64_t nwords;
  const uint64_t* chunk_word;    // [nchunks] first payload word of each chunk
  const uint16_t* brick_len;     // [nbricks]
  const uint32_t* brick_off;     // [nbricks] first bit of each brick within its chunk
  int L;                         // floor(log2(tau_i))
  int pad_;
};

// One box of one field for the retrieval kernel (Algorithm 2 on the bricks
// that meet the box, components k0+1..k).  A launch runs a list of jobs, each
// on its own units of bricks.
// Division of 32-bit unsigned n by an invariant d >= 1 with one high
// multiply (Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994): t = mulhi(m, n), n / d = (t + ((n - t) >> s1)) >> s2
// with l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, s1 = min(l, 1),
// s2 = max(l - 1, 0).  Exact for every n and d below 2^32.
struct DivMagic {
  uint32_t m;
  uint8_t s1, s2;
  uint16_t pad_;
};

struct BoxJob {
  const CompDesc* comp;          // device array of the field's n descriptors
  int64_t dims[3], nb[3];
  int64_t lo[3], hi[3];          // box, element units, half-open
  int64_t bl[3], bn[3];          // first brick and brick counts of the box
  int64_t nbox;                  // bricks meeting the box
  int64_t unit_begin;            // first unit of this job within the launch
  int k0, k;
  int umult;                     // a unit is 16 * umult bricks
  int pad_;
  DivMagic dv_bn0, dv_bn1;       // division by bn[0] and bn[1] (used when nbox < 2^32)
  DivMagic dv_ub;                // division by the bricks of a unit, 16 * umult
  int32_t pad2_[2];
  void* out;                     // box values of T (read too when k0 > 0)
  const void* cache;             // full-field cached partial sums of T, or null
  const uint8_t* level;          // per brick: k of the cached partial sum (0: none)
};

// Launch parameters of the retrieval kernel.
struct RetrieveParams {
  BoxJob job0;                   // the job when jobs is null
  const BoxJob* jobs;            // device array of njobs jobs sorted by unit_begin, or null
  int njobs;
  int write;                     // 0: parse and check only
  int64_t nunits;                // units over all jobs
  unsigned int* err;             // bit 0: a stream failed to parse
  uint64_t* spill;               // per-CTA plane words that do not fit in shared memory
  int grid;                      // CTAs launched (persistent over units)
  int pad_;
};

enum { kFlagNonFinite = 1u, kFlagPoolOverflow = 2u, kFlagStageTimeout = 4u };

// Batched construction: one persistent launch over the chunks of many
// fields.  The work list is implicit: slot s (schedule order) covers field
// slot_field[s], cut into items of slot_width[s] chunks (1 for a 3D field,
// whose chunk the whole CTA codes; more for 1D/2D fields, one warp per
// chunk); item g belongs to the slot s with slot_first[s] <= g <
// slot_first[s + 1].
struct BatchParams {
  const CompressParams* fields;  // device array, one per field
  const int32_t* slot_field;     // [nslots]
  const int32_t* slot_width;     // [nslots]
  const int32_t* slot_ndims;     // [nslots] dimensionality of the slot's field
  const int64_t* slot_first;     // [nslots + 1]
  int nslots;
  int per_fetch;                 // items a CTA claims per atomic
  int64_t nitems;
  unsigned long long* next;      // work counter (zeroed before the launch)
};

// Segmented scan of chunk word counts: segment s is entries
// [seg_start[s], seg_start[s] + seg_len[s]) of the chunk arrays.
struct ScanParams {
  const uint32_t* nwords;
  uint64_t* word_off;
  uint64_t* totals;              // [nseg]
  const uint32_t* chunk_counts;  // [entries][5]
  unsigned long long* counts;    // [nseg][5]
  const uint64_t* chunk_maxerr;
  unsigned long long* maxerr;    // [nseg]
  const int64_t* seg_start;
  const int64_t* seg_len;
  int nseg;
  int pad_;
};

// Launchers (each returns the launch error).
// device_field: the field is device memory (not host memory mapped into the
// device), so the 3D kernel may stage its bricks with TMA tile copies.
cudaError_t launch_compress(int dtype, int ndims, const CompressParams& p, cudaStream_t s, bool device_field = false);
cudaError_t launch_retrieve(int dtype, int ndims, const RetrieveParams& p, cudaStream_t s);
// 1D and 2D fields (one thread per brick); called by the two above.
cudaError_t launch_compress_small(int dtype, int ndims, const CompressParams& p, cudaStream_t s);
cudaError_t launch_retrieve_small(int dtype, int ndims, const RetrieveParams& p, cudaStream_t s);
cudaError_t launch_scan_chunks(const uint32_t* nwords, uint64_t* word_off, uint64_t* totals,
                               const uint32_t* chunk_counts, unsigned long long* counts,
                               const uint64_t* chunk_maxerr, unsigned long long* maxerr, int n,
                               int64_t nchunks, cudaStream_t s);
cudaError_t launch_pack(const uint64_t* pool, const uint32_t* nwords, const uint64_t* chunk_pool,
                        const uint64_t* word_off, const uint64_t* comp_base, uint64_t* payload, int n,
                        int64_t nchunks, cudaStream_t s);
// Batched construction: the 3D part (minb: CTAs of 16 warps per SM the
// kernel variant is built for, 1 or 2) and the 1D/2D part (warps per CTA: 2,
// 4, 8 or 16); the grids are the persistent CTAs that fit.
cudaError_t launch_compress_batch(int dtype, int minb, const BatchParams* d_bp, int grid, cudaStream_t s);
int compress_batch_grid(int dtype, int minb);
cudaError_t launch_compress_batch_small(int dtype, int warps, const BatchParams* d_bp, int grid, cudaStream_t s);
int compress_batch_small_grid(int dtype, int warps);
// Both parts in one kernel of 16-warp CTAs over one queue (persistent grid).
cudaError_t launch_compress_batch_mixed(int dtype, const BatchParams* d_bp, int grid, cudaStream_t s);
int compress_batch_mixed_grid(int dtype);
cudaError_t launch_scan_segments(const ScanParams* d_sp, int nseg, cudaStream_t s);
cudaError_t launch_pack_segments(const uint64_t* pool, const uint32_t* nwords, const uint64_t* chunk_pool,
                                 const uint64_t* word_off, const int64_t* seg_start, const uint64_t* seg_base,
                                 int nseg, int64_t nentries, uint64_t* payload, cudaStream_t s);
cudaError_t launch_brick_offsets(const uint16_t* brick_len, uint32_t* brick_off, int n, int64_t nbricks,
                                 cudaStream_t s);
cudaError_t launch_range(int dtype, const void* x, int64_t count, unsigned long long* enc, unsigned int* flags,
                         cudaStream_t s);

// Check words of the debug build's kernel translation units (always 0 in a
// release build); reset clears them.
uint32_t check_word_compress(int reset);
uint32_t check_word_small(int reset);
uint32_t check_word_retrieve(int reset);
uint32_t check_word_batch(int reset);

// Sets the message pc_last_error() returns on this thread.
void set_last_error(const char* msg);

// CTAs of a persistent retrieval launch over nunits units, brick pairs per
// warp of a unit for ncomp components, and the spill words a launch of grid
// CTAs needs.
int retrieve_grid(int dtype, int ndims, int64_t nunits);
int retrieve_unit_mult(int ncomp);
size_t retrieve_spill_words(int dtype, int ndims, int grid);

// Finite-difference derivatives (pcz_fd.cu): omega_z = v_x - u_y and the
// second derivative along one axis, over nx * ny * nz values.
cudaError_t launch_fd_vorticity_z(int dtype, const void* u, const void* v, void* out, int64_t nx, int64_t ny,
                                  int64_t nz, double h, cudaStream_t st);
cudaError_t launch_fd_second(int dtype, const void* w, void* out, int64_t nx, int64_t ny, int64_t nz, int axis,
                             double h, cudaStream_t st);

}  // namespace pcz

// pcz_host.h -- host-side pieces shared by the C-ABI translation units
// (pcz_api.cu, pcz_serve.cu): the component streams object and a few
// helpers.  Internal to libpcz.
#pragma once

#include <cstdint>
#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/pcz.h"
#include "pcz_kernels.h"

// The n component streams of one field, resident on the device, with the
// per-component metadata a query needs (tolerances, Sec. 6.2).
struct pc_streams {
  int device = 0;
  int ndims = 0;
  int64_t dims[3] = {1, 1, 1};
  int64_t nb[3] = {1, 1, 1};
  int64_t nbricks = 0, nchunks = 0;
  pc_dtype dtype = PC_F32;
  int n = 0;
  double tau[pcz::kMaxComponents] = {};
  int L[pcz::kMaxComponents] = {};
  uint64_t words[pcz::kMaxComponents] = {};      // payload words per component
  uint64_t word_base[pcz::kMaxComponents] = {};  // component's first word in d_payload
  uint64_t counts[pcz::kMaxComponents][5] = {};
  double measured[pcz::kMaxComponents] = {};      // computed tolerance max |fl(x - x~_i)| (Sec. 4.3)
  uint64_t* d_payload = nullptr;     // all components back to back
  uint64_t* d_chunk_word = nullptr;  // [n][nchunks]
  uint16_t* d_brick_len = nullptr;   // [n][nbricks]
  uint32_t* d_brick_off = nullptr;   // [n][nbricks] derived: first bit of each brick in its chunk
  pcz::CompDesc* d_desc = nullptr;   // [n]
  unsigned int* d_err = nullptr;
  void* d_index = nullptr;           // the allocation holding chunk words .. d_err (none for a batch's streams)
  std::shared_ptr<void> backing;     // set when the device arrays live in arenas shared by a batch
  // The library's launches that read the arrays: per stream an event recorded
  // behind the latest one.  pc_streams_free waits for these, not for the
  // whole device.  sync_device: an event could not be made, so it waits for
  // the device instead.
  mutable std::mutex use_mu;
  mutable std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;
  mutable bool sync_device = false;
};

namespace pcz {

// An NVTX range over one C-ABI call, for timeline tools (nsys, ncu's range
// filters); free when no tool is attached.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Records msg for pc_last_error() and returns st.
pc_status api_fail(pc_status st, const std::string& msg);
// Maps a CUDA error to PC_ERR_OOM / PC_ERR_CUDA (clearing a sticky launch error).
pc_status api_cuda_fail(cudaError_t e, const char* what);
size_t dtype_size(pc_dtype t);
// Box of a query in element units (whole field when box is null); PC_ERR_ARG
// when it is empty or leaves the field.
pc_status check_box(const pc_streams* s, const pc_box* box, int64_t lo[3], int64_t hi[3]);
// Retrieval job over a box (components k0+1..k into out); unit_begin = 0.
BoxJob make_box_job(const pc_streams* s, int k0, int k, const int64_t lo[3], const int64_t hi[3], void* out);
int64_t box_job_units(const BoxJob& J);
// Exact double of a T bit pattern.
double value_of_bits(uint64_t b, pc_dtype dt);
// floor(log2 tau) and the bit pattern of the largest T not above tau.
int floor_log2_of(double tau);
uint64_t tau_bits_of(double tau, pc_dtype dt);
bool tolerances_valid(const double* tau, int n);
void field_geometry(int ndims, const int64_t* dims, int64_t d3[3], int64_t nb[3], int64_t* nbricks,
                    int64_t* nchunks);
bool device_pointer(const void* p);
// Stream-ordered scratch from the library's own memory pool (freed with
// cudaFreeAsync on a stream).
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t st);
// Records that work just queued on st reads the arrays of s.
void note_use(const pc_streams* s, cudaStream_t st);

}  // namespace pcz

// Host-side plan object and the helpers shared by the ABI, batching, tuning and serving code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <vector>

#include "motif_internal.h"

struct motif_plan_s {
  // problem (Sec. I.A: n sequences of length t; pattern length l; d allowed mismatches)
  int n = 0, t = 0, l = 0, d = 0;
  int W = 0;                 // windows per sequence, t - l + 1 (may be <= 0)
  int wstride = 0;           // padded windows per row
  motif_opts opts{};
  cudaStream_t stream = nullptr;
  int device = 0, sms = 0;

  // kernel configuration
  int kind = MOTIF_KERNEL_GROUP;
  int p = 4;                 // candidates per lane (CAND) or suffix bases ks (GROUP)
  int span0 = 2;
  bool tiled = false;        // GROUP k=4 fresh passes use the prefix-tiled form
  bool tiled_in_batch = false;  // ... and inside a batch (where few, long tiles run side by side)
  int seq_block = 0;         // tiled with bitmap output: sequences per (tile, block) item; 0 = none
  int lkind = 0;             // step kernel variant of a single search (launch_kind of kind, p)
  int block = 256, grid = 0;
  size_t smem = 0;
  uint64_t lo = 0, hi = 0;   // candidate range
  uint64_t unit_lo = 0, unit_hi = 0, chunk_units = 0, nchunks = 0, rest_threshold = 0;

  // device memory owned by the plan
  char* d_chars = nullptr;
  size_t chars_bytes = 0;
  uint2* d_planes = nullptr;
  uint64_t* d_codes = nullptr;
  int* d_err = nullptr;
  uint32_t* d_qidx[2] = {nullptr, nullptr};
  uint64_t* d_qmask[2] = {nullptr, nullptr};
  uint64_t qcap = 0;
  int qmask_words = 0;
  uint64_t want_qcap = 0;    // queue size of the current configuration (allocated lazily)
  int want_qwords = 0;
  uint64_t* d_out = nullptr;
  int64_t out_cap = 0;
  void* d_sort = nullptr;
  size_t sort_bytes = 0;
  // Bitmap output (MOTIF_OUTPUT_BITMAP): one bit per code of [bm_base, bm_base + 32*bm_words),
  // and the compaction's block counts.
  bool bitmap = false;
  uint64_t bm_base = 0, bm_words = 0;
  uint32_t* d_bitmap = nullptr;
  unsigned* d_bm_scratch = nullptr;
  uint64_t bm_alloc_words = 0;
  motif::JobDesc* d_job = nullptr;
  motif::JobState* d_state = nullptr;
  motif::StepCtl* d_ctl = nullptr;
  unsigned long long* d_total = nullptr;
  int64_t device_bytes = 0;

  // CUDA graphs: init + while(step) for the uploaded descriptor, and the device-path sort.
  cudaGraphExec_t g_steps = nullptr;
  cudaGraphExec_t g_sort = nullptr;
  motif::JobDesc* h_desc = nullptr;  // pinned copy of the uploaded descriptor
  // Host staging: the characters of a small host load (validated while they are copied in, so
  // the load need not wait for the device), and, pinned, the final count plus the first codes of
  // a blocking search (read back with one wait).
  char* h_chars = nullptr;
  cudaEvent_t h_chars_done = nullptr;  // recorded after the staged characters' upload
  uint64_t* h_res = nullptr;           // [1 + kResultPeek]
  uint64_t* desc_out = nullptr;      // output buffer named by the uploaded descriptor
  int64_t desc_cap = -1;
  uint64_t* gs_out = nullptr;        // buffers the sort graph was built for
  int64_t gs_cap = -1;
  void* gs_scratch = nullptr;
  int64_t graph_searches = 0;        // graph launches since the last fold (launch accounting)
  unsigned last_steps = 0;           // steps of the last folded search

  // Candidates seeded by the d-neighbourhoods of the first sequence's windows
  // (MOTIF_SEED_NEIGHBOURHOOD): the difference patterns, the seed bitmap over
  // [seed_base, seed_base + 32*seed_words) and its count scratch.
  bool seeded = false;
  uint64_t npat = 0;
  uint64_t* d_pat = nullptr;
  uint32_t* d_seed = nullptr;
  unsigned* d_seed_scratch = nullptr;
  unsigned long long* d_seed_count = nullptr;
  uint64_t seed_base = 0, seed_words = 0, seed_alloc_words = 0, pat_alloc = 0;

  // Ragged / masked input (motif_load_seqs_var): per-row lengths and window counts, window
  // flags, and whether some row has no valid window (then nothing can be accepted).
  bool ragged = false;
  bool empty_row = false;
  int32_t* d_lens = nullptr;
  int32_t* d_wrow = nullptr;
  uint8_t* d_valid = nullptr;
  int* d_empty = nullptr;

  bool loaded = false;
  bool check_alpha = false;  // device-loaded characters not yet validated on the host
  motif_stats_t stats{};
  // Four events per search (steps begin/end, sort begin/end), folded into the statistics by
  // motif_stats; `evq_used` quads are pending.
  std::vector<cudaEvent_t> evq;
  size_t evq_used = 0;
  double sum_search_ms = 0, sum_sort_ms = 0;
  int64_t sum_searches = 0;
};

namespace motif {

// The library's stream-ordered memory pool of a device (made on first use): freed blocks up to
// kPoolKeepBytes stay in it between synchronisations instead of going back to the driver, so
// the many small buffers of short-lived plans and served jobs come back without a new mapping.
constexpr uint64_t kPoolKeepBytes = (uint64_t)256 << 20;
cudaMemPool_t device_pool(int device);
// Stream-ordered device memory from that pool (freed with cudaFreeAsync); null on failure.
void* pool_alloc(int device, size_t bytes, cudaStream_t s);
// Device memory through the plan's allocator (or the device's pool, stream-ordered).
void* plan_alloc(motif_plan_s* p, size_t bytes);
void plan_free(motif_plan_s* p, void* ptr, size_t bytes);

// Ball table of ks on the plan's device (built once per device and ks).
const uint64_t* ball_table(int device, int ks, cudaStream_t s);

// Fills the device descriptor of the plan's job (host copy).
void fill_desc(const motif_plan_s* p, JobDesc* jd, uint64_t* out, uint64_t out_cap);

// (Re)applies the kernel configuration: variant, grid, shared memory and chunking.
int plan_configure(motif_plan_s* p);
// The host part of plan creation: arguments, options, range, window stride, device and SM
// count checked and set (no device memory).  A motif_status.
int plan_init_host(motif_plan_s* p, int32_t n, int32_t t, int32_t l, int32_t d,
                   const motif_opts* opts);
// The tuning cache's choice (kernel AUTO) and plan_configure.
int plan_configure_host(motif_plan_s* p);
// Allocates the survivor queues and the default output buffer on first use.
int plan_ensure_buffers(motif_plan_s* p);
void free_bitmap(motif_plan_s* p);
void free_seed(motif_plan_s* p);
// Builds the seed bitmap of a seeded plan for its loaded sequences (on stream s).
int prepare_seed(motif_plan_s* p, cudaStream_t s);
// Drops the plan's cached graphs and descriptor upload (after a configuration change).
void invalidate_graphs(motif_plan_s* p);

// Launches steps for a job table until no job is active (polling every `group` steps), or
// blindly `max_steps` steps when poll == false.  Returns a motif_status.
int run_steps(int kind, int pv, const JobDesc* d_jobs, JobState* d_states, int njobs,
              StepCtl* d_ctl, int grid, int block, size_t smem, int max_steps, bool poll,
              int timeout_ms, cudaStream_t s, int* steps_run);

int status_from_cuda(cudaError_t e);

// Next free event quad of the plan (grown on demand); nullptr on failure.
cudaEvent_t* next_event_quad(motif_plan_s* p);
// Waits for the plan's stream and folds pending event quads into the statistics.
int fold_event_quads(motif_plan_s* p);

// Copies a cached tuning choice for the plan's shape into *o; false when none is cached.
bool tune_lookup(const motif_plan_s* p, motif_opts* o);

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

inline double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace motif

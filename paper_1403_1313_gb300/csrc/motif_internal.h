// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/motif.h"

namespace motif {

constexpr int kMaxL = 31;            // 4^l must fit in 64 bits
constexpr int kWinAlign = 8;         // window rows padded to a multiple of 8 (four 128-bit loads)
constexpr int kMaxKs = 4;            // GROUP kernel: at most 4 suffix bases (256-bit masks)
constexpr int kPassNone = -1;

// CAND and BITSLICE plans share their units (one candidate each), chunks and queues.
inline bool cand_like(int kind) {
  return kind == MOTIF_KERNEL_CAND || kind == MOTIF_KERNEL_BITSLICE;
}

// Per-job descriptor, written by the host before a job's first step and read-only on the device.
struct JobDesc {
  int32_t n, t, l, d;
  int32_t W;                 // windows per sequence, t - l + 1 (> 0 for every device job)
  int32_t wstride;           // row stride of planes / codes in windows (multiple of kWinAlign)
  const uint2* planes;       // [n][wstride] compressed bit planes (E, O) of each window
  const uint64_t* codes;     // [n][wstride] packed 2l-bit code of each window
  int32_t kind;              // unit semantics: MOTIF_KERNEL_CAND (also for BITSLICE plans) or
                             // MOTIF_KERNEL_GROUP
  int32_t ks;                // GROUP: suffix bases per group (1..kMaxKs); CAND: 0
  int32_t cpt;               // CAND: candidates per lane in a fresh pass (1, 2 or 4)
  int32_t span0;             // sequences a fresh pass scans before the first compaction
  int32_t tiled;             // GROUP k=4: fresh passes use the prefix-tiled form (see search.cu)
  int32_t seq_block;         // tiled with bitmap output: 0 = a work item is one tile walked
                             //   through every sequence (with the skip); k > 0 = a work item is
                             //   (tile, block of k sequences), whose survivors are ANDed into
                             //   the bitmap (which then starts as all ones)
  uint64_t lo, hi;           // candidate range [lo, hi)
  uint64_t unit_lo, unit_hi; // work units of the range: candidates (CAND) or groups (GROUP)
  uint64_t chunk_units;      // units per chunk (bounds the queues)
  uint64_t nchunks;
  uint64_t rest_threshold;   // a queue pass with <= this many entries finishes every sequence
  uint32_t* qidx[2];         // ping-pong survivor queues: unit offset within the chunk
  uint64_t* qmask[2];        // GROUP: alive masks, mask_words(ks) words per entry
  uint64_t qcap;             // entries per queue (>= chunk_units)
  uint64_t* out;             // accepted codes, appended
  uint64_t out_cap;
  const uint64_t* ball;      // GROUP: Hamming-ball table for ks (see ball_table_words)
  unsigned long long* units; // counting launches (kKindTiledCount): kTiledUnits counters
  uint32_t* bitmap;          // non-null: accepted codes set bit (code - bm_base) here instead of
  uint64_t bm_base;          //   being appended to out (bm_base is a multiple of 64)
  const uint8_t* valid;      // ragged / masked rows: [n][wstride] window flags (null = all valid);
  const int32_t* wrow;       //   per-row window counts (null = W); read by the tally kernel only
  const uint32_t* seed;      // non-null: only candidates whose bit (code - seed_base) is set are
  uint64_t seed_base;        //   searched, from the second sequence on (fresh CAND passes)
};

// Per-job device state, advanced by the last CTA of every step.
struct JobState {
  unsigned long long cursor;     // next work item of the current pass
  unsigned long long qcount[2];  // entries in each queue
  unsigned long long out_count;  // accepted codes (may exceed out_cap)
  unsigned long long chunk;      // current chunk
  int32_t pass_seq;              // first sequence of the current pass (0 = fresh chunk)
  int32_t qsel;                  // input queue of a queue pass
  int32_t done;
  int32_t error;
  unsigned long long steps;      // steps in which the job had work
  unsigned long long pad[2];
};

// Step control block (one per launch sequence).
struct StepCtl {
  unsigned int ctas_done;        // CTAs finished in the current step
  unsigned int tiles_per_warp;   // 0 = unlimited; else each warp grabs at most this many tiles
  unsigned int active_jobs;      // written by the last CTA: jobs not yet done
  unsigned int steps;            // steps executed
  unsigned int max_steps;        // graph while-loops stop after this many steps (0 = no bound)
  unsigned int rotate;           // != 0: CTA b starts its walk over the jobs at job b % njobs
};

__host__ __device__ inline int mask_words(int ks) { return ks <= 3 ? 1 : (1 << (2 * ks - 6)); }
// Ball table for ks: for every suffix value v in [0, 4^ks) and radius r in [0, ks], the
// 4^ks-bit mask of suffixes within Hamming distance r of v; mask_words(ks) words per entry.
__host__ __device__ inline int ball_table_words(int ks) {
  return (1 << (2 * ks)) * (ks + 1) * mask_words(ks);
}

// Process-wide count of kernel launches issued by the library.
void note_launches(int n);
unsigned long long launches_total();

// ---- launchers (stream-ordered, no host synchronisation) ---------------------------------
// Ragged rows (lens[s] characters each), optionally masking windows with characters outside
// ACGTacgt; *d_err is set on such a character when mask_unknown is 0, *d_empty when some row has
// no valid window.  Invalid positions are filled with copies of valid windows of their row.
cudaError_t launch_pack_var(const char* d_chars, int64_t stride, int n, int l, int wstride,
                            const int32_t* d_lens, int mask_unknown, uint2* planes,
                            uint64_t* codes, uint8_t* valid, int* d_err, int* d_empty,
                            cudaStream_t s);
// Packs n rows of t characters into window planes and codes; with d_err, a character outside
// ACGTacgt sets *d_err (checked while packing, or alone when t < l); d_err null: no check.
cudaError_t launch_pack(const char* d_chars, int64_t stride, int n, int t, int l, int wstride,
                        uint2* planes, uint64_t* codes, int* d_err, cudaStream_t s);
// Fills the Hamming-ball table for ks (ball_table_words(ks) words).
cudaError_t launch_ball_table(uint64_t* table, int ks, cudaStream_t s);
// Step kernel variants: kind = MOTIF_KERNEL_CAND or MOTIF_KERNEL_BITSLICE with p = candidates
// per lane (1, 2, 4), MOTIF_KERNEL_GROUP with p = ks (1..4), or kKindTiledSplit with p = 4.
// Every job of one launch must use the same variant.
//
// kKindTiledSplit is a launch-only kind: the GROUP k = 4 kernel that also runs tiled passes split
// into (tile, sequence block) items (JobDesc::seq_block > 0).  Its jobs' descriptors keep
// MOTIF_KERNEL_GROUP; launches that hold no split job use the plain GROUP kernel, whose
// whole-tile loop compiles without the split's code.
constexpr int kKindTiledSplit = MOTIF_KERNEL_BITSLICE + 1;
// kKindTiled (p = 4) is the launch-only kind of the kernel whose only pass is the whole-tile
// prefix-tiled pass; a launch uses it when every job of its table runs that pass
// (JobDesc::tiled, JobDesc::seq_block == 0).
constexpr int kKindTiled = kKindTiledSplit + 1;
// kKindTiledCount (p = 4): the same kernel also adding the tiled pass's unit counts to
// JobDesc::units (motif_count_tiled_work only).
constexpr int kKindTiledCount = kKindTiledSplit + 2;
constexpr int kLaunchKinds = kKindTiledCount + 1;
// Unit counts of the whole-tile tiled pass (JobDesc::units, motif_count_tiled_work), in order:
// tile-sequence visits, windows filtered (W per visit), map marks (windows at tile-prefix
// distance d), listed windows (distance below d), scan rounds (live warps x ceil(listed / 32)),
// warp hit iterations (per scan round the largest hit count of a live lane of the warp), lane hits.
constexpr int kTiledUnits = 7;
// The step kernel variant of a launch: `split` when a job of the table is split into sequence
// blocks, `all_tiled` when every job of the table runs the tiled pass.
inline int launch_kind(int kind, int p, bool split, bool all_tiled = false) {
  if (kind != MOTIF_KERNEL_GROUP || p != 4) return kind;
  if (split) return kKindTiledSplit;
  return all_tiled ? kKindTiled : kind;
}
// Dynamic shared memory of a step kernel variant: kind is a unit kind (MOTIF_KERNEL_*) or a
// launch-only kind (kKindTiledSplit, kKindTiled).
size_t step_smem_bytes(int kind, int p, int wstride, int block);
cudaError_t step_kernel_attrs(int kind, int p, size_t smem);
int step_max_ctas_per_sm(int kind, int p, int block, size_t smem);
cudaError_t launch_step(int kind, int p, const JobDesc* d_jobs, JobState* d_states, int njobs,
                        StepCtl* d_ctl, int grid, int block, size_t smem, cudaStream_t s);
// Adds a step-kernel node to graph g.  With use_cond != 0 the kernel sets `cond`, the
// condition of the while node whose body g is, to continue while jobs remain.
cudaError_t add_step_node(cudaGraph_t g, int kind, int p, const JobDesc* d_jobs,
                          JobState* d_states, int njobs, StepCtl* d_ctl, int grid, int block,
                          size_t smem, cudaGraphConditionalHandle cond, int use_cond,
                          cudaGraphNode_t* node);
// Zeroes njobs states and initialises the step control block.
cudaError_t launch_init_steps(JobState* d_states, int njobs, StepCtl* d_ctl, unsigned max_steps,
                              unsigned tiles_per_warp, unsigned rotate, cudaStream_t s);
cudaError_t add_init_node(cudaGraph_t g, JobState* d_states, int njobs, StepCtl* d_ctl,
                          unsigned max_steps, unsigned tiles_per_warp, unsigned rotate,
                          cudaGraphNode_t* node);
// Builds and instantiates init -> while(step) over a job table: one launch runs every step.
// rotate != 0 spreads the CTAs' starting jobs (batches); 0 keeps table (arrival) order.
// one_step: init -> step, for tables whose every job finishes in one step (one tiled pass over
// a single chunk, with no tile budget per step).
cudaError_t build_step_graph(int kind, int p, const JobDesc* d_jobs, JobState* d_states,
                             int njobs, StepCtl* d_ctl, int grid, int block, size_t smem,
                             unsigned max_steps, unsigned rotate, cudaGraphExec_t* exec,
                             bool one_step = false);
cudaError_t launch_count(const JobDesc* d_job, unsigned long long* d_total, int grid, int block,
                         cudaStream_t s);
// Canonical (group, window) prefix-compare tally of the GROUP formulation with ks suffix bases.
cudaError_t launch_count_group(const JobDesc* d_job, int ks, unsigned long long* d_total, int grid,
                               int block, cudaStream_t s);
// Sorts d_codes[0 .. *d_count) ascending and removes repeats in place (count updated) when
// *d_count <= cap.  known_count >= 0 lets the host skip the path that cannot apply.
size_t sort_scratch_bytes(int64_t cap, int sms);
// Bitmap output: writes the codes base + i of the set bits i of bm (nwords 32-bit words) to out
// in ascending order (at most cap of them) and their number to *count.  scratch holds
// bitmap_scratch_words(nwords) words.
uint64_t bitmap_scratch_words(uint64_t nwords);
// Number of set bits of bm (nwords words) into *count (the first two kernels of the compaction).
cudaError_t launch_bitmap_count(const uint32_t* bm, uint64_t nwords, unsigned* scratch,
                                unsigned long long* count, cudaStream_t s);
// Sets bit (c - base) of `seed` for every code c = codes0[j] ^ pat[r] (j < W, r < npat) that
// lies in [lo, hi): the candidates within d of a window of the first sequence.
cudaError_t launch_seed_scatter(const uint64_t* codes0, int W, const uint64_t* pat,
                                uint64_t npat, uint64_t lo, uint64_t hi, uint32_t* seed,
                                uint64_t base, cudaStream_t s);
cudaError_t launch_bitmap_compact(const uint32_t* bm, uint64_t nwords, uint64_t base,
                                  uint64_t* out, int64_t cap, unsigned* scratch,
                                  unsigned long long* count, cudaStream_t s);
// Many jobs at once (batches).  A SortTask sorts codes[0 .. *count) in place when
// 1 < *count <= min(4096, cap) (one CTA per task; larger lists take launch_sort_unique).
struct SortTask {
  uint64_t* codes;
  unsigned long long* count;
  long long cap;
};
cudaError_t launch_small_sort_tasks(const SortTask* d_tasks, int ntasks, cudaStream_t s);
// A BitmapTask compacts one bitmap as launch_bitmap_compact does; the tasks' blocks form one grid:
// task k owns blocks [d_first[k], d_first[k+1]), bitmap_task_blocks(nwords) of them, and its
// scratch holds at least that many words.
struct BitmapTask {
  const uint32_t* bm;
  uint64_t nwords;
  uint64_t base;
  uint64_t* out;
  long long cap;
  unsigned* scratch;
  unsigned long long* count;
};
uint64_t bitmap_task_blocks(uint64_t nwords);
cudaError_t launch_bitmap_compact_tasks(const BitmapTask* d_tasks, const unsigned* d_first,
                                        int ntasks, unsigned total_blocks, cudaStream_t s);
cudaError_t launch_sort_unique(uint64_t* d_codes, unsigned long long* d_count, int64_t cap,
                               int key_bits, void* scratch, int sms, long long known_count,
                               cudaStream_t s);
// Graph form of launch_sort_unique (the multi-CTA path under a conditional IF node).
cudaError_t add_sort_nodes(cudaGraph_t g, cudaGraphNode_t dep, uint64_t* d_codes,
                           unsigned long long* d_count, int64_t cap, int key_bits, void* scratch,
                           int sms, cudaGraphNode_t* last);

}  // namespace motif

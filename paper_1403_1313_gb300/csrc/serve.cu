// Serving: continuous batching of motif-search jobs.
//
// Clients submit loaded plans; a scheduler thread owns one device job table.  Between device
// steps it admits queued jobs (first come, first served) while table slots and the device
// memory budget allow, launches one step of the multi-job step kernel (every active job advances
// by up to a bounded number of tiles, so new arrivals never wait behind a long job), reads back
// the job states, and retires finished jobs: their codes are sorted/de-duplicated on the device,
// copied to the host and handed to motif_poll.  A job's result does not depend on which other
// jobs shared its steps: each job only reads its own windows and writes its own queues/output.
#include <string.h>

#include <algorithm>
#include <array>
#include <condition_variable>
#include <deque>
#include <iterator>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "plan.h"

using namespace motif;

namespace motif_serve {

// Chunk of a served job's per-group passes (its survivor queues hold one chunk); a tiled job
// takes its whole range as one chunk, since the tiled pass uses no queues.
constexpr uint64_t kServeChunkGroups = 1ull << 20;
// How long a queued job of another kernel variant than the active table's may be passed over by
// later jobs before admission stops so that the table drains for it.
constexpr double kHeadWaitMs = 50.0;

struct Job {
  int64_t id = 0;
  int n = 0, t = 0, l = 0, d = 0, W = 0, wstride = 0;
  int kind = MOTIF_KERNEL_GROUP, pv = 4, span0 = 2, sms = 0;
  bool tiled = false;
  int seq_block = 0;  // tiled with bitmap output: sequences per (tile, block) item
  size_t smem = 0;
  uint64_t lo = 0, hi = 0, unit_lo = 0, unit_hi = 0, chunk_units = 0, nchunks = 0, rest = 0;
  uint2* planes = nullptr;    // one allocation: the planes, then the codes
  uint64_t* codes = nullptr;
  size_t win_bytes = 0;
  // Pinned staging of a job submitted from host rows: its characters, read by the pack kernel
  // on the submit stream; back to the pool when the job is released.
  uint64_t* stage = nullptr;
  size_t stage_cap = 0;
  uint32_t* qidx[2] = {nullptr, nullptr};
  uint64_t* qmask[2] = {nullptr, nullptr};
  uint64_t qcap = 0;
  int words = 0;
  uint64_t* out = nullptr;
  int64_t out_cap = 0;
  void* sort = nullptr;
  size_t sort_bytes = 0;
  // Bitmap output for dense results (the plan's choice): one bit per code of
  // [bm_base, bm_base + 32*bm_words), compacted in order when the job finishes.
  uint32_t* bitmap = nullptr;
  unsigned* bm_scratch = nullptr;
  uint64_t bm_base = 0, bm_words = 0;
  int64_t footprint = 0;
  const uint64_t* ball = nullptr;     // Hamming-ball table for pv on the server's device
  cudaEvent_t ready = nullptr;        // recorded after the window copies (submit stream)
  double t_submit = 0, t_admit = 0, t_done = 0, gpu_ms = 0;
  int status = MOTIF_OK;
  bool done = false;
  uint64_t* result = nullptr;  // the accepted codes, in a pinned block of the server's pool
  size_t result_cap = 0;       // codes the block holds
  int64_t result_size = 0;
};

struct Server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread th;
  bool running = false, stopping = false;
  motif_server_opts o{};
  int device = 0, sms = 0;
  cudaStream_t stream = nullptr;         // scheduler thread only
  cudaStream_t submit_stream = nullptr;  // client threads (window copies); guarded by submit_mu
  std::mutex submit_mu;
  std::deque<Job*> queue;
  std::vector<Job*> active;       // table order = admission order
  std::map<int64_t, Job*> jobs;   // every job not yet released by motif_poll
  int64_t next_id = 1;
  int64_t budget_used = 0;
  JobDesc* d_jobs = nullptr;
  JobState* d_states = nullptr;
  StepCtl* d_ctl = nullptr;
  int kind = -1, pv = -1, grid = 0, block = 256;
  size_t smem = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // Pinned host blocks for results, by capacity in codes (guarded by mu): a result is copied at
  // full link rate into pages that are already mapped, and motif_poll gives its block back.
  std::mutex pool_mu;  // guards host_free (taken by the scheduler, given back by motif_poll)
  std::multimap<size_t, uint64_t*> host_free;
  size_t host_free_bytes = 0;
  // Retirement of a step's finished jobs together (retire_finished): pinned staging of their
  // sort / compaction tasks and of the table's states, and the tasks' device copies.
  JobState* h_states = nullptr;
  // The table's upload: pinned descriptors and states, the step control, and the host's copy of
  // the device states as of the last step or upload (the jobs' states move with them when the
  // table is compacted, on the host, and go up with the next upload).
  JobDesc* h_jobs = nullptr;
  JobState* h_table = nullptr;
  StepCtl* h_ctl = nullptr;
  std::vector<JobState> mirror;
  // The retirement of a step's finished jobs runs on its own stream, during the next step: the
  // step's state snapshot (two, alternating) and the final counts read from it.
  cudaStream_t retire_stream = nullptr;
  JobState* d_snap[2] = {nullptr, nullptr};
  JobState* h_fin = nullptr;
  SortTask* h_sort_tasks = nullptr;
  BitmapTask* h_bm_tasks = nullptr;
  unsigned* h_bm_first = nullptr;
  SortTask* d_sort_tasks = nullptr;
  BitmapTask* d_bm_tasks = nullptr;
  unsigned* d_bm_first = nullptr;
};

constexpr size_t kHostPoolBytes = (size_t)2 << 30;  // pinned result blocks kept for reuse

// A pinned block for at least `n` codes.  Blocks come in powers of two of at least 1,024 codes;
// a pooled one of the request's size class, or the next one up, is reused, else a new block of
// the class is allocated.  Null when pinned memory is exhausted.
uint64_t* host_take(Server* S, size_t n, size_t* cap) {
  size_t c = 1024;
  while (c < n) c <<= 1;
  {
    std::lock_guard<std::mutex> g(S->pool_mu);
    auto it = S->host_free.lower_bound(c);
    if (it != S->host_free.end() && it->first <= 2 * c) {
      uint64_t* b = it->second;
      *cap = it->first;
      S->host_free_bytes -= it->first * 8;
      S->host_free.erase(it);
      return b;
    }
  }
  uint64_t* b = nullptr;
  if (cudaHostAlloc((void**)&b, c * 8, 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  *cap = c;
  return b;
}

// Returns a block to the pool.  Blocks that do not fit the pool's bound go to `evicted`, for the
// caller to free once it has released its locks: cudaFreeHost may wait for the device, which
// must not hold up the scheduler.
void host_give(Server* S, uint64_t* b, size_t cap, std::vector<uint64_t*>* evicted) {
  if (!b) return;
  std::lock_guard<std::mutex> g(S->pool_mu);
  if (cap * 8 > kHostPoolBytes) {
    evicted->push_back(b);
    return;
  }
  while (S->host_free_bytes + cap * 8 > kHostPoolBytes && !S->host_free.empty()) {
    auto big = std::prev(S->host_free.end());  // evict the largest pooled blocks first
    S->host_free_bytes -= big->first * 8;
    evicted->push_back(big->second);
    S->host_free.erase(big);
  }
  S->host_free.emplace(cap, b);
  S->host_free_bytes += cap * 8;
}

std::mutex g_life;  // guards g_srv creation / destruction
Server* g_srv = nullptr;

// Device memory in the order of stream s (the scheduler's stream by default); freed on the
// scheduler's stream once nothing uses it any more.
void* salloc_on(Server* S, size_t b, cudaStream_t s) {
  if (b == 0) return nullptr;
  return pool_alloc(S->device, b, s);
}
void* salloc(Server* S, size_t b) { return salloc_on(S, b, S->stream); }
void sfree(Server* S, void* p) {
  if (p) cudaFreeAsync(p, S->stream);
}

// Gives a job's character staging back to the pool.  (A block given back while the job's pack
// kernel may still read it only ever spoils the windows of that job, which is being discarded:
// every later user of the block packs on the same stream, after it.)
void release_stage(Server* S, Job* j) {
  if (!j->stage) return;
  std::vector<uint64_t*> evicted;
  host_give(S, j->stage, j->stage_cap, &evicted);
  for (uint64_t* b : evicted) cudaFreeHost(b);
  j->stage = nullptr;
}

void release_windows_from_client(Server* S, Job* j) {
  std::lock_guard<std::mutex> g(S->submit_mu);
  if (j->planes) cudaFreeAsync(j->planes, S->submit_stream);  // the codes share it
  j->planes = nullptr;
  j->codes = nullptr;
  if (j->ready) cudaEventDestroy(j->ready);
  j->ready = nullptr;
  release_stage(S, j);
}

// Queues, output and sort scratch: held only while the job is admitted.
void release_run_buffers(Server* S, Job* j) {
  for (int i = 0; i < 2; ++i) {
    sfree(S, j->qidx[i]);
    sfree(S, j->qmask[i]);
    j->qidx[i] = nullptr;
    j->qmask[i] = nullptr;
  }
  sfree(S, j->out);
  sfree(S, j->sort);
  sfree(S, j->bitmap);
  sfree(S, j->bm_scratch);
  j->out = nullptr;
  j->sort = nullptr;
  j->bitmap = nullptr;
  j->bm_scratch = nullptr;
}

// Everything, including the job's private window copies.
void release_buffers(Server* S, Job* j) {
  for (int i = 0; i < 2; ++i) {
    sfree(S, j->qidx[i]);
    sfree(S, j->qmask[i]);
    j->qidx[i] = nullptr;
    j->qmask[i] = nullptr;
  }
  sfree(S, j->out);
  sfree(S, j->sort);
  sfree(S, j->bitmap);
  sfree(S, j->bm_scratch);
  sfree(S, j->planes);  // the codes share it
  j->out = nullptr;
  j->sort = nullptr;
  j->bitmap = nullptr;
  j->bm_scratch = nullptr;
  j->planes = nullptr;
  j->codes = nullptr;
  if (j->ready) cudaEventDestroy(j->ready);
  j->ready = nullptr;
  release_stage(S, j);
}

int64_t footprint_of(const Job* j) {
  return (int64_t)(2 * j->qcap * (4 + 8 * (uint64_t)j->words) + 8 * (uint64_t)(1 << 16) +
                   4 * j->bm_words);
}

bool allocate_job(Server* S, Job* j) {
  for (int i = 0; i < 2; ++i) {
    j->qidx[i] = (uint32_t*)salloc(S, j->qcap * 4);
    j->qmask[i] = (uint64_t*)salloc(S, j->qcap * 8 * (uint64_t)j->words);
    if (!j->qidx[i] || !j->qmask[i]) return false;
  }
  j->out_cap = 1 << 16;
  j->out = (uint64_t*)salloc(S, (size_t)j->out_cap * 8);
  if (!j->out) return false;
  if (j->bm_words) {  // cleared on the scheduler's stream, before the job's first step
    j->bitmap = (uint32_t*)salloc(S, j->bm_words * 4);
    j->bm_scratch = (unsigned*)salloc(S, bitmap_scratch_words(j->bm_words) * 4);
    if (!j->bitmap || !j->bm_scratch) return false;
    // all ones where (tile, sequence block) items AND their survivors in
    if (cudaMemsetAsync(j->bitmap, j->seq_block > 0 ? 0xFF : 0, j->bm_words * 4, S->stream) !=
        cudaSuccess)
      return false;
  }
  return true;
}

void fill_job_desc(const Job* j, JobDesc* jd) {
  memset(jd, 0, sizeof(*jd));
  jd->n = j->n; jd->t = j->t; jd->l = j->l; jd->d = j->d;
  jd->W = j->W; jd->wstride = j->wstride;
  jd->planes = j->planes; jd->codes = j->codes;
  jd->kind = j->kind; jd->ks = j->pv; jd->cpt = 1; jd->span0 = j->span0;
  jd->tiled = j->tiled ? 1 : 0;
  jd->seq_block = j->seq_block;
  jd->lo = j->lo; jd->hi = j->hi; jd->unit_lo = j->unit_lo; jd->unit_hi = j->unit_hi;
  jd->chunk_units = j->chunk_units; jd->nchunks = j->nchunks; jd->rest_threshold = j->rest;
  jd->qidx[0] = j->qidx[0]; jd->qidx[1] = j->qidx[1];
  jd->qmask[0] = j->qmask[0]; jd->qmask[1] = j->qmask[1];
  jd->qcap = j->qcap;
  jd->out = j->out; jd->out_cap = (uint64_t)j->out_cap;
  jd->ball = j->ball;
  jd->bitmap = j->bitmap;
  jd->bm_base = j->bm_base;
}

int max_active(const Server* S) { return S->o.max_active > 0 ? S->o.max_active : 64; }

// (Re)builds the graph that replays one step launch over the table.
int prepare_launch(Server* S, int kind, int pv, size_t smem) {
  if (S->kind == kind && S->pv == pv && S->smem >= smem && (S->exec || !S->o.use_graph))
    return MOTIF_OK;
  smem = std::max(smem, S->smem);
  // GROUP k = 4 tables run the kernel variant with the split tiled pass: jobs of either form
  // share the table as they arrive.
  const int lk = launch_kind(kind, pv, true);
  if (step_kernel_attrs(lk, pv, smem) != cudaSuccess) return MOTIF_ERR_CUDA;
  const int per_sm = step_max_ctas_per_sm(lk, pv, S->block, smem);
  if (per_sm <= 0) return MOTIF_ERR_ARG;
  S->kind = kind;
  S->pv = pv;
  S->smem = smem;
  S->grid = per_sm * S->sms;
  if (S->exec) { cudaGraphExecDestroy(S->exec); S->exec = nullptr; }
  if (S->graph) { cudaGraphDestroy(S->graph); S->graph = nullptr; }
  if (S->o.use_graph) {
    // One step-kernel node, built explicitly (no stream capture, so client threads can never
    // leak work into the graph).
    cudaGraph_t g = nullptr;
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e == cudaSuccess)
      e = add_step_node(g, lk, pv, S->d_jobs, S->d_states, max_active(S), S->d_ctl, S->grid,
                        S->block, S->smem, 0, 0, &node);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&S->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      S->exec = nullptr;
      return status_from_cuda(e);
    }
  }
  return MOTIF_OK;
}

// Tile budget per warp and step: bounds the length of one step, so that arrivals are admitted
// soon.  While jobs wait for admission (backlog) the default budget is four times larger: a
// full table gains more from fewer, longer steps (less scheduling per job) than a waiting job
// loses.
unsigned tiles_per_warp(const Server* S, bool backlog) {
  const unsigned warps = (unsigned)S->grid * (unsigned)(S->block / 32);
  if (S->o.step_tiles > 0) return std::max(1u, (unsigned)S->o.step_tiles / std::max(1u, warps));
  return backlog ? 192 : 48;
}

// Uploads descriptors of the active jobs; states of jobs that moved down are copied, states of
// newly admitted jobs zeroed, and unused slots marked done.
// Uploads the descriptors and states of the table, two copies from pinned memory: the state of
// slot i is the host copy's state of slot old_slot[i], or zero for a newly admitted job
// (old_slot[i] < 0); unused slots are marked done.  The pinned buffers are written again only
// after the next step's wait, so the copies are complete by then.
int upload_table(Server* S, const std::vector<int>& old_slot) {
  const int cap = max_active(S);
  const int nact = (int)S->active.size();
  memset(S->h_jobs, 0, sizeof(JobDesc) * cap);
  memset(S->h_table, 0, sizeof(JobState) * cap);
  for (int i = 0; i < nact; ++i) {
    fill_job_desc(S->active[i], &S->h_jobs[i]);
    if (old_slot[i] >= 0) S->h_table[i] = S->mirror[old_slot[i]];
  }
  for (int i = nact; i < cap; ++i) S->h_table[i].done = 1;
  S->mirror.assign(S->h_table, S->h_table + cap);
  cudaError_t e = cudaMemcpyAsync(S->d_jobs, S->h_jobs, sizeof(JobDesc) * cap,
                                  cudaMemcpyHostToDevice, S->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->d_states, S->h_table, sizeof(JobState) * cap,
                        cudaMemcpyHostToDevice, S->stream);
  return status_from_cuda(e);
}

// Copies a finished job's `count` ascending codes from its output buffer to a pinned host block,
// on stream r.
int copy_result(Server* S, Job* j, unsigned long long fc, cudaStream_t r) {
  j->result_size = (int64_t)fc;
  if (fc) {
    j->result = host_take(S, fc, &j->result_cap);
    if (!j->result) return MOTIF_ERR_OOM;
  }
  cudaError_t e = cudaSuccess;
  if (fc) e = cudaMemcpyAsync(j->result, j->out, fc * 8, cudaMemcpyDeviceToHost, r);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r);
  return status_from_cuda(e);
}

// Bitmap output whose codes outgrew the buffer: compacts the job's bitmap in order into its
// output buffer again (grown, and the compaction repeated, until the codes fit), counting at
// cnt, and copies the codes to the host; on stream r.
int finish_bitmap_job(Server* S, Job* j, unsigned long long* cnt, cudaStream_t r) {
  unsigned long long fc = 0;
  for (;;) {
    cudaError_t e = launch_bitmap_compact(j->bitmap, j->bm_words, j->bm_base, j->out, j->out_cap,
                                          j->bm_scratch, cnt, r);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&fc, cnt, sizeof(fc), cudaMemcpyDeviceToHost, r);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r);
    if (e != cudaSuccess) return status_from_cuda(e);
    if (fc <= (unsigned long long)j->out_cap) break;
    sfree(S, j->out);
    j->out_cap = (int64_t)fc;
    j->out = (uint64_t*)salloc_on(S, (size_t)j->out_cap * 8, r);
    if (!j->out) return MOTIF_ERR_OOM;
  }
  return copy_result(S, j, fc, r);
}

// A job that finished in a step: the job, its slot in that step's table and the step's state
// snapshot (whose out_count of the slot the sort / compaction counts in).
struct Finished {
  Job* j;
  int slot;
  JobState state;
};

// Finishes the jobs of one step (their codes fit their buffers), all at once, on the retire
// stream while the next step runs: one launch sorts every list of at most 4096 codes, a radix
// sort runs per larger list and three launches compact every bitmap, counting in the step's
// snapshot `snap`; one wait then reads every final count, the results are copied to pinned
// host blocks together, and one more wait ends the copies.  A bitmap job whose codes outgrow
// its buffer takes finish_bitmap_job alone.  Sets each job's status.
void retire_finished(Server* S, const std::vector<Finished>& fin, JobState* snap) {
  cudaStream_t r = S->retire_stream;
  int nsmall = 0, nbm = 0;
  unsigned bm_blocks = 0;
  for (const Finished& f : fin) {
    Job* j = f.j;
    j->status = MOTIF_OK;
    const unsigned long long found = f.state.out_count;
    unsigned long long* cnt = &snap[f.slot].out_count;
    if (j->bitmap) {
      S->h_bm_first[nbm] = bm_blocks;
      S->h_bm_tasks[nbm++] = BitmapTask{j->bitmap, j->bm_words, j->bm_base, j->out,
                                        (long long)j->out_cap, j->bm_scratch, cnt};
      bm_blocks += (unsigned)bitmap_task_blocks(j->bm_words);
    } else if (found > 4096) {
      const size_t need = sort_scratch_bytes(j->out_cap, S->sms);
      j->sort = salloc_on(S, need, r);
      j->sort_bytes = need;
      if (!j->sort ||
          launch_sort_unique(j->out, cnt, j->out_cap, 2 * j->l, j->sort, S->sms,
                             (long long)found, r) != cudaSuccess)
        j->status = j->sort ? MOTIF_ERR_CUDA : MOTIF_ERR_OOM;
    } else if (found > 1) {
      S->h_sort_tasks[nsmall++] = SortTask{j->out, cnt, (long long)j->out_cap};
    }
  }
  S->h_bm_first[nbm] = bm_blocks;
  cudaError_t e = cudaSuccess;
  if (nsmall)
    e = cudaMemcpyAsync(S->d_sort_tasks, S->h_sort_tasks, sizeof(SortTask) * nsmall,
                        cudaMemcpyHostToDevice, r);
  if (e == cudaSuccess && nbm)
    e = cudaMemcpyAsync(S->d_bm_tasks, S->h_bm_tasks, sizeof(BitmapTask) * nbm,
                        cudaMemcpyHostToDevice, r);
  if (e == cudaSuccess && nbm)
    e = cudaMemcpyAsync(S->d_bm_first, S->h_bm_first, sizeof(unsigned) * (nbm + 1),
                        cudaMemcpyHostToDevice, r);
  if (e == cudaSuccess) e = launch_small_sort_tasks(S->d_sort_tasks, nsmall, r);
  if (e == cudaSuccess)
    e = launch_bitmap_compact_tasks(S->d_bm_tasks, S->d_bm_first, nbm, bm_blocks, r);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->h_fin, snap, sizeof(JobState) * max_active(S),
                        cudaMemcpyDeviceToHost, r);
  if (e == cudaSuccess) e = cudaStreamSynchronize(r);
  if (e != cudaSuccess) {
    for (const Finished& f : fin) f.j->status = MOTIF_ERR_CUDA;
    return;
  }
  for (const Finished& f : fin) {
    Job* j = f.j;
    if (j->status != MOTIF_OK) continue;
    const unsigned long long fc = S->h_fin[f.slot].out_count;
    if (j->bitmap && fc > (unsigned long long)j->out_cap) {  // grow, compact again, copy
      j->status = finish_bitmap_job(S, j, &snap[f.slot].out_count, r);
      continue;
    }
    j->result_size = (int64_t)fc;
    if (!fc) continue;
    j->result = host_take(S, fc, &j->result_cap);
    if (!j->result) { j->status = MOTIF_ERR_OOM; continue; }
    if (cudaMemcpyAsync(j->result, j->out, fc * 8, cudaMemcpyDeviceToHost, r) != cudaSuccess)
      j->status = MOTIF_ERR_CUDA;
  }
  if (cudaStreamSynchronize(r) != cudaSuccess)
    for (const Finished& f : fin) f.j->status = MOTIF_ERR_CUDA;
}

// Marks retired jobs done (under the lock) and releases their device buffers.
void mark_done(Server* S, const std::vector<Finished>& fin) {
  for (const Finished& f : fin) {
    Job* j = f.j;
    j->t_done = now_ms();
    j->done = true;
    S->budget_used -= j->footprint;
    release_buffers(S, j);
  }
  if (!fin.empty()) S->cv_done.notify_all();
}

// Fails every job of the table and those still retiring (a CUDA error), under the lock.
void fail_all(Server* S, std::vector<Finished>* retiring) {
  for (Job* j : S->active) { j->status = MOTIF_ERR_CUDA; j->done = true; }
  for (const Finished& f : *retiring) { f.j->status = MOTIF_ERR_CUDA; f.j->done = true; }
  S->active.clear();
  retiring->clear();
  S->cv_done.notify_all();
}

// The scheduler loop.  Each turn: admission (under the lock), the upload of a changed table,
// the launch of one step, then, while that step runs, the retirement of the jobs that finished
// in the step before (on the retire stream); then the wait for the step and the compaction of
// the table (finished jobs leave it at once: their codes and counts stay in their buffers and in
// the step's state snapshot, one of two, until they are retired in the next turn).
void scheduler(Server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  bool dirty = true;
  std::vector<int> old_slot;
  std::vector<Finished> retiring;  // finished in the last step, retired in this turn
  int snap_buf = 0;                // the snapshot buffer of the next step
  for (;;) {
    // Admission, in arrival order, while slots and the memory budget allow.  The table runs one
    // kernel variant, so a job of another variant waits until the table drains; later jobs of
    // the table's variant are admitted past it until it has waited kHeadWaitMs, after which
    // nothing more is admitted and the table drains for it.  A job that does not fit the memory
    // budget stops admission (memory is granted in arrival order; jobs still retiring hold
    // theirs).
    const int64_t budget = S->o.device_budget > 0 ? S->o.device_budget : (8ll << 30);
    old_slot.assign(S->active.size(), 0);
    for (size_t i = 0; i < S->active.size(); ++i) old_slot[i] = (int)i;
    for (auto it = S->queue.begin();
         it != S->queue.end() && (int)S->active.size() < max_active(S);) {
      Job* j = *it;
      if (!S->active.empty() && (j->kind != S->kind || j->pv != S->pv)) {
        if (now_ms() - j->t_submit > kHeadWaitMs) break;  // the oldest passed-over job
        ++it;
        continue;
      }
      j->footprint = footprint_of(j);
      if (!S->active.empty() && S->budget_used + j->footprint > budget) break;
      if (!allocate_job(S, j)) {
        release_run_buffers(S, j);  // keeps the window copies: the job stays queued
        if (S->active.empty() && retiring.empty()) {  // cannot ever fit: fail the job
          release_buffers(S, j);
          it = S->queue.erase(it);
          j->status = MOTIF_ERR_OOM;
          j->done = true;
          j->t_done = now_ms();
          S->cv_done.notify_all();
          continue;
        }
        break;
      }
      it = S->queue.erase(it);
      if (j->ready) cudaStreamWaitEvent(S->stream, j->ready, 0);  // its windows are copied
      if (prepare_launch(S, j->kind, j->pv, j->smem) != MOTIF_OK) {
        release_buffers(S, j);
        j->status = MOTIF_ERR_CUDA;
        j->done = true;
        j->t_done = now_ms();
        S->cv_done.notify_all();
        continue;
      }
      j->t_admit = now_ms();
      S->budget_used += j->footprint;
      S->active.push_back(j);
      old_slot.push_back(-1);
      dirty = true;
    }
    if (S->active.empty()) {
      if (!retiring.empty()) {  // nothing to overlap: retire the last step's jobs now
        lk.unlock();
        retire_finished(S, retiring, S->d_snap[snap_buf ^ 1]);
        lk.lock();
        mark_done(S, retiring);
        retiring.clear();
        continue;
      }
      if (S->stopping) break;
      S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
      continue;
    }
    // From here to the compaction the lock is not held: the table (S->active) is the scheduler
    // thread's own, and clients read a job's results only after its done flag is set under the
    // lock, so submissions and polls go on meanwhile.
    const int nact = (int)S->active.size();
    const bool backlog = !S->queue.empty();
    lk.unlock();
    if (dirty) {
      const int rc = upload_table(S, old_slot);
      if (rc != MOTIF_OK) {
        lk.lock();
        fail_all(S, &retiring);
        continue;
      }
      dirty = false;
    }
    // One device step over the whole table, then its state snapshot (for the retirement of the
    // jobs that finish in it) and the host copy of the states.
    JobState* snap = S->d_snap[snap_buf];
    *S->h_ctl = StepCtl{};
    S->h_ctl->tiles_per_warp = tiles_per_warp(S, backlog);
    cudaError_t e = cudaMemcpyAsync(S->d_ctl, S->h_ctl, sizeof(StepCtl), cudaMemcpyHostToDevice,
                                    S->stream);
    cudaEventRecord(S->ev0, S->stream);
    if (e == cudaSuccess) {
      if (S->exec) {
        e = cudaGraphLaunch(S->exec, S->stream);
        note_launches(1);
      } else {
        e = launch_step(launch_kind(S->kind, S->pv, true), S->pv, S->d_jobs, S->d_states,
                        max_active(S), S->d_ctl, S->grid, S->block, S->smem, S->stream);
      }
    }
    cudaEventRecord(S->ev1, S->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(snap, S->d_states, sizeof(JobState) * max_active(S),
                          cudaMemcpyDeviceToDevice, S->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(S->h_states, snap, sizeof(JobState) * nact, cudaMemcpyDeviceToHost,
                          S->stream);
    // The jobs of the step before retire while this one runs; they are marked done with the
    // compaction below (one turn of the lock per step).
    std::vector<Finished> retired;
    if (!retiring.empty()) {
      retire_finished(S, retiring, S->d_snap[snap_buf ^ 1]);
      retired.swap(retiring);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    float step_ms = 0;
    cudaEventElapsedTime(&step_ms, S->ev0, S->ev1);
    if (e != cudaSuccess) {
      lk.lock();
      mark_done(S, retired);
      fail_all(S, &retiring);
      continue;
    }
    const std::vector<JobState> st(S->h_states, S->h_states + nact);
    std::copy(st.begin(), st.end(), S->mirror.begin());
    // Compaction: finished jobs leave the table (to be retired next turn); jobs whose list
    // outgrew its buffer start again in place with a larger one.
    std::vector<Job*> keep;
    std::vector<int> moved, failed;
    for (int i = 0; i < nact; ++i) {
      Job* j = S->active[i];
      j->gpu_ms += step_ms;
      if (!st[i].done) { keep.push_back(j); moved.push_back(i); continue; }
      const unsigned long long found = st[i].out_count;
      if (!j->bitmap && found > (unsigned long long)j->out_cap) {
        sfree(S, j->out);
        j->out_cap = (int64_t)found;
        j->out = (uint64_t*)salloc(S, (size_t)j->out_cap * 8);
        if (!j->out) {
          j->status = MOTIF_ERR_OOM;
          failed.push_back(i);
        } else {
          S->mirror[i] = JobState{};  // it starts again
          keep.push_back(j);
          moved.push_back(i);
          dirty = true;  // descriptor changed
        }
        continue;
      }
      retiring.push_back(Finished{j, i, st[i]});
    }
    snap_buf ^= 1;
    lk.lock();
    mark_done(S, retired);
    for (const int i : failed) {
      Job* j = S->active[i];
      j->t_done = now_ms();
      j->done = true;
      S->budget_used -= j->footprint;
      release_buffers(S, j);
      S->cv_done.notify_all();
    }
    if (keep.size() != (size_t)nact) {
      // The remaining jobs move down to their new slots, their states with them in the host
      // copy; the next upload (at the loop's top, after admission) takes them to the device.
      S->active = keep;
      std::vector<JobState> moved_states(S->mirror.size());
      for (size_t i = 0; i < moved.size(); ++i) moved_states[i] = S->mirror[moved[i]];
      S->mirror.swap(moved_states);
      dirty = true;
    }
  }
  // Shutdown: fail whatever is still queued.
  for (Job* j : S->queue) {
    j->status = MOTIF_ERR_STATE;
    j->done = true;
  }
  S->queue.clear();
  S->cv_done.notify_all();
}

// Frees the server's fixed buffers, streams, events and graph; each may be unset (a start that
// failed part way).
void free_fixed(Server* S) {
  if (S->exec) cudaGraphExecDestroy(S->exec);
  if (S->graph) cudaGraphDestroy(S->graph);
  for (void* d : {(void*)S->d_jobs, (void*)S->d_states, (void*)S->d_ctl, (void*)S->d_sort_tasks,
                  (void*)S->d_bm_tasks, (void*)S->d_bm_first, (void*)S->d_snap[0],
                  (void*)S->d_snap[1]})
    if (d) cudaFree(d);
  for (void* h : {(void*)S->h_states, (void*)S->h_sort_tasks, (void*)S->h_bm_tasks,
                  (void*)S->h_bm_first, (void*)S->h_jobs, (void*)S->h_table, (void*)S->h_ctl,
                  (void*)S->h_fin})
    if (h) cudaFreeHost(h);
  if (S->ev0) cudaEventDestroy(S->ev0);
  if (S->ev1) cudaEventDestroy(S->ev1);
  if (S->submit_stream) {
    cudaStreamSynchronize(S->submit_stream);
    cudaStreamDestroy(S->submit_stream);
  }
  if (S->retire_stream) cudaStreamDestroy(S->retire_stream);
  if (S->stream) cudaStreamDestroy(S->stream);
}

int start_locked(const motif_server_opts* opts) {
  if (g_srv) return MOTIF_ERR_STATE;
  Server* S = new Server();
  if (opts) S->o = *opts;
  cudaDeviceProp prop;
  if (cudaGetDevice(&S->device) != cudaSuccess ||
      cudaGetDeviceProperties(&prop, S->device) != cudaSuccess) {
    delete S;
    return MOTIF_ERR_CUDA;
  }
  S->sms = prop.multiProcessorCount;
  const int cap = max_active(S);
  if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->submit_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&S->d_jobs, sizeof(JobDesc) * cap) != cudaSuccess ||
      cudaMalloc(&S->d_states, sizeof(JobState) * cap) != cudaSuccess ||
      cudaMalloc(&S->d_ctl, sizeof(StepCtl)) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_states, sizeof(JobState) * cap, 0) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_jobs, sizeof(JobDesc) * cap, 0) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_table, sizeof(JobState) * cap, 0) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_ctl, sizeof(StepCtl), 0) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_fin, sizeof(JobState) * cap, 0) != cudaSuccess ||
      cudaMalloc(&S->d_snap[0], sizeof(JobState) * cap) != cudaSuccess ||
      cudaMalloc(&S->d_snap[1], sizeof(JobState) * cap) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->retire_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_sort_tasks, sizeof(SortTask) * cap, 0) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_bm_tasks, sizeof(BitmapTask) * cap, 0) != cudaSuccess ||
      cudaHostAlloc((void**)&S->h_bm_first, sizeof(unsigned) * (cap + 1), 0) != cudaSuccess ||
      cudaMalloc(&S->d_sort_tasks, sizeof(SortTask) * cap) != cudaSuccess ||
      cudaMalloc(&S->d_bm_tasks, sizeof(BitmapTask) * cap) != cudaSuccess ||
      cudaMalloc(&S->d_bm_first, sizeof(unsigned) * (cap + 1)) != cudaSuccess ||
      cudaEventCreate(&S->ev0) != cudaSuccess || cudaEventCreate(&S->ev1) != cudaSuccess) {
    free_fixed(S);
    delete S;
    return MOTIF_ERR_CUDA;
  }
  S->running = true;
  g_srv = S;
  S->th = std::thread(scheduler, S);
  return MOTIF_OK;
}

}  // namespace motif_serve

using namespace motif_serve;

extern "C" int motif_server_start(const motif_server_opts* opts) {
  std::lock_guard<std::mutex> g(g_life);
  return start_locked(opts);
}

extern "C" int motif_server_stop(void) {
  Server* S;
  {
    std::lock_guard<std::mutex> g(g_life);
    S = g_srv;
    if (!S) return MOTIF_ERR_STATE;
    g_srv = nullptr;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  S->th.join();
  cudaStreamSynchronize(S->stream);
  cudaStreamSynchronize(S->submit_stream);  // the pack kernels have read their staging
  for (auto& kv : S->jobs) {
    release_buffers(S, kv.second);
    if (kv.second->result) cudaFreeHost(kv.second->result);
    delete kv.second;
  }
  for (auto& kv : S->host_free) cudaFreeHost(kv.second);
  S->host_free.clear();
  cudaStreamSynchronize(S->stream);
  free_fixed(S);
  delete S;
  return MOTIF_OK;
}

namespace motif_serve {

// Builds and queues the job of a configured plan.  Its windows are the plan's packed windows
// (seqs == NULL: copied on the submit stream) or are packed on the submit stream from the n host
// rows at seqs (row r at seqs + r * stride, characters already checked).
int submit_job(motif_plan_s* p, const char* seqs, int64_t stride, int64_t* job_id) {
  Server* S;
  {
    std::lock_guard<std::mutex> lg(g_life);
    if (!g_srv) {
      int rc = start_locked(nullptr);
      if (rc) return rc;
    }
    S = g_srv;
  }
  if (S->device != p->device) return MOTIF_ERR_ARG;
  Job* j = new Job();
  j->t_submit = now_ms();
  j->n = p->n; j->t = p->t; j->l = p->l; j->d = p->d; j->W = p->W; j->wstride = p->wstride;
  j->sms = S->sms;
  j->kind = MOTIF_KERNEL_GROUP;
  j->pv = std::min(kMaxKs, p->l);
  j->span0 = j->pv >= 3 ? 2 : 1;
  j->smem = step_smem_bytes(j->kind, j->pv, std::max(j->wstride, kWinAlign), 256);
  j->lo = p->lo; j->hi = p->hi;
  const int shift = 2 * j->pv;
  j->unit_lo = j->lo >> shift;
  j->unit_hi = j->hi > j->lo ? ((j->hi - 1) >> shift) + 1 : j->unit_lo;
  const uint64_t units = j->unit_hi - j->unit_lo;
  j->chunk_units = std::max<uint64_t>(1, std::min(units, kServeChunkGroups));
  j->nchunks = units == 0 || j->W <= 0 || p->empty_row
                   ? 0
                   : (units + j->chunk_units - 1) / j->chunk_units;
  j->qcap = j->chunk_units;
  j->words = mask_words(j->pv);
  j->tiled = j->pv == 4 && j->l >= 8 && j->W <= 65535 && j->unit_lo % 256 == 0 &&
             (j->chunk_units % 256 == 0 || units <= j->chunk_units);
  if (j->tiled && units > 0) {  // the tiled pass uses no queues: one chunk, one-entry queues
    j->chunk_units = units;
    j->nchunks = j->W <= 0 || p->empty_row ? 0 : 1;
    j->qcap = 1;
  }
  if (p->bitmap) {  // the plan's output choice: dense results go to a bitmap over the range
    j->bm_base = p->bm_base;
    j->bm_words = p->bm_words;
    j->seq_block = j->tiled && p->tiled_in_batch ? p->seq_block : 0;
  }
  j->rest = (uint64_t)256 * S->sms;
  if (j->nchunks > 0) {
    std::lock_guard<std::mutex> sg(S->submit_mu);
    j->ball = ball_table(S->device, j->pv, S->submit_stream);
    if (!j->ball) { delete j; return MOTIF_ERR_CUDA; }
    // Private copies of the packed windows, made on the submit stream; the scheduler's stream
    // waits for `ready` before the job's first step, and the plan's stream waits for it too, so
    // the plan may be reused or destroyed as soon as this returns.
    j->win_bytes = (size_t)j->n * j->wstride * 8;  // a multiple of 16 bytes
    j->planes = (uint2*)pool_alloc(S->device, 2 * j->win_bytes, S->submit_stream);
    cudaError_t e = j->planes ? cudaSuccess : cudaErrorMemoryAllocation;
    if (e == cudaSuccess)
      j->codes = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(j->planes) + j->win_bytes);
    if (seqs) {
      // The rows go into a pinned staging block, row after row, and the pack kernel reads them
      // there (pinned memory is in the device's address space), on the submit stream.
      const size_t chars = (size_t)j->n * j->t;
      if (e == cudaSuccess) {
        j->stage = host_take(S, (chars + 7) / 8, &j->stage_cap);
        if (!j->stage) e = cudaErrorMemoryAllocation;
      }
      char* d_stage = nullptr;  // the block's device address (an error, not a fault, if unmapped)
      if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&d_stage, j->stage, 0);
      if (e == cudaSuccess) {
        char* dst = reinterpret_cast<char*>(j->stage);
        for (int r = 0; r < j->n; ++r)
          memcpy(dst + (size_t)r * j->t, seqs + (size_t)r * stride, (size_t)j->t);
        e = launch_pack(d_stage, j->t, j->n, j->t, j->l, j->wstride, j->planes, j->codes,
                        nullptr, S->submit_stream);
      }
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->ready, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(j->ready, S->submit_stream);
    } else {
      // Private copies of the plan's windows, ordered after its packing; the plan's stream
      // waits for `ready` too, so the plan may be reused or destroyed as soon as this returns.
      cudaEvent_t packed = nullptr;
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&packed, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(packed, p->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(S->submit_stream, packed, 0);
      if (packed) cudaEventDestroy(packed);  // released once the waits have seen it
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->planes, p->d_planes, j->win_bytes, cudaMemcpyDeviceToDevice,
                            S->submit_stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(j->codes, p->d_codes, j->win_bytes, cudaMemcpyDeviceToDevice,
                            S->submit_stream);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->ready, cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(j->ready, S->submit_stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, j->ready, 0);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (j->planes) cudaFreeAsync(j->planes, S->submit_stream);
      if (j->ready) cudaEventDestroy(j->ready);
      release_stage(S, j);
      delete j;
      return status_from_cuda(e);
    }
  }
  std::lock_guard<std::mutex> lk(S->mu);
  const int max_q = S->o.max_queued > 0 ? S->o.max_queued : 4096;
  if ((int)S->queue.size() >= max_q) {
    release_windows_from_client(S, j);
    delete j;
    return MOTIF_ERR_BUSY;
  }
  j->id = S->next_id++;
  S->jobs[j->id] = j;
  if (j->nchunks == 0) {  // no windows or empty range: nothing survives
    j->done = true;
    j->t_done = now_ms();
  } else {
    S->queue.push_back(j);
    S->cv_work.notify_all();
  }
  *job_id = j->id;
  return MOTIF_OK;
}

// True when every character of the n rows is one of ACGTacgt.
bool host_chars_valid(const char* seqs, int64_t stride, int n, int t) {
  static const std::array<uint8_t, 256> valid = [] {
    std::array<uint8_t, 256> a{};
    for (unsigned char c : {'A', 'C', 'G', 'T', 'a', 'c', 'g', 't'}) a[c] = 1;
    return a;
  }();
  unsigned bad = 0;
  for (int r = 0; r < n; ++r) {
    const unsigned char* row = reinterpret_cast<const unsigned char*>(seqs) + (size_t)r * stride;
    for (int c = 0; c < t; ++c) bad |= valid[row[c]] ^ 1u;
  }
  return bad == 0;
}

}  // namespace motif_serve

extern "C" int motif_submit(motif_plan p, int64_t* job_id) {
  if (!p || !job_id) return MOTIF_ERR_ARG;
  if (!p->loaded) return MOTIF_ERR_STATE;
  DeviceGuard g(p->device);
  // Validate device-loaded characters before accepting the job (host loads were checked while
  // they were staged; their windows are ordered before the job's copies by an event).
  if (p->check_alpha) {
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return MOTIF_ERR_CUDA;
    int err = 0;
    if (cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return MOTIF_ERR_CUDA;
    p->check_alpha = false;
    if (err) { p->loaded = false; return MOTIF_ERR_ALPHABET; }
  }
  return submit_job(p, nullptr, 0, job_id);
}

extern "C" int motif_submit_seqs(const char* seqs, int64_t stride, int32_t n, int32_t t,
                                 int32_t l, int32_t d, const motif_opts* opts, int64_t* job_id) {
  if (!seqs || !job_id) return MOTIF_ERR_ARG;
  // A plan without device memory carries the configuration (the same choices as
  // motif_plan_create makes); its options may name no stream or allocator of their own.
  std::unique_ptr<motif_plan_s> p(new (std::nothrow) motif_plan_s());
  if (!p) return MOTIF_ERR_OOM;
  int rc = plan_init_host(p.get(), n, t, l, d, opts);
  if (rc) return rc;
  if (stride < t) return MOTIF_ERR_ARG;
  if (!host_chars_valid(seqs, stride, n, t)) return MOTIF_ERR_ALPHABET;
  rc = plan_configure_host(p.get());
  if (rc) return rc;
  return submit_job(p.get(), seqs, stride, job_id);
}

extern "C" int motif_poll(int64_t job_id, uint64_t* out_codes, int64_t capacity,
                          int64_t* out_count, int32_t timeout_ms, motif_stats_t* stats) {
  if (!out_count || capacity < 0 || (capacity > 0 && !out_codes)) return MOTIF_ERR_ARG;
  Server* S;
  {
    std::lock_guard<std::mutex> g(g_life);
    S = g_srv;
  }
  if (!S) return MOTIF_ERR_NOTFOUND;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(job_id);
  if (it == S->jobs.end()) return MOTIF_ERR_NOTFOUND;
  Job* j = it->second;
  if (!j->done && timeout_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return j->done; });
  if (!j->done) return MOTIF_PENDING;
  *out_count = j->result_size;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->candidates = j->hi - j->lo;
    stats->survivors = (uint64_t)j->result_size;
    stats->queue_ms = j->t_admit > 0 ? j->t_admit - j->t_submit : 0;
    stats->total_ms = j->t_done - j->t_submit;
    stats->search_ms = j->gpu_ms;
    stats->device_bytes = j->footprint;
    stats->kernel = j->kind;
  }
  if (j->status == MOTIF_OK && j->result_size > capacity) return MOTIF_ERR_CAPACITY;
  // The job is released: once it leaves the map nobody else reaches it (the scheduler let go of
  // it when it marked it done), so the copy out runs without the lock.
  S->jobs.erase(it);
  lk.unlock();
  if (j->result_size > 0) memcpy(out_codes, j->result, (size_t)j->result_size * 8);
  const int st = j->status;
  std::vector<uint64_t*> evicted;
  host_give(S, j->result, j->result_cap, &evicted);
  delete j;  // the scheduler released its device buffers when it retired the job
  for (uint64_t* b : evicted) cudaFreeHost(b);
  return st;
}

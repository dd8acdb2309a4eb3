// Batching and tuning.
//
// motif_batch_search runs many uneven jobs in one job table: every step launch walks all jobs
// and pulls tiles of whichever passes still have work, so small jobs fill the SMs that a large
// job's tail leaves idle and no job pays its own launch-and-drain cost.  The launch sequence can
// be captured once in a CUDA graph and replayed until every job is done.
//
// motif_autotune times candidate configurations on a sub-range of the plan's candidates and
// keeps the fastest, in the plan and in a process-wide cache keyed by the job's shape.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "plan.h"

using namespace motif;

namespace motif_batch {

// Per-device streams, job-table buffers and step graphs reused across batch calls.
struct BatchCtx {
  cudaStream_t stream = nullptr;       // steps, then the jobs' sorts / compactions
  cudaStream_t copy_stream = nullptr;  // each job's codes to the host, once the counts are known
  JobDesc* d_jobs = nullptr;
  JobState* d_states = nullptr;
  StepCtl* d_ctl = nullptr;
  JobState* h_states = nullptr;            // pinned: every job's state after its sort
  StepCtl* h_ctl = nullptr;                // pinned: the step control after a table's steps
  SortTask* h_sort_tasks = nullptr;        // pinned staging of the sort / compaction tasks
  BitmapTask* h_bm_tasks = nullptr;
  unsigned* h_bm_first = nullptr;
  SortTask* d_sort_tasks = nullptr;
  BitmapTask* d_bm_tasks = nullptr;
  unsigned* d_bm_first = nullptr;
  cudaEvent_t sorts_done = nullptr;    // the group's sorts and compactions, for the copy stream
  cudaEvent_t copies_done = nullptr;
  // Instantiated step graphs by (kind, p, jobs, grid, block, smem, max_steps); they name d_jobs,
  // d_states and d_ctl, so they are dropped when those are re-allocated.
  std::map<std::tuple<int, int, int, int, int, size_t, int>, cudaGraphExec_t> graphs;
  int cap = 0;
};
std::mutex g_mu;
BatchCtx g_ctx[64];

void drop_graphs(BatchCtx& c) {
  for (auto& kv : c.graphs) cudaGraphExecDestroy(kv.second);
  c.graphs.clear();
}

int ensure_ctx(int dev, int njobs, BatchCtx** out) {
  if (dev < 0 || dev >= 64) return MOTIF_ERR_ARG;
  BatchCtx& c = g_ctx[dev];
  for (cudaStream_t* s : {&c.stream, &c.copy_stream})
    if (!*s && cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) != cudaSuccess)
      return MOTIF_ERR_CUDA;
  for (cudaEvent_t* ev : {&c.copies_done, &c.sorts_done})
    if (!*ev && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess)
      return MOTIF_ERR_CUDA;
  if (njobs > c.cap) {
    drop_graphs(c);
    if (c.d_jobs) cudaFree(c.d_jobs);
    if (c.d_states) cudaFree(c.d_states);
    for (void* h : {(void*)c.h_states, (void*)c.h_sort_tasks, (void*)c.h_bm_tasks,
                    (void*)c.h_bm_first})
      if (h) cudaFreeHost(h);
    for (void* d : {(void*)c.d_sort_tasks, (void*)c.d_bm_tasks, (void*)c.d_bm_first})
      if (d) cudaFree(d);
    c.d_jobs = nullptr;
    c.d_states = nullptr;
    c.h_states = nullptr;
    c.h_sort_tasks = nullptr;
    c.h_bm_tasks = nullptr;
    c.h_bm_first = nullptr;
    c.d_sort_tasks = nullptr;
    c.d_bm_tasks = nullptr;
    c.d_bm_first = nullptr;
    c.cap = 0;
    if (!c.d_ctl && cudaMalloc(&c.d_ctl, sizeof(StepCtl)) != cudaSuccess) return MOTIF_ERR_OOM;
    if (!c.h_ctl && cudaHostAlloc((void**)&c.h_ctl, sizeof(StepCtl), 0) != cudaSuccess) {
      c.h_ctl = nullptr;
      return MOTIF_ERR_OOM;
    }
    const int cap = std::max(njobs, 64);
    if (cudaMalloc(&c.d_jobs, sizeof(JobDesc) * cap) != cudaSuccess ||
        cudaMalloc(&c.d_states, sizeof(JobState) * cap) != cudaSuccess ||
        cudaHostAlloc((void**)&c.h_states, sizeof(JobState) * cap, 0) != cudaSuccess ||
        cudaHostAlloc((void**)&c.h_sort_tasks, sizeof(SortTask) * cap, 0) != cudaSuccess ||
        cudaHostAlloc((void**)&c.h_bm_tasks, sizeof(BitmapTask) * cap, 0) != cudaSuccess ||
        cudaHostAlloc((void**)&c.h_bm_first, sizeof(unsigned) * (cap + 1), 0) != cudaSuccess ||
        cudaMalloc(&c.d_sort_tasks, sizeof(SortTask) * cap) != cudaSuccess ||
        cudaMalloc(&c.d_bm_tasks, sizeof(BitmapTask) * cap) != cudaSuccess ||
        cudaMalloc(&c.d_bm_first, sizeof(unsigned) * (cap + 1)) != cudaSuccess)
      return MOTIF_ERR_OOM;
    c.cap = cap;
  }
  *out = &c;
  return MOTIF_OK;
}

// Runs the job table [0, njobs) of one kernel variant to completion on ctx->stream.  one_step:
// every job of the table finishes in one step (one tiled pass over a single chunk), so the graph
// holds no loop.  The graph path only enqueues: the step control's copy to c->h_ctl follows the
// graph, and the caller's wait (table_status) reads it; the per-step path waits itself.
int run_table(BatchCtx* c, int kind, int pv, int njobs, int grid, int block, size_t smem,
              int max_steps, bool use_graph, int timeout_ms, bool one_step) {
  cudaStream_t s = c->stream;
  if (!use_graph) {
    return run_steps(kind, pv, c->d_jobs, c->d_states, njobs, c->d_ctl, grid, block, smem,
                     max_steps, true, timeout_ms, s, nullptr);
  }
  // One graph launch: init, then a while loop of step launches that ends when every job is
  // done (or after max_steps steps).  The instantiated graph is kept for later batches of the
  // same shape.
  const auto key = std::make_tuple(kind, pv, njobs, grid, block, smem, one_step ? -1 : max_steps);
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaSuccess;
  auto it = c->graphs.find(key);
  if (it != c->graphs.end()) {
    exec = it->second;
  } else {
    e = build_step_graph(kind, pv, c->d_jobs, c->d_states, njobs, c->d_ctl, grid, block, smem,
                         (unsigned)max_steps, 1, &exec, one_step);
    if (e == cudaSuccess) {
      if (c->graphs.size() >= 16) drop_graphs(*c);
      c->graphs[key] = exec;
    }
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, s);
  (void)timeout_ms;
  return status_from_cuda(e);
}

// After the wait that follows a graph-launched table: every job done (else the step bound ended
// the loop first).
int table_status(BatchCtx* c, bool use_graph) {
  if (!use_graph) return MOTIF_OK;  // run_steps checked it
  note_launches(1 + (int)c->h_ctl->steps);
  return c->h_ctl->active_jobs == 0 ? MOTIF_OK : MOTIF_ERR_TIMEOUT;
}

}  // namespace motif_batch

using namespace motif_batch;

extern "C" int motif_batch_search(int32_t njobs, const motif_plan* plans,
                                  uint64_t* const* out_codes, const int64_t* capacities,
                                  int64_t* out_counts, int32_t* statuses, int32_t use_graph) {
  if (njobs < 1 || !plans || !out_codes || !capacities || !out_counts || !statuses)
    return MOTIF_ERR_ARG;
  for (int j = 0; j < njobs; ++j) {
    if (!plans[j] || capacities[j] < 0 || (capacities[j] > 0 && !out_codes[j])) return MOTIF_ERR_ARG;
    if (plans[j]->device != plans[0]->device) return MOTIF_ERR_ARG;
    statuses[j] = plans[j]->loaded ? MOTIF_OK : MOTIF_ERR_STATE;
    out_counts[j] = 0;
  }
  DeviceGuard g(plans[0]->device);
  std::lock_guard<std::mutex> lk(g_mu);
  BatchCtx* c = nullptr;
  int rc = ensure_ctx(plans[0]->device, njobs, &c);
  if (rc) return rc;
  // Every plan's pending work (loads) must finish before the batch stream reads its windows:
  // one wait per distinct stream (plans usually share one).
  std::vector<cudaStream_t> streams;
  for (int j = 0; j < njobs; ++j)
    if (std::find(streams.begin(), streams.end(), plans[j]->stream) == streams.end())
      streams.push_back(plans[j]->stream);
  for (cudaStream_t st : streams)
    if (cudaStreamSynchronize(st) != cudaSuccess) return MOTIF_ERR_CUDA;
  for (int j = 0; j < njobs; ++j) {
    if (plans[j]->check_alpha) {
      int err = 0;
      cudaMemcpy(&err, plans[j]->d_err, sizeof(int), cudaMemcpyDeviceToHost);
      plans[j]->check_alpha = false;
      if (err) { plans[j]->loaded = false; statuses[j] = MOTIF_ERR_ALPHABET; }
    }
  }
  const double t0 = now_ms();
  // Group the device jobs by kernel variant; each group runs as one table.  Where every job of
  // a group ends in one step (the whole tiled pass over one chunk), its jobs with bitmap output
  // (the dense ones, whose results are large) form a table of their own that runs first: their
  // result copies then overlap the steps of the tables after them.  (Jobs of several passes
  // keep one table: alone, their short late steps would leave the GPU idle.)
  std::vector<int> dev_jobs;
  std::map<std::pair<int, int>, bool> one_step_group;
  for (int j = 0; j < njobs; ++j) {
    motif_plan_s* p = plans[j];
    if (statuses[j] != MOTIF_OK || p->W <= 0 || p->hi <= p->lo || p->nchunks == 0 ||
        p->empty_row)
      continue;
    if (plan_ensure_buffers(p) != MOTIF_OK) {
      statuses[j] = MOTIF_ERR_OOM;
      continue;
    }
    dev_jobs.push_back(j);
    auto it = one_step_group.emplace(std::make_pair(p->kind, p->p), true).first;
    it->second = it->second && p->tiled_in_batch && p->nchunks == 1;
  }
  // The buffers are made on the plans' streams, and the batch stream uses them.
  for (cudaStream_t st : streams)
    if (cudaStreamSynchronize(st) != cudaSuccess) return MOTIF_ERR_CUDA;
  std::map<std::tuple<int, int, int>, std::vector<int>> groups;
  for (const int j : dev_jobs) {
    motif_plan_s* p = plans[j];
    const bool first = p->bitmap && one_step_group[std::make_pair(p->kind, p->p)];
    groups[std::make_tuple(first ? 0 : 1, p->kind, p->p)].push_back(j);
  }
  std::vector<char> redo(njobs, 0);
  // The event after the last table's sorts (the copies of every table end together before the
  // call returns), the tables' device times summed, and the jobs that ran.
  cudaEvent_t last_sorts = nullptr;
  float tot_steps = 0, tot_sort = 0;
  std::vector<int> ran;
  auto drop_copy_events = [&]() {
    if (last_sorts) cudaEventDestroy(last_sorts);
    last_sorts = nullptr;
  };
  // An error return with the earlier tables' copies still in flight waits for them first.
  auto bail = [&](int status) {
    cudaStreamSynchronize(c->stream);
    cudaStreamSynchronize(c->copy_stream);
    drop_copy_events();
    return status;
  };
  for (auto& kv : groups) {
    const int kind = std::get<1>(kv.first), pv = std::get<2>(kv.first);
    const std::vector<int>& ids = kv.second;
    std::vector<JobDesc> descs(ids.size());
    size_t smem = 0;
    int max_steps = 0, grid = 0, block = 256, timeout = 0;
    for (size_t i = 0; i < ids.size(); ++i) {
      motif_plan_s* p = plans[ids[i]];
      fill_desc(p, &descs[i], p->d_out, (uint64_t)p->out_cap);
      descs[i].tiled = p->tiled_in_batch ? 1 : 0;
      descs[i].seq_block = p->tiled_in_batch ? p->seq_block : 0;
      smem = std::max(smem, p->smem);
      max_steps = std::max<int>(max_steps, (int)std::min<uint64_t>(p->nchunks * p->n + 2, 1 << 30));
      block = p->block;
      timeout = std::max(timeout, p->opts.timeout_ms > 0 ? p->opts.timeout_ms : 60000);
    }
    // The split-capable kernel variant only where a job of the table is split; the tiled-only
    // kernel where every job runs the whole-tile tiled pass.
    bool split = false, all_tiled = true, one_step = true;
    for (const JobDesc& jd : descs) {
      split = split || jd.seq_block > 0;
      all_tiled = all_tiled && jd.tiled;
      one_step = one_step && jd.tiled && jd.nchunks == 1;
    }
    const int lkind = launch_kind(kind, pv, split, all_tiled);
    if (step_kernel_attrs(lkind, pv, smem) != cudaSuccess) return bail(MOTIF_ERR_CUDA);
    grid = step_max_ctas_per_sm(lkind, pv, block, smem) * plans[ids[0]]->sms;
    if (grid <= 0) return bail(MOTIF_ERR_ARG);
    cudaError_t e = cudaMemcpyAsync(c->d_jobs, descs.data(), sizeof(JobDesc) * ids.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    for (size_t i = 0; i < ids.size() && e == cudaSuccess; ++i) {
      motif_plan_s* p = plans[ids[i]];
      if (p->bitmap)  // all ones where (tile, sequence block) items AND their survivors in
        e = cudaMemsetAsync(p->d_bitmap, descs[i].seq_block > 0 ? 0xFF : 0, p->bm_words * 4,
                            c->stream);
      if (e == cudaSuccess && p->seeded && prepare_seed(p, c->stream) != MOTIF_OK)
        e = cudaErrorUnknown;
    }
    // Zero the states; CTAs rotate their starting job so every job's tiles start at once.
    if (e == cudaSuccess)
      e = launch_init_steps(c->d_states, (int)ids.size(), c->d_ctl, 0, 0, 1, c->stream);
    if (e != cudaSuccess) return bail(status_from_cuda(e));
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    for (auto& x : ev) cudaEventCreate(&x);
    // Leaves nothing in flight (copies into the caller's buffers included) before returning.
    auto fail = [&](int status) {
      cudaStreamSynchronize(c->stream);
      cudaStreamSynchronize(c->copy_stream);
      for (auto& x : ev) cudaEventDestroy(x);
      return bail(status);
    };
    cudaEventRecord(ev[0], c->stream);
    rc = run_table(c, lkind, pv, (int)ids.size(), grid, block, smem, max_steps, use_graph != 0,
                   timeout, one_step);
    cudaEventRecord(ev[1], c->stream);
    if (rc) return fail(rc);
    e = cudaMemcpyAsync(c->h_states, c->d_states, sizeof(JobState) * ids.size(),
                        cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(status_from_cuda(e));
    rc = table_status(c, use_graph != 0);
    if (rc) return fail(rc);
    const std::vector<JobState> st(c->h_states, c->h_states + ids.size());
    // Sort/dedup (or compact) every job's codes in its own buffer on the batch stream, the jobs
    // together: one launch sorts every list of at most 4096 codes (a CTA per job), a radix sort
    // runs per larger list, and three launches compact every bitmap.  One copy then brings back
    // every final count, and each job's codes go to the host on the copy stream, largest first.
    int nsmall = 0, nbm = 0;
    unsigned bm_blocks = 0;
    std::vector<char> sorted(ids.size(), 0);
    for (size_t i = 0; i < ids.size(); ++i) {
      const int j = ids[i];
      motif_plan_s* p = plans[j];
      const unsigned long long found = st[i].out_count;
      if (found > (unsigned long long)p->out_cap) {
        redo[j] = 1;  // the plan's own buffer was too small: rerun this job alone below
        continue;
      }
      unsigned long long* cnt = &c->d_states[i].out_count;
      if (p->bitmap) {
        c->h_bm_first[nbm] = bm_blocks;
        c->h_bm_tasks[nbm++] = BitmapTask{p->d_bitmap, p->bm_words, p->bm_base, p->d_out,
                                          (long long)p->out_cap, p->d_bm_scratch, cnt};
        bm_blocks += (unsigned)bitmap_task_blocks(p->bm_words);
      } else if (found <= 4096) {
        if (found > 1) c->h_sort_tasks[nsmall++] = SortTask{p->d_out, cnt, (long long)p->out_cap};
      } else {
        const size_t need = sort_scratch_bytes(p->out_cap, p->sms);
        if (need > p->sort_bytes) {
          plan_free(p, p->d_sort, p->sort_bytes);
          p->d_sort = plan_alloc(p, need);
          cudaStreamSynchronize(p->stream);  // the scratch is used on the batch stream
          p->sort_bytes = p->d_sort ? need : 0;
          if (p->g_sort) {  // a cached sort graph may name the old scratch
            cudaGraphExecDestroy(p->g_sort);
            p->g_sort = nullptr;
          }
          if (!p->d_sort) { statuses[j] = MOTIF_ERR_OOM; continue; }
        }
        e = launch_sort_unique(p->d_out, cnt, p->out_cap, 2 * p->l, p->d_sort, p->sms,
                               (long long)found, c->stream);
        if (e != cudaSuccess) return fail(status_from_cuda(e));
      }
      sorted[i] = 1;
    }
    c->h_bm_first[nbm] = bm_blocks;
    if (nsmall)
      e = cudaMemcpyAsync(c->d_sort_tasks, c->h_sort_tasks, sizeof(SortTask) * nsmall,
                          cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && nbm)
      e = cudaMemcpyAsync(c->d_bm_tasks, c->h_bm_tasks, sizeof(BitmapTask) * nbm,
                          cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && nbm)
      e = cudaMemcpyAsync(c->d_bm_first, c->h_bm_first, sizeof(unsigned) * (nbm + 1),
                          cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_small_sort_tasks(c->d_sort_tasks, nsmall, c->stream);
    if (e == cudaSuccess)
      e = launch_bitmap_compact_tasks(c->d_bm_tasks, c->d_bm_first, nbm, bm_blocks, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], c->stream);  // sorts done
    if (e == cudaSuccess) e = cudaEventRecord(c->sorts_done, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->h_states, c->d_states, sizeof(JobState) * ids.size(),
                          cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(status_from_cuda(e));
    std::vector<size_t> order;
    for (size_t i = 0; i < ids.size(); ++i)
      if (sorted[i]) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
      return c->h_states[a].out_count > c->h_states[b].out_count;
    });
    e = cudaStreamWaitEvent(c->copy_stream, c->sorts_done, 0);
    if (e != cudaSuccess) return fail(status_from_cuda(e));
    for (const size_t i : order) {
      const int j = ids[i];
      motif_plan_s* p = plans[j];
      const unsigned long long fc = c->h_states[i].out_count;
      if (fc > (unsigned long long)p->out_cap) {  // a bitmap job outgrew the plan's buffer
        redo[j] = 1;
        continue;
      }
      out_counts[j] = (int64_t)fc;
      p->stats.survivors = fc;
      p->stats.candidates = p->hi - p->lo;
      if ((int64_t)fc > capacities[j]) {
        statuses[j] = MOTIF_ERR_CAPACITY;
        continue;
      }
      if (fc) {
        e = cudaMemcpyAsync(out_codes[j], p->d_out, fc * 8, cudaMemcpyDeviceToHost,
                            c->copy_stream);
        if (e != cudaSuccess) return fail(status_from_cuda(e));
      }
    }
    // The copies run on while the next table steps (ev[0..2] have completed: the wait on the
    // states above came after them).
    float steps_ms = 0, sort_ms = 0;
    cudaEventElapsedTime(&steps_ms, ev[0], ev[1]);
    cudaEventElapsedTime(&sort_ms, ev[1], ev[2]);
    tot_steps += steps_ms;
    tot_sort += sort_ms;
    ran.insert(ran.end(), ids.begin(), ids.end());
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    drop_copy_events();
    last_sorts = ev[2];
  }
  {
    // Every table's copies end here, timed on the batch stream.
    cudaEvent_t end = nullptr;
    cudaError_t e = cudaEventCreate(&end);
    if (e == cudaSuccess) e = cudaEventRecord(c->copies_done, c->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->copies_done, 0);
    if (e == cudaSuccess) e = cudaEventRecord(end, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      if (end) cudaEventDestroy(end);
      return bail(status_from_cuda(e));
    }
    float copy_ms = 0;  // the copy time not hidden under the steps and sorts
    if (last_sorts) cudaEventElapsedTime(&copy_ms, last_sorts, end);
    for (const int j : ran) {  // the batch's device times, shared by its jobs
      plans[j]->stats.search_ms = tot_steps;
      plans[j]->stats.sort_ms = tot_sort;
      plans[j]->stats.queue_ms = copy_ms;
    }
    cudaEventDestroy(end);
    drop_copy_events();
  }
  for (int j = 0; j < njobs; ++j) {
    if (!redo[j]) continue;
    int64_t cnt = 0;
    statuses[j] = motif_search(plans[j], out_codes[j], capacities[j], &cnt);
    out_counts[j] = cnt;
  }
  const double ms = now_ms() - t0;
  for (int j = 0; j < njobs; ++j) plans[j]->stats.total_ms = ms;
  for (int j = 0; j < njobs; ++j)
    if (statuses[j] != MOTIF_OK) return statuses[j];
  return MOTIF_OK;
}

// ---- autotuner ---------------------------------------------------------------------------------

namespace motif_tune {

struct Choice {
  int kernel, block, ctas_per_sm, cands_per_thread, compact_levels, suffix_bases;
  double cand_per_s;
};
std::mutex g_tmu;
std::map<std::string, Choice> g_cache;

std::string key_of(const motif_plan_s* p) {
  char buf[128];
  snprintf(buf, sizeof(buf), "w%d_l%d_d%d_n%d_W%d_sm%d", p->l <= 16 ? 32 : 64, p->l, p->d, p->n,
           p->W, p->sms);
  return buf;
}

// A loaded entry is kept only within the option rules every plan checks (kernel, block,
// candidates per lane, suffix bases, non-negative counts), so a damaged cache file cannot make
// the plans it matches fail.
bool choice_ok(const Choice& c) {
  return c.kernel >= MOTIF_KERNEL_AUTO && c.kernel <= MOTIF_KERNEL_BITSLICE && c.block >= 0 &&
         c.block <= 256 && c.block % 32 == 0 && c.ctas_per_sm >= 0 &&
         (c.cands_per_thread == 0 || c.cands_per_thread == 1 || c.cands_per_thread == 2 ||
          c.cands_per_thread == 4) &&
         c.compact_levels >= 0 && c.suffix_bases >= 0 && c.suffix_bases <= motif::kMaxKs;
}

void apply(motif_opts* o, const Choice& c) {
  o->kernel = c.kernel;
  o->block = c.block;
  o->ctas_per_sm = c.ctas_per_sm;
  o->cands_per_thread = c.cands_per_thread;
  o->compact_levels = c.compact_levels;
  o->suffix_bases = c.suffix_bases;
}

}  // namespace motif_tune

using namespace motif_tune;

extern "C" int motif_autotune(motif_plan p, int32_t budget_ms, motif_opts* best) {
  if (!p) return MOTIF_ERR_ARG;
  if (!p->loaded) return MOTIF_ERR_STATE;
  DeviceGuard g(p->device);
  const std::string key = key_of(p);
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      apply(&p->opts, it->second);
      int rc = plan_configure(p);
      if (best) *best = p->opts;
      return rc;
    }
  }
  std::vector<Choice> cands;
  if (p->l >= 8) cands.push_back({MOTIF_KERNEL_TILED, 256, 0, 0, 0, 4, 0});
  for (int ks = 2; ks <= kMaxKs; ++ks) {
    if (ks > p->l) break;
    for (int span : {1, 2})
      for (int cps : {0, 2})
        cands.push_back({MOTIF_KERNEL_GROUP, 256, cps, 0, span, ks, 0});
  }
  for (int cpt : {1, 2, 4}) cands.push_back({MOTIF_KERNEL_CAND, 256, 0, cpt, 1, 0, 0});
  if (p->d <= 7)
    for (int cpt : {1, 2, 4}) cands.push_back({MOTIF_KERNEL_BITSLICE, 256, 0, cpt, 1, 0, 0});
  const motif_opts saved = p->opts;
  const uint64_t full_lo = p->lo, full_hi = p->hi;
  const uint64_t span_c = full_hi - full_lo;
  const double t_start = now_ms();
  Choice win{};
  win.cand_per_s = -1;
  for (const Choice& c : cands) {
    if (budget_ms > 0 && now_ms() - t_start > budget_ms && win.cand_per_s > 0) break;
    motif_opts o = saved;
    apply(&o, c);
    // Sub-range sized for the kernel's speed: the per-candidate kernel is ~50x slower.
    const uint64_t want = cand_like(c.kernel) ? (1ull << 22) : (1ull << 26);
    o.range_lo = full_lo;
    o.range_hi = full_lo + std::min<uint64_t>(span_c, want);
    p->opts = o;
    p->lo = o.range_lo;
    p->hi = o.range_hi;
    if (plan_configure(p) != MOTIF_OK) continue;
    int64_t cnt = 0;
    std::vector<uint64_t> tmp(1 << 16);
    double best_ms = 1e30;
    for (int rep = 0; rep < 2; ++rep) {
      const int st = motif_search(p, tmp.data(), (int64_t)tmp.size(), &cnt);
      if (st != MOTIF_OK && st != MOTIF_ERR_CAPACITY) { best_ms = 1e30; break; }
      best_ms = std::min(best_ms, p->stats.search_ms + p->stats.sort_ms);
    }
    if (best_ms >= 1e30) continue;
    Choice r = c;
    r.cand_per_s = (double)(p->hi - p->lo) / (best_ms * 1e-3);
    if (r.cand_per_s > win.cand_per_s) win = r;
  }
  p->opts = saved;
  p->lo = full_lo;
  p->hi = full_hi;
  if (win.cand_per_s <= 0) {
    plan_configure(p);
    return MOTIF_ERR_CUDA;
  }
  apply(&p->opts, win);
  p->opts.range_lo = saved.range_lo;
  p->opts.range_hi = saved.range_hi;
  int rc = plan_configure(p);
  {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_cache[key] = win;
  }
  if (best) *best = p->opts;
  return rc;
}

extern "C" int motif_tune_cache_save(const char* path) {
  if (!path) return MOTIF_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_tmu);
  FILE* f = fopen(path, "w");
  if (!f) return MOTIF_ERR_ARG;
  fprintf(f, "{\n");
  size_t i = 0;
  for (auto& kv : g_cache) {
    const Choice& c = kv.second;
    fprintf(f,
            "  \"%s\": {\"kernel\": %d, \"block\": %d, \"ctas_per_sm\": %d, "
            "\"cands_per_thread\": %d, \"compact_levels\": %d, \"suffix_bases\": %d, "
            "\"cand_per_s\": %.6g}%s\n",
            kv.first.c_str(), c.kernel, c.block, c.ctas_per_sm, c.cands_per_thread,
            c.compact_levels, c.suffix_bases, c.cand_per_s, ++i < g_cache.size() ? "," : "");
  }
  fprintf(f, "}\n");
  fclose(f);
  return MOTIF_OK;
}

extern "C" int motif_tune_cache_load(const char* path) {
  if (!path) return MOTIF_ERR_ARG;
  FILE* f = fopen(path, "r");
  if (!f) return MOTIF_ERR_ARG;
  char line[512];
  std::lock_guard<std::mutex> lk(g_tmu);
  while (fgets(line, sizeof(line), f)) {
    char key[128];
    Choice c{};
    if (sscanf(line,
               " \"%127[^\"]\": {\"kernel\": %d, \"block\": %d, \"ctas_per_sm\": %d, "
               "\"cands_per_thread\": %d, \"compact_levels\": %d, \"suffix_bases\": %d, "
               "\"cand_per_s\": %lf",
               key, &c.kernel, &c.block, &c.ctas_per_sm, &c.cands_per_thread, &c.compact_levels,
               &c.suffix_bases, &c.cand_per_s) == 8 &&
        choice_ok(c))
      g_cache[key] = c;
  }
  fclose(f);
  return MOTIF_OK;
}

namespace motif {
// Applies a cached tuning choice to fresh plans created with MOTIF_KERNEL_AUTO.
bool tune_lookup(const motif_plan_s* p, motif_opts* o) {
  std::lock_guard<std::mutex> lk(g_tmu);
  auto it = g_cache.find(key_of(p));
  if (it == g_cache.end()) return false;
  apply(o, it->second);
  return true;
}
}  // namespace motif

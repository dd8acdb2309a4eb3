// C ABI: plans, window loading (K0), the search (K1 steps + K2 sort/dedup), the compare
// counter, statistics and small helpers.  Everything device-side runs on the plan's stream.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <atomic>
#include <mutex>
#include <vector>

#include "plan.h"

// Codes a blocking search reads back speculatively with its count (one wait for small results).
constexpr int64_t kResultPeek = 512;
// A plan's pinned host block: the read-back words, then (16-byte aligned) the search descriptor.
constexpr size_t kDescOffset = ((1 + kResultPeek) * sizeof(uint64_t) + 15) & ~(size_t)15;
constexpr size_t kHostBlockBytes = kDescOffset + sizeof(motif::JobDesc);

// Pinned host blocks of plans, shared by all plans of the process: the read-back words of a
// blocking search ([1 + kResultPeek]) and then the descriptor a search uploads.  A plan takes
// one at its first search and gives it back when destroyed, so plans that live for one search
// do not pin and unpin memory each time.
static std::mutex g_res_mu;
static std::vector<uint64_t*> g_res_free;

static uint64_t* take_result_block() {
  {
    std::lock_guard<std::mutex> g(g_res_mu);
    if (!g_res_free.empty()) {
      uint64_t* b = g_res_free.back();
      g_res_free.pop_back();
      return b;
    }
  }
  uint64_t* b = nullptr;
  if (cudaHostAlloc((void**)&b, kHostBlockBytes, 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return b;
}

static void give_result_block(uint64_t* b) {
  if (!b) return;
  std::lock_guard<std::mutex> g(g_res_mu);
  g_res_free.push_back(b);
}

using motif::JobDesc;
using motif::JobState;
using motif::StepCtl;

namespace motif {

int status_from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return MOTIF_OK;
  if (e == cudaErrorMemoryAllocation) return MOTIF_ERR_OOM;
  return MOTIF_ERR_CUDA;
}

namespace {
std::atomic<unsigned long long> g_launches{0};
}
void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
unsigned long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

cudaEvent_t* next_event_quad(motif_plan_s* p) {
  if (p->evq_used * 4 + 4 > p->evq.size()) {
    const size_t grow = std::max<size_t>(16, p->evq.size() / 4) * 4;
    for (size_t i = 0; i < grow; ++i) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      p->evq.push_back(e);
    }
  }
  return &p->evq[4 * p->evq_used++];
}

int fold_event_quads(motif_plan_s* p) {
  if (p->evq_used == 0 && p->graph_searches == 0) return MOTIF_OK;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return status_from_cuda(e);
  if (p->graph_searches > 0) {
    // Each graph launch ran an init kernel and one step kernel per step; every search of the
    // plan since the last fold ran the same number of steps as the last one.
    StepCtl ctl{};
    if (cudaMemcpy(&ctl, p->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost) == cudaSuccess) {
      p->last_steps = ctl.steps;
      note_launches((int)(p->graph_searches * (1 + (int64_t)ctl.steps)));
    }
    p->graph_searches = 0;
  }
  for (size_t q = 0; q < p->evq_used; ++q) {
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, p->evq[4 * q], p->evq[4 * q + 1]);
    cudaEventElapsedTime(&b, p->evq[4 * q + 2], p->evq[4 * q + 3]);
    p->sum_search_ms += a;
    p->sum_sort_ms += b;
    p->sum_searches += 1;
    p->stats.search_ms = a;
    p->stats.sort_ms = b;
  }
  cudaGetLastError();
  p->evq_used = 0;
  return MOTIF_OK;
}

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64] = {};
}  // namespace

cudaMemPool_t device_pool(int device) {
  if (device < 0 || device >= 64) return nullptr;
  std::lock_guard<std::mutex> g(g_pool_mu);
  if (!g_pool[device]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = kPoolKeepBytes;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaGetLastError();
      cudaMemPoolDestroy(pool);
      return nullptr;
    }
    g_pool[device] = pool;
  }
  return g_pool[device];
}

void* pool_alloc(int device, size_t bytes, cudaStream_t s) {
  void* ptr = nullptr;
  cudaMemPool_t pool = device_pool(device);
  if (!pool || cudaMallocFromPoolAsync(&ptr, bytes, pool, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return ptr;
}

void* plan_alloc(motif_plan_s* p, size_t bytes) {
  if (bytes == 0) return nullptr;
  void* ptr = nullptr;
  if (p->opts.alloc) ptr = p->opts.alloc(bytes, p->stream, p->opts.alloc_ctx);
  else ptr = pool_alloc(p->device, bytes, p->stream);
  if (ptr) p->device_bytes += (int64_t)bytes;
  return ptr;
}

void plan_free(motif_plan_s* p, void* ptr, size_t bytes) {
  if (!ptr) return;
  if (p->opts.free) p->opts.free(ptr, p->stream, p->opts.alloc_ctx);
  else cudaFreeAsync(ptr, p->stream);
  p->device_bytes -= (int64_t)bytes;
}

namespace {
std::mutex g_ball_mu;
uint64_t* g_ball[64][kMaxKs + 1] = {};
}  // namespace

const uint64_t* ball_table(int device, int ks, cudaStream_t s) {
  if (device < 0 || device >= 64 || ks < 1 || ks > kMaxKs) return nullptr;
  std::lock_guard<std::mutex> g(g_ball_mu);
  if (!g_ball[device][ks]) {
    uint64_t* t = nullptr;
    if (cudaMalloc(&t, (size_t)ball_table_words(ks) * 8) != cudaSuccess) return nullptr;
    if (launch_ball_table(t, ks, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      cudaFree(t);
      return nullptr;
    }
    g_ball[device][ks] = t;
  }
  return g_ball[device][ks];
}

void fill_desc(const motif_plan_s* p, JobDesc* jd, uint64_t* out, uint64_t out_cap) {
  memset(jd, 0, sizeof(*jd));
  jd->n = p->n; jd->t = p->t; jd->l = p->l; jd->d = p->d;
  jd->W = p->W; jd->wstride = p->wstride;
  jd->planes = p->d_planes; jd->codes = p->d_codes;
  jd->kind = cand_like(p->kind) ? MOTIF_KERNEL_CAND : p->kind;
  jd->ks = p->kind == MOTIF_KERNEL_GROUP ? p->p : 0;
  jd->cpt = cand_like(p->kind) ? p->p : 1;
  jd->span0 = p->span0;
  jd->tiled = p->tiled ? 1 : 0;
  jd->seq_block = p->tiled ? p->seq_block : 0;
  jd->lo = p->lo; jd->hi = p->hi;
  jd->unit_lo = p->unit_lo; jd->unit_hi = p->unit_hi;
  jd->chunk_units = p->chunk_units; jd->nchunks = p->nchunks;
  jd->rest_threshold = p->rest_threshold;
  jd->qidx[0] = p->d_qidx[0]; jd->qidx[1] = p->d_qidx[1];
  jd->qmask[0] = p->d_qmask[0]; jd->qmask[1] = p->d_qmask[1];
  jd->qcap = p->qcap;
  jd->out = out; jd->out_cap = out_cap;
  jd->ball = p->kind == MOTIF_KERNEL_GROUP ? ball_table(p->device, p->p, p->stream) : nullptr;
  jd->bitmap = p->bitmap ? p->d_bitmap : nullptr;
  jd->bm_base = p->bm_base;
  jd->valid = p->ragged ? p->d_valid : nullptr;
  jd->wrow = p->ragged ? p->d_wrow : nullptr;
  jd->seed = p->seeded ? p->d_seed : nullptr;
  jd->seed_base = p->seed_base;
}

// Number of l-base difference patterns with at most d differing bases: sum C(l,k) 3^k.
static uint64_t pattern_count(int l, int d) {
  uint64_t term = 1, sum = 0;
  for (int k = 0; k <= std::min(d, l); ++k) {
    sum += term;
    if (sum > (1ull << 40)) return sum;
    term = term * (uint64_t)(l - k) / (uint64_t)(k + 1) * 3;
  }
  return sum;
}

// Every code-space XOR mask that changes at most d bases of an l-mer (each changed base gets
// one of its 3 other values).
static void difference_patterns(int l, int d, std::vector<uint64_t>& out) {
  out.clear();
  std::vector<int> pos;
  // depth-first over increasing positions; each chosen position takes a nonzero 2-bit digit
  struct Rec {
    int l, d;
    std::vector<uint64_t>* out;
    void go(int from, int left, uint64_t mask) {
      out->push_back(mask);
      if (left == 0) return;
      for (int i = from; i < l; ++i)
        for (uint64_t v = 1; v <= 3; ++v) go(i + 1, left - 1, mask | (v << (2 * (l - 1 - i))));
    }
  } rec{l, d, &out};
  rec.go(0, std::min(d, l), 0);
}

// Probability, for uniform i.i.d. bases, that a candidate matches one sequence: a window
// matches with pw = sum_{k<=d} C(l,k) 3^k / 4^l, some of the W windows with
// q = 1 - (1 - pw)^W.
static double match_probability(const motif_plan_s* p) {
  double term = 1.0, sum = 0.0;  // C(l,k) 3^k
  for (int k = 0; k <= std::min(p->d, p->l); ++k) {
    sum += term;
    term = term * (p->l - k) / (k + 1) * 3.0;
  }
  const double pw = std::min(1.0, sum / std::pow(4.0, p->l));
  return pw >= 1.0 ? 1.0 : -std::expm1((double)std::max(p->W, 0) * std::log1p(-pw));
}

// Expected number of accepted codes of the plan's range (all n sequences matched: q^n).
static double expected_survivors(const motif_plan_s* p) {
  return (double)(p->hi - p->lo) * std::pow(match_probability(p), p->n);
}

static void free_queues(motif_plan_s* p) {
  for (int i = 0; i < 2; ++i) {
    plan_free(p, p->d_qidx[i], p->qcap * 4);
    plan_free(p, p->d_qmask[i], p->qcap * 8 * (size_t)p->qmask_words);
    p->d_qidx[i] = nullptr;
    p->d_qmask[i] = nullptr;
  }
  p->qcap = 0;
  p->qmask_words = 0;
}

int plan_configure(motif_plan_s* p) {
  const motif_opts& o = p->opts;
  // Kernel variant.
  if (o.kernel < MOTIF_KERNEL_AUTO || o.kernel > MOTIF_KERNEL_BITSLICE) return MOTIF_ERR_ARG;
  int kind = o.kernel == MOTIF_KERNEL_CAND ? MOTIF_KERNEL_CAND : MOTIF_KERNEL_GROUP;
  if (o.kernel == MOTIF_KERNEL_BITSLICE)  // the bit-sliced counter holds distances up to 7
    kind = p->d <= 7 ? MOTIF_KERNEL_BITSLICE : MOTIF_KERNEL_CAND;
  int pv;
  if (cand_like(kind)) {  // BITSLICE holds more state per candidate: one per lane by default
    pv = o.cands_per_thread > 0 ? o.cands_per_thread : (kind == MOTIF_KERNEL_BITSLICE ? 1 : 2);
    if (pv != 1 && pv != 2 && pv != 4) return MOTIF_ERR_ARG;
  } else {
    pv = o.suffix_bases > 0 ? o.suffix_bases : 4;
    if (pv > kMaxKs) return MOTIF_ERR_ARG;
    if (pv > p->l) pv = p->l;
  }
  const int span0 = o.compact_levels > 0 ? std::min(o.compact_levels, 2)
                                         : (kind == MOTIF_KERNEL_GROUP && pv >= 3 ? 2 : 1);
  const int block = o.block > 0 ? o.block : 256;
  if (block % 32 != 0 || block > 256) return MOTIF_ERR_ARG;
  const size_t smem = step_smem_bytes(kind, pv, std::max(p->wstride, kWinAlign), block);
  {
    cudaError_t e = step_kernel_attrs(kind, pv, smem);
    if (e != cudaSuccess) return status_from_cuda(e);
  }
  int per_sm = step_max_ctas_per_sm(kind, pv, block, smem);
  if (per_sm <= 0) return MOTIF_ERR_ARG;
  if (o.ctas_per_sm > 0) per_sm = std::min(per_sm, o.ctas_per_sm);
  // Units and chunking.
  const int shift = kind == MOTIF_KERNEL_GROUP ? 2 * pv : 0;
  const uint64_t unit_lo = p->lo >> shift;
  const uint64_t unit_hi = p->hi > p->lo ? ((p->hi - 1) >> shift) + 1 : unit_lo;
  const uint64_t units = unit_hi - unit_lo;
  const uint64_t max_chunk = kind == MOTIF_KERNEL_GROUP ? (1ull << 22) : (1ull << 28);
  const uint64_t chunk = std::max<uint64_t>(1, std::min(units, max_chunk));
  const int words = kind == MOTIF_KERNEL_GROUP ? mask_words(pv) : 0;
  if (chunk != p->qcap || words != p->qmask_words) free_queues(p);  // re-made on first use
  p->want_qcap = chunk;
  p->want_qwords = words;
  invalidate_graphs(p);
  // The prefix-tiled first pass (GROUP, k = 4): 256 lanes per CTA whose groups share all but
  // their last 4 prefix bases, so tiles must start on multiples of 256 groups.
  const bool want_tiled = o.kernel == MOTIF_KERNEL_AUTO || o.kernel == MOTIF_KERNEL_TILED;
  const bool tiled_ok = want_tiled && kind == MOTIF_KERNEL_GROUP && pv == 4 && block == 256 &&
                        p->l >= 8 && p->W <= 65535 && unit_lo % 256 == 0 &&
                        (chunk % 256 == 0 || units <= chunk);
  // Tiles that walk through most sequences (q > 0.52), fewer than the grid's CTAs: alone, they
  // leave the GPU partly idle for the whole search (few_long_tiles: fewer than 64, most of it).
  const bool long_tiles = match_probability(p) > 0.52;
  const bool few_long_tiles = long_tiles && units / 256 < 64;
  const bool underfilled_long_tiles = long_tiles && units / 256 < (uint64_t)per_sm * p->sms;
  // Output: a bitmap over the range (rounded out to whole 256-code groups) where it holds at
  // most 2^31 bits and the expected survivors make a list at least 1/2048 of its size; and,
  // for long tiles that do not fill the grid, where it is small (at most 2^24 bits): the skip
  // saves little in such tiles, and with a bitmap they split into (tile, sequence block) items
  // that fill the GPU.
  const uint64_t bm_base = p->lo & ~255ull;
  const uint64_t bm_bits = ((p->hi + 255) & ~255ull) - bm_base;
  if (o.output < MOTIF_OUTPUT_AUTO || o.output > MOTIF_OUTPUT_BITMAP) return MOTIF_ERR_ARG;
  bool bitmap = o.output == MOTIF_OUTPUT_BITMAP ||
                (o.output == MOTIF_OUTPUT_AUTO &&
                 (expected_survivors(p) * 2048.0 >= (double)bm_bits ||
                  (tiled_ok && underfilled_long_tiles && o.seq_block != -1 &&
                   bm_bits <= (1ull << 24))));
  if (bm_bits > (1ull << 31)) {
    if (o.output == MOTIF_OUTPUT_BITMAP) return MOTIF_ERR_ARG;
    bitmap = false;
  }
  p->bitmap = bitmap && p->hi > p->lo;
  p->bm_base = bm_base;
  p->bm_words = p->bitmap ? bm_bits / 32 : 0;
  // With bitmap output the expected survivors (at least 1/2048 of the range: 32 per tile of
  // 65536 codes) keep every tile alive to the last sequence, so the skip saves nothing there and
  // a tile splits into (tile, sequence block) items at no extra work; the blocks are sized so
  // that the items cover the grid four times over.
  if (o.seq_block < -1) return MOTIF_ERR_ARG;
  p->seq_block = 0;
  if (tiled_ok && p->bitmap && o.seq_block != -1) {
    if (o.seq_block > 0) {
      p->seq_block = std::min(o.seq_block, p->n);
    } else {
      const uint64_t tiles = (std::min(units, chunk) + 255) / 256;
      const uint64_t blocks =
          std::min<uint64_t>(p->n, (4ull * per_sm * p->sms + tiles - 1) / tiles);
      if (blocks > 1) p->seq_block = (int)((p->n + blocks - 1) / blocks);
    }
  }
  // AUTO leaves the tiled pass out for few long tiles that do not split into sequence blocks:
  // the per-group passes run those faster alone.  A batch runs its jobs side by side, so there
  // every eligible AUTO job stays tiled.
  p->tiled = tiled_ok && !(o.kernel == MOTIF_KERNEL_AUTO && few_long_tiles && p->seq_block == 0);
  p->tiled_in_batch = tiled_ok;
  // A split search runs on the step kernel variant that has the split; its occupancy decides the
  // grid.
  // A tiled plan runs the kernel whose only pass is the tiled pass (split plans: the step kernel
  // variant with the split); its dynamic shared memory is that of the GROUP kernel, which covers
  // the tile map and the list heads.
  p->lkind = launch_kind(kind, pv, p->tiled && p->seq_block > 0, p->tiled);
  if (p->lkind != kind) {
    if (step_kernel_attrs(p->lkind, pv, smem) != cudaSuccess) return MOTIF_ERR_CUDA;
    int ps = step_max_ctas_per_sm(p->lkind, pv, block, smem);
    if (ps <= 0) return MOTIF_ERR_ARG;
    per_sm = o.ctas_per_sm > 0 ? std::min(ps, o.ctas_per_sm) : ps;
  }
  // Candidate seeding by the first sequence's d-neighbourhoods (per-candidate kernels only).
  if (o.seed < MOTIF_SEED_ALL || o.seed > MOTIF_SEED_NEIGHBOURHOOD) return MOTIF_ERR_ARG;
  p->seeded = o.seed == MOTIF_SEED_NEIGHBOURHOOD;
  if (p->seeded) {
    if (!cand_like(kind)) return MOTIF_ERR_ARG;
    p->npat = pattern_count(p->l, p->d);
    p->seed_base = p->lo & ~63ull;
    const uint64_t bits = ((p->hi + 63) & ~63ull) - p->seed_base;
    if (p->npat > (1ull << 24) || bits > (1ull << 36)) return MOTIF_ERR_ARG;
    p->seed_words = std::max<uint64_t>(bits / 32, 1);
  }
  // A plan that runs the tiled pass alone and in batches never uses the survivor queues (the
  // tiled pass takes every sequence of a tile): its whole range is one chunk, so the pass does
  // not stop at chunk boundaries, and its queues hold a single entry.
  uint64_t plan_chunk = chunk;
  if (p->tiled && p->tiled_in_batch && units > 0) {
    plan_chunk = units;
    if (p->qcap != 1) free_queues(p);
    p->want_qcap = 1;
  }
  p->kind = kind;
  p->p = pv;
  p->span0 = span0;
  p->block = block;
  p->grid = per_sm * p->sms;
  p->smem = smem;
  p->unit_lo = unit_lo;
  p->unit_hi = unit_hi;
  p->chunk_units = plan_chunk;
  p->nchunks = units == 0 ? 0 : (units + plan_chunk - 1) / plan_chunk;
  p->rest_threshold = (uint64_t)256 * p->sms;
  if (kind == MOTIF_KERNEL_GROUP && !ball_table(p->device, pv, p->stream)) return MOTIF_ERR_CUDA;
  return MOTIF_OK;
}

void invalidate_graphs(motif_plan_s* p) {
  if (p->g_steps) cudaGraphExecDestroy(p->g_steps);
  if (p->g_sort) cudaGraphExecDestroy(p->g_sort);
  p->g_steps = p->g_sort = nullptr;
  p->desc_out = nullptr;
  p->desc_cap = -1;
  p->gs_out = nullptr;
  p->gs_cap = -1;
  p->gs_scratch = nullptr;
}

void free_seed(motif_plan_s* p) {
  if (p->d_pat) plan_free(p, p->d_pat, p->pat_alloc * 8);
  if (p->d_seed) plan_free(p, p->d_seed, (p->seed_alloc_words + 1) * 4);
  if (p->d_seed_scratch)
    plan_free(p, p->d_seed_scratch, bitmap_scratch_words(p->seed_alloc_words) * 4);
  if (p->d_seed_count) plan_free(p, p->d_seed_count, sizeof(unsigned long long));
  p->d_pat = nullptr;
  p->d_seed = nullptr;
  p->d_seed_scratch = nullptr;
  p->d_seed_count = nullptr;
  p->seed_alloc_words = p->pat_alloc = 0;
}

int prepare_seed(motif_plan_s* p, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(p->d_seed, 0, (p->seed_words + 1) * 4, s);
  if (e == cudaSuccess)
    e = launch_seed_scatter(p->d_codes, p->W, p->d_pat, p->npat, p->lo, p->hi, p->d_seed,
                            p->seed_base, s);
  return status_from_cuda(e);
}

void free_bitmap(motif_plan_s* p) {
  if (p->d_bitmap) plan_free(p, p->d_bitmap, p->bm_alloc_words * 4);
  if (p->d_bm_scratch) plan_free(p, p->d_bm_scratch, bitmap_scratch_words(p->bm_alloc_words) * 4);
  p->d_bitmap = nullptr;
  p->d_bm_scratch = nullptr;
  p->bm_alloc_words = 0;
}

int plan_ensure_buffers(motif_plan_s* p) {
  if (!p->d_qidx[0]) {
    invalidate_graphs(p);
    for (int i = 0; i < 2; ++i) {
      p->d_qidx[i] = (uint32_t*)plan_alloc(p, p->want_qcap * 4);
      if (!p->d_qidx[i]) return MOTIF_ERR_OOM;
      if (p->want_qwords) {
        p->d_qmask[i] = (uint64_t*)plan_alloc(p, p->want_qcap * 8 * (size_t)p->want_qwords);
        if (!p->d_qmask[i]) return MOTIF_ERR_OOM;
      }
    }
    p->qcap = p->want_qcap;
    p->qmask_words = p->want_qwords;
  }
  if (!p->d_out) {
    invalidate_graphs(p);
    p->d_out = (uint64_t*)plan_alloc(p, (size_t)(1 << 16) * 8);
    if (!p->d_out) return MOTIF_ERR_OOM;
    p->out_cap = 1 << 16;
  }
  if (p->seeded && (p->seed_alloc_words != p->seed_words || p->pat_alloc != p->npat)) {
    free_seed(p);
    std::vector<uint64_t> pat;
    difference_patterns(p->l, p->d, pat);
    p->d_pat = (uint64_t*)plan_alloc(p, pat.size() * 8);
    // one word past the bitmap: a fresh pass reads each lane's 32 bits as two words
    p->d_seed = (uint32_t*)plan_alloc(p, (p->seed_words + 1) * 4);
    p->d_seed_scratch = (unsigned*)plan_alloc(p, bitmap_scratch_words(p->seed_words) * 4);
    p->d_seed_count = (unsigned long long*)plan_alloc(p, sizeof(unsigned long long));
    p->desc_out = nullptr;  // the descriptor names the seed bitmap
    if (!p->d_pat || !p->d_seed || !p->d_seed_scratch || !p->d_seed_count) {
      free_seed(p);
      return MOTIF_ERR_OOM;
    }
    p->pat_alloc = pat.size();
    p->seed_alloc_words = p->seed_words;
    cudaError_t e = cudaMemcpyAsync(p->d_pat, pat.data(), pat.size() * 8,
                                    cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);  // `pat` is a local vector
    if (e != cudaSuccess) return status_from_cuda(e);
  }
  if (p->bitmap && p->bm_alloc_words != p->bm_words) {
    free_bitmap(p);
    p->d_bitmap = (uint32_t*)plan_alloc(p, p->bm_words * 4);
    p->d_bm_scratch = (unsigned*)plan_alloc(p, bitmap_scratch_words(p->bm_words) * 4);
    p->desc_out = nullptr;  // the descriptor names the bitmap
    if (!p->d_bitmap || !p->d_bm_scratch) {
      free_bitmap(p);
      return MOTIF_ERR_OOM;
    }
    p->bm_alloc_words = p->bm_words;
  }
  return MOTIF_OK;
}

int run_steps(int kind, int pv, const JobDesc* d_jobs, JobState* d_states, int njobs,
              StepCtl* d_ctl, int grid, int block, size_t smem, int max_steps, bool poll,
              int timeout_ms, cudaStream_t s, int* steps_run) {
  const double t0 = now_ms();
  int launched = 0;
  const int group = 8;
  while (launched < max_steps) {
    const int todo = poll ? std::min(group, max_steps - launched) : max_steps - launched;
    for (int i = 0; i < todo; ++i) {
      cudaError_t e = launch_step(kind, pv, d_jobs, d_states, njobs, d_ctl, grid, block, smem, s);
      if (e != cudaSuccess) return status_from_cuda(e);
    }
    launched += todo;
    if (!poll) break;
    unsigned active = 0;
    cudaError_t e = cudaMemcpyAsync(&active, &d_ctl->active_jobs, sizeof(unsigned),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_from_cuda(e);
    if (active == 0) break;
    if (timeout_ms > 0 && now_ms() - t0 > timeout_ms) {
      if (steps_run) *steps_run = launched;
      return MOTIF_ERR_TIMEOUT;
    }
  }
  if (steps_run) *steps_run = launched;
  return MOTIF_OK;
}

}  // namespace motif

using namespace motif;

namespace motif_api {

constexpr const char* kVersion = "motif-gb300 0.1 (sm_103a)";

int validate_args(int32_t n, int32_t t, int32_t l, int32_t d) {
  if (n < 1 || t < 1 || l < 1 || l > kMaxL || d < 0) return MOTIF_ERR_ARG;
  return MOTIF_OK;
}

int timeout_of(const motif_plan_s* p) { return p->opts.timeout_ms > 0 ? p->opts.timeout_ms : 60000; }

// Upper bound on steps for one job: every chunk needs at most n passes.
int max_steps_of(const motif_plan_s* p) {
  const uint64_t s = p->nchunks * (uint64_t)p->n + 2;
  return s > (uint64_t)(1 << 30) ? (1 << 30) : (int)s;
}

int ensure_out(motif_plan_s* p, int64_t need) {
  if (need <= p->out_cap) return MOTIF_OK;
  p->desc_out = nullptr;  // the descriptor names the output buffer
  plan_free(p, p->d_out, (size_t)p->out_cap * 8);
  p->d_out = (uint64_t*)plan_alloc(p, (size_t)need * 8);
  p->out_cap = p->d_out ? need : 0;
  return p->d_out ? MOTIF_OK : MOTIF_ERR_OOM;
}

int ensure_sort(motif_plan_s* p, int64_t cap) {
  const size_t need = sort_scratch_bytes(cap, p->sms);
  if (need <= p->sort_bytes) return MOTIF_OK;
  plan_free(p, p->d_sort, p->sort_bytes);
  p->d_sort = plan_alloc(p, need);
  p->sort_bytes = p->d_sort ? need : 0;
  return p->d_sort ? MOTIF_OK : MOTIF_ERR_OOM;
}

// The sort graph over (out, cap): the one-CTA sort, and, when `scratch` (sized for cap) is
// given, the multi-CTA sort under a conditional IF node that runs only when the count needs it.
// A count above cap (an overflowed search) is left as it is.
int ensure_sort_graph(motif_plan_s* p, uint64_t* out, int64_t cap, void* scratch) {
  if (p->g_sort && p->gs_out == out && p->gs_cap == cap && p->gs_scratch == scratch)
    return MOTIF_OK;
  if (p->g_sort) cudaGraphExecDestroy(p->g_sort);
  p->g_sort = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphNode_t last;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e == cudaSuccess)
    e = add_sort_nodes(g, nullptr, out, &p->d_state->out_count, cap, 2 * p->l, scratch, p->sms,
                       &last);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->g_sort, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    p->g_sort = nullptr;
    return status_from_cuda(e);
  }
  p->gs_out = out;
  p->gs_cap = cap;
  p->gs_scratch = scratch;
  return MOTIF_OK;
}

int check_alphabet(motif_plan_s* p) {
  if (!p->check_alpha) return MOTIF_OK;
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return status_from_cuda(e);
  p->check_alpha = false;
  if (err) {
    p->loaded = false;
    return MOTIF_ERR_ALPHABET;
  }
  return MOTIF_OK;
}

// Enqueues one search of the plan writing into (out, cap): descriptor, state reset, steps.
int enqueue_search(motif_plan_s* p, uint64_t* out, uint64_t cap, bool poll) {
  int rc = plan_ensure_buffers(p);
  if (rc) return rc;
  if (p->nchunks == 0) {
    cudaError_t e = cudaMemsetAsync(p->d_state, 0, sizeof(JobState), p->stream);
    return status_from_cuda(e);
  }
  if (p->bitmap) {  // all ones where (tile, sequence block) items AND their survivors in
    const int fill = p->tiled && p->seq_block > 0 ? 0xFF : 0;
    cudaError_t e = cudaMemsetAsync(p->d_bitmap, fill, p->bm_words * 4, p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
  }
  if (p->seeded) {
    rc = prepare_seed(p, p->stream);
    if (rc) return rc;
  }
  // Upload the descriptor when (out, cap) changed; it lives in pinned memory so the copy is
  // stream-ordered without blocking the host.
  if (p->desc_out != out || p->desc_cap != (int64_t)cap) {
    if (!p->h_desc) {  // the descriptor's place in the plan's pinned host block
      if (!p->h_res && !(p->h_res = take_result_block())) return MOTIF_ERR_OOM;
      p->h_desc = reinterpret_cast<JobDesc*>(reinterpret_cast<char*>(p->h_res) + kDescOffset);
    }
    cudaError_t e = cudaStreamSynchronize(p->stream);  // the previous upload has completed
    if (e != cudaSuccess) return status_from_cuda(e);
    fill_desc(p, p->h_desc, out, cap);
    if (p->kind == MOTIF_KERNEL_GROUP && !p->h_desc->ball) return MOTIF_ERR_CUDA;
    e = cudaMemcpyAsync(p->d_job, p->h_desc, sizeof(JobDesc), cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    p->desc_out = out;
    p->desc_cap = (int64_t)cap;
  }
  // Profiling aid: MOTIF_NO_GRAPH=1 launches the same step kernel directly (profilers do not
  // list kernels inside conditional graph nodes); the blocking path polls, the device path
  // launches the step bound blindly.
  static const bool no_graph = getenv("MOTIF_NO_GRAPH") != nullptr;
  if (no_graph || p->opts.launch == MOTIF_LAUNCH_DIRECT) {
    cudaError_t e = launch_init_steps(p->d_state, 1, p->d_ctl, 0, 0, 0, p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    return run_steps(p->lkind, p->p, p->d_job, p->d_state, 1, p->d_ctl, p->grid, p->block, p->smem,
                     max_steps_of(p), poll, timeout_of(p), p->stream, nullptr);
  }
  // One graph launch runs every step: init, then a while loop whose body is the step kernel.
  if (!p->g_steps) {
    // A tiled plan takes its whole range as one chunk, so its one pass is done in one step.
    const bool one_step = p->tiled && p->nchunks == 1;
    cudaError_t e = build_step_graph(p->lkind, p->p, p->d_job, p->d_state, 1, p->d_ctl, p->grid,
                                     p->block, p->smem, (unsigned)max_steps_of(p), 0, &p->g_steps,
                                     one_step);
    if (e != cudaSuccess) {
      p->g_steps = nullptr;
      return status_from_cuda(e);
    }
  }
  ++p->graph_searches;
  return status_from_cuda(cudaGraphLaunch(p->g_steps, p->stream));
}

__global__ void finalize_count_kernel(const int* err, const unsigned long long* count,
                                      int64_t* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = *err ? -1 : (int64_t)*count;
}

// Compacts the plan's bitmap into (out, cap) on its stream; the count goes to the job state.
int compact_bitmap(motif_plan_s* p, uint64_t* out, int64_t cap) {
  return status_from_cuda(launch_bitmap_compact(p->d_bitmap, p->bm_words, p->bm_base, out, cap,
                                                p->d_bm_scratch, &p->d_state->out_count,
                                                p->stream));
}

// motif_search with bitmap output: one search, then compactions of the same bitmap until the
// plan's buffer holds every code (no second search), then the copy to the caller.
int search_bitmap(motif_plan_s* p, uint64_t* out_codes, int64_t capacity, int64_t* out_count,
                  cudaEvent_t* ev, double t0) {
  cudaEventRecord(ev[0], p->stream);
  int rc = enqueue_search(p, p->d_out, (uint64_t)p->out_cap, true);
  if (rc) return rc;
  cudaEventRecord(ev[1], p->stream);
  cudaEventRecord(ev[2], p->stream);
  // One wait reads the count and, speculatively, the first codes (as the list path does).
  if (!p->h_res && !(p->h_res = take_result_block())) return MOTIF_ERR_OOM;
  unsigned long long found = 0;
  int64_t peek = 0;
  for (;;) {
    rc = compact_bitmap(p, p->d_out, p->out_cap);
    if (rc) return rc;
    peek = std::min<int64_t>(std::min<int64_t>(p->out_cap, capacity), kResultPeek);
    cudaError_t e = cudaMemcpyAsync(p->h_res, &p->d_state->out_count, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess && peek > 0)
      e = cudaMemcpyAsync(p->h_res + 1, p->d_out, (size_t)peek * 8, cudaMemcpyDeviceToHost,
                          p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    found = p->h_res[0];
    if (found <= (unsigned long long)p->out_cap) break;
    rc = ensure_out(p, (int64_t)found);
    if (rc) return rc;
  }
  cudaEventRecord(ev[3], p->stream);
  *out_count = (int64_t)found;
  rc = fold_event_quads(p);
  if (rc) return rc;
  p->stats.survivors = found;
  if ((int64_t)found > capacity) {
    p->stats.total_ms = now_ms() - t0;
    return MOTIF_ERR_CAPACITY;
  }
  if ((int64_t)found <= peek) {
    if (found) memcpy(out_codes, p->h_res + 1, (size_t)found * 8);
  } else {
    cudaError_t e = cudaMemcpyAsync(out_codes, p->d_out, found * 8, cudaMemcpyDeviceToHost,
                                    p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
  }
  p->stats.total_ms = now_ms() - t0;
  return MOTIF_OK;
}

}  // namespace motif_api

using namespace motif_api;

extern "C" {

const char* motif_version(void) { return kVersion; }

const char* motif_strerror(int status) {
  switch (status) {
    case MOTIF_OK: return "ok";
    case MOTIF_PENDING: return "pending";
    case MOTIF_ERR_ARG: return "invalid argument";
    case MOTIF_ERR_ALPHABET: return "character outside ACGTacgt";
    case MOTIF_ERR_CAPACITY: return "output capacity too small";
    case MOTIF_ERR_OOM: return "out of memory";
    case MOTIF_ERR_CUDA: return "CUDA error";
    case MOTIF_ERR_TIMEOUT: return "timed out";
    case MOTIF_ERR_BUSY: return "queue full";
    case MOTIF_ERR_STATE: return "invalid state for this call";
    case MOTIF_ERR_NOTFOUND: return "unknown job";
    default: return "unknown status";
  }
}

void motif_opts_default(motif_opts* o) {
  if (o) memset(o, 0, sizeof(*o));
}

}  // extern "C"

namespace motif {

int plan_init_host(motif_plan_s* p, int32_t n, int32_t t, int32_t l, int32_t d,
                   const motif_opts* opts) {
  int rc = validate_args(n, t, l, d);
  if (rc) return rc;
  if (opts) p->opts = *opts;
  p->n = n; p->t = t; p->l = l; p->d = d;
  p->W = t - l + 1;
  p->wstride = p->W > 0 ? (p->W + kWinAlign - 1) / kWinAlign * kWinAlign : 0;
  const uint64_t space = 1ull << (2 * l);
  p->lo = p->opts.range_lo;
  p->hi = p->opts.range_hi ? p->opts.range_hi : space;
  if (p->hi > space || p->lo > p->hi) return MOTIF_ERR_ARG;
  if (p->opts.launch != MOTIF_LAUNCH_GRAPH && p->opts.launch != MOTIF_LAUNCH_DIRECT)
    return MOTIF_ERR_ARG;
  p->stream = (cudaStream_t)p->opts.stream;
  // (one attribute query: a full cudaGetDeviceProperties costs more than the rest of a small
  // plan's set-up)
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MOTIF_ERR_CUDA;
  }
  return MOTIF_OK;
}

int plan_configure_host(motif_plan_s* p) {
  if (p->opts.kernel == MOTIF_KERNEL_AUTO) tune_lookup(p, &p->opts);
  return plan_configure(p);
}

}  // namespace motif

extern "C" {

int motif_plan_create(int32_t n, int32_t t, int32_t l, int32_t d, const motif_opts* opts,
                      motif_plan* out) {
  if (!out) return MOTIF_ERR_ARG;
  *out = nullptr;
  motif_plan_s* p = new (std::nothrow) motif_plan_s();
  if (!p) return MOTIF_ERR_OOM;
  int rc = plan_init_host(p, n, t, l, d, opts);
  if (rc) { delete p; return rc; }
  const size_t chars = (size_t)n * t;
  const size_t wins = (size_t)n * std::max(p->wstride, 0);
  p->d_chars = (char*)plan_alloc(p, chars);
  p->chars_bytes = chars;
  p->d_planes = wins ? (uint2*)plan_alloc(p, wins * 8) : nullptr;
  p->d_codes = wins ? (uint64_t*)plan_alloc(p, wins * 8) : nullptr;
  p->d_err = (int*)plan_alloc(p, sizeof(int));
  p->d_job = (JobDesc*)plan_alloc(p, sizeof(JobDesc));
  p->d_state = (JobState*)plan_alloc(p, sizeof(JobState));
  p->d_ctl = (StepCtl*)plan_alloc(p, sizeof(StepCtl));
  p->d_total = (unsigned long long*)plan_alloc(p, sizeof(unsigned long long));
  if (!p->d_chars || (wins && (!p->d_planes || !p->d_codes)) || !p->d_err || !p->d_job ||
      !p->d_state || !p->d_ctl || !p->d_total) {
    motif_plan_destroy(p);
    return MOTIF_ERR_OOM;
  }
  rc = plan_configure_host(p);
  if (rc) { motif_plan_destroy(p); return rc; }
  *out = p;
  return MOTIF_OK;
}

static void free_ragged(motif_plan p) {
  plan_free(p, p->d_lens, sizeof(int32_t) * (size_t)p->n);
  plan_free(p, p->d_wrow, sizeof(int32_t) * (size_t)p->n);
  plan_free(p, p->d_valid, (size_t)p->n * (size_t)std::max(p->wstride, 0));
  plan_free(p, p->d_empty, sizeof(int));
  p->d_lens = p->d_wrow = nullptr;
  p->d_valid = nullptr;
  p->d_empty = nullptr;
}


void motif_plan_destroy(motif_plan p) {
  if (!p) return;
  DeviceGuard g(p->device);
  cudaStreamSynchronize(p->stream);
  free_queues(p);
  plan_free(p, p->d_chars, p->chars_bytes);
  const size_t wins = (size_t)p->n * std::max(p->wstride, 0);
  plan_free(p, p->d_planes, wins * 8);
  plan_free(p, p->d_codes, wins * 8);
  plan_free(p, p->d_err, sizeof(int));
  plan_free(p, p->d_job, sizeof(JobDesc));
  plan_free(p, p->d_state, sizeof(JobState));
  plan_free(p, p->d_ctl, sizeof(StepCtl));
  plan_free(p, p->d_total, sizeof(unsigned long long));
  plan_free(p, p->d_out, (size_t)p->out_cap * 8);
  plan_free(p, p->d_sort, p->sort_bytes);
  free_bitmap(p);
  free_seed(p);
  free_ragged(p);
  cudaStreamSynchronize(p->stream);
  for (cudaEvent_t ev : p->evq)
    if (ev) cudaEventDestroy(ev);
  invalidate_graphs(p);
  free(p->h_chars);
  if (p->h_chars_done) cudaEventDestroy(p->h_chars_done);
  give_result_block(p->h_res);
  delete p;
}

// Packs the plan's characters.  checked: validated on the host already (no device check);
// otherwise the device check's flag is read now (sync_check) or by the next call that waits.
// The flag is cleared either way: the device search path reports it.
static int load_common(motif_plan p, bool sync_check, bool checked = false) {
  if (p->ragged) p->desc_out = nullptr;  // the descriptor names the ragged-row buffers
  p->ragged = false;
  p->empty_row = false;
  cudaError_t e = cudaMemsetAsync(p->d_err, 0, sizeof(int), p->stream);
  if (e == cudaSuccess)
    e = launch_pack(p->d_chars, p->t, p->n, p->t, p->l, p->wstride, p->d_planes, p->d_codes,
                    checked ? nullptr : p->d_err, p->stream);
  if (e != cudaSuccess) return status_from_cuda(e);
  p->loaded = true;
  p->check_alpha = !checked;
  return sync_check && !checked ? check_alphabet(p) : MOTIF_OK;
}

// Host loads up to this size are validated on the host while they are copied into the plan's
// staging buffer: a few microseconds, against a wait for the device's check.
constexpr size_t kHostCheckBytes = (size_t)1 << 16;

// Copies the n rows into the plan's staging buffer; false if a character is outside
// ACGTacgt.
static bool stage_checked(motif_plan_s* p, const char* seqs, int64_t stride) {
  static const std::array<uint8_t, 256> valid = [] {
    std::array<uint8_t, 256> a{};
    for (unsigned char c : {'A', 'C', 'G', 'T', 'a', 'c', 'g', 't'}) a[c] = 1;
    return a;
  }();
  unsigned bad = 0;
  for (int r = 0; r < p->n; ++r) {
    const unsigned char* src = reinterpret_cast<const unsigned char*>(seqs) + (size_t)r * stride;
    char* dst = p->h_chars + (size_t)r * p->t;
    for (int c = 0; c < p->t; ++c) {
      bad |= valid[src[c]] ^ 1u;
      dst[c] = (char)src[c];
    }
  }
  return bad == 0;
}

int motif_load_seqs(motif_plan p, const char* seqs, int64_t stride) {
  if (!p || !seqs || stride < p->t) return MOTIF_ERR_ARG;
  DeviceGuard g(p->device);
  p->loaded = false;
  const size_t bytes = (size_t)p->n * p->t;
  if (bytes <= kHostCheckBytes) {
    cudaError_t e = cudaSuccess;
    if (!p->h_chars_done) {
      e = cudaEventCreateWithFlags(&p->h_chars_done, cudaEventDisableTiming);
      if (e != cudaSuccess) {
        p->h_chars_done = nullptr;
        return status_from_cuda(e);
      }
    } else {
      e = cudaEventSynchronize(p->h_chars_done);  // the previous upload has read the staging
      if (e != cudaSuccess) return status_from_cuda(e);
    }
    // plain host memory: pinning it would cost more than it saves on an upload of a few
    // kilobytes, for plans that live for one search
    if (!p->h_chars && !(p->h_chars = (char*)malloc(bytes))) return MOTIF_ERR_OOM;
    if (!stage_checked(p, seqs, stride)) return MOTIF_ERR_ALPHABET;
    e = cudaMemcpyAsync(p->d_chars, p->h_chars, bytes, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaEventRecord(p->h_chars_done, p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    return load_common(p, false, true);  // validated above
  }
  cudaError_t e = cudaMemcpy2DAsync(p->d_chars, p->t, seqs, (size_t)stride, p->t, p->n,
                                    cudaMemcpyHostToDevice, p->stream);
  if (e != cudaSuccess) return status_from_cuda(e);
  return load_common(p, true);
}

int motif_load_seqs_device(motif_plan p, const char* d_seqs, int64_t stride) {
  if (!p || !d_seqs || stride < p->t) return MOTIF_ERR_ARG;
  DeviceGuard g(p->device);
  p->loaded = false;
  cudaError_t e = cudaMemcpy2DAsync(p->d_chars, p->t, d_seqs, (size_t)stride, p->t, p->n,
                                    cudaMemcpyDeviceToDevice, p->stream);
  if (e != cudaSuccess) return status_from_cuda(e);
  return load_common(p, false);
}

int motif_load_seqs_var(motif_plan p, const char* seqs, int64_t stride, const int32_t* lengths,
                        int32_t mask_unknown) {
  if (!p || !seqs || !lengths || stride < 1) return MOTIF_ERR_ARG;
  for (int r = 0; r < p->n; ++r)
    if (lengths[r] < 0 || lengths[r] > p->t || lengths[r] > stride) return MOTIF_ERR_ARG;
  DeviceGuard g(p->device);
  p->loaded = false;
  if (!p->d_lens) {
    p->d_lens = (int32_t*)plan_alloc(p, sizeof(int32_t) * (size_t)p->n);
    p->d_wrow = (int32_t*)plan_alloc(p, sizeof(int32_t) * (size_t)p->n);
    p->d_valid = p->wstride > 0 ? (uint8_t*)plan_alloc(p, (size_t)p->n * p->wstride) : nullptr;
    p->d_empty = (int*)plan_alloc(p, sizeof(int));
    if (!p->d_lens || !p->d_wrow || (p->wstride > 0 && !p->d_valid) || !p->d_empty) {
      free_ragged(p);
      return MOTIF_ERR_OOM;
    }
  }
  // Rows staged on the host at the plan's stride t (bytes past a row's length are never read
  // as part of a valid window).
  std::vector<char> rows((size_t)p->n * p->t, 'A');
  std::vector<int32_t> wrow(p->n);
  for (int r = 0; r < p->n; ++r) {
    memcpy(rows.data() + (size_t)r * p->t, seqs + (size_t)r * stride, (size_t)lengths[r]);
    wrow[r] = std::max(0, lengths[r] - p->l + 1);
  }
  cudaError_t e = cudaMemcpyAsync(p->d_chars, rows.data(), rows.size(), cudaMemcpyHostToDevice,
                                  p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_lens, lengths, sizeof(int32_t) * p->n, cudaMemcpyHostToDevice,
                        p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_wrow, wrow.data(), sizeof(int32_t) * p->n, cudaMemcpyHostToDevice,
                        p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_err, 0, sizeof(int), p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_empty, 0, sizeof(int), p->stream);
  if (e == cudaSuccess && p->wstride > 0)
    e = launch_pack_var(p->d_chars, p->t, p->n, p->l, p->wstride, p->d_lens,
                        mask_unknown ? 1 : 0, p->d_planes, p->d_codes, p->d_valid, p->d_err,
                        p->d_empty, p->stream);
  int flags[2] = {0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&flags[0], p->d_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&flags[1], p->d_empty, sizeof(int), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return status_from_cuda(e);
  if (flags[0]) return MOTIF_ERR_ALPHABET;
  p->ragged = true;
  p->empty_row = flags[1] != 0;
  p->desc_out = nullptr;  // the descriptor names the ragged-row buffers
  p->check_alpha = false;
  p->loaded = true;
  return MOTIF_OK;
}



int motif_search(motif_plan p, uint64_t* out_codes, int64_t capacity, int64_t* out_count) {
  if (!p || !out_count || capacity < 0 || (capacity > 0 && !out_codes)) return MOTIF_ERR_ARG;
  if (!p->loaded) return MOTIF_ERR_STATE;
  DeviceGuard g(p->device);
  const double t0 = now_ms();
  int rc = check_alphabet(p);
  if (rc) return rc;
  p->stats.candidates = p->hi - p->lo;
  p->stats.kernel = p->tiled ? MOTIF_KERNEL_TILED : p->kind;
  p->stats.grid = p->grid;
  p->stats.block = p->block;
  p->stats.smem_bytes = (int32_t)p->smem;
  *out_count = 0;
  if (p->W <= 0 || p->hi <= p->lo || p->empty_row) {  // no windows, an empty range, or a row
                                                      // with no valid window: nothing survives
    p->stats.survivors = 0;
    p->stats.search_ms = p->stats.sort_ms = 0;
    p->stats.total_ms = now_ms() - t0;
    return MOTIF_OK;
  }
  cudaEvent_t* ev = next_event_quad(p);
  if (!ev) return MOTIF_ERR_CUDA;
  if (p->bitmap) return search_bitmap(p, out_codes, capacity, out_count, ev, t0);
  // List output: the steps and the sort graph run back to back, then one wait reads the final
  // count and, speculatively, the first codes.  A count above the buffer means the search
  // overflowed it (the sort leaves such a count alone): the buffer grows and the search reruns.
  if (!p->h_res && !(p->h_res = take_result_block())) return MOTIF_ERR_OOM;
  unsigned long long final_count = 0;
  int64_t peek = 0;
  bool sorted = false;  // the graph's multi-CTA branch covers every count up to the buffer's
  for (;;) {
    rc = plan_ensure_buffers(p);
    if (rc) return rc;
    // The graph holds the multi-CTA sort (one more node, which runs even when it returns at
    // once, and needs scratch sized for the buffer) only once the plan's previous result needed
    // it; until then the one-CTA sort alone, and a larger result is sorted below with one more
    // wait.
    sorted = p->out_cap <= 4096 ||
             (p->stats.survivors > 4096 && p->d_sort &&
              p->sort_bytes >= sort_scratch_bytes(p->out_cap, p->sms));
    rc = ensure_sort_graph(p, p->d_out, p->out_cap, sorted ? p->d_sort : nullptr);
    if (rc) return rc;
    cudaEventRecord(ev[0], p->stream);
    rc = enqueue_search(p, p->d_out, (uint64_t)p->out_cap, true);
    if (rc) return rc;
    cudaEventRecord(ev[1], p->stream);
    cudaEventRecord(ev[2], p->stream);
    cudaError_t e = cudaGraphLaunch(p->g_sort, p->stream);
    note_launches(1);
    cudaEventRecord(ev[3], p->stream);
    peek = std::min<int64_t>(std::min<int64_t>(p->out_cap, capacity), kResultPeek);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->h_res, &p->d_state->out_count, sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess && peek > 0)
      e = cudaMemcpyAsync(p->h_res + 1, p->d_out, (size_t)peek * 8, cudaMemcpyDeviceToHost,
                          p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    final_count = p->h_res[0];
    if (final_count <= (unsigned long long)p->out_cap) break;
    rc = ensure_out(p, (int64_t)std::max<unsigned long long>(final_count,
                                                             2 * (unsigned long long)p->out_cap));
    if (rc) return rc;
  }
  if (final_count > 4096 && !sorted) {  // more codes than the one-CTA sort takes: sort them now
    rc = ensure_sort(p, p->out_cap);
    if (rc) return rc;
    cudaError_t e = launch_sort_unique(p->d_out, &p->d_state->out_count, p->out_cap, 2 * p->l,
                                       p->d_sort, p->sms, (long long)final_count, p->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->h_res, &p->d_state->out_count, sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    final_count = p->h_res[0];
    peek = 0;  // the codes read back with the count were not sorted yet
  }
  *out_count = (int64_t)final_count;
  rc = fold_event_quads(p);
  if (rc) return rc;
  p->stats.survivors = final_count;
  if ((int64_t)final_count > capacity) {
    p->stats.total_ms = now_ms() - t0;
    return MOTIF_ERR_CAPACITY;
  }
  if ((int64_t)final_count <= peek) {
    if (final_count) memcpy(out_codes, p->h_res + 1, (size_t)final_count * 8);
  } else {
    cudaError_t e = cudaMemcpyAsync(out_codes, p->d_out, final_count * 8, cudaMemcpyDeviceToHost,
                                    p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
  }
  p->stats.total_ms = now_ms() - t0;
  return MOTIF_OK;
}

int motif_search_device(motif_plan p, uint64_t* d_out_codes, int64_t capacity,
                        int64_t* d_out_count) {
  if (!p || !d_out_count || capacity < 0 || (capacity > 0 && !d_out_codes)) return MOTIF_ERR_ARG;
  if (!p->loaded) return MOTIF_ERR_STATE;
  DeviceGuard g(p->device);
  int rc = MOTIF_OK;
  p->stats.candidates = p->hi - p->lo;
  p->stats.kernel = p->tiled ? MOTIF_KERNEL_TILED : p->kind;
  p->stats.grid = p->grid;
  p->stats.block = p->block;
  p->stats.smem_bytes = (int32_t)p->smem;
  if (capacity > 4096 && !p->bitmap) {
    rc = ensure_sort(p, capacity);
    if (rc) return rc;
  }
  if (p->W <= 0 || p->hi <= p->lo || p->empty_row) {
    cudaError_t e = cudaMemsetAsync(p->d_state, 0, sizeof(JobState), p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
  } else if (p->bitmap) {
    cudaEvent_t* ev = next_event_quad(p);
    if (!ev) return MOTIF_ERR_CUDA;
    cudaEventRecord(ev[0], p->stream);
    rc = enqueue_search(p, d_out_codes, (uint64_t)capacity, false);
    if (rc) return rc;
    cudaEventRecord(ev[1], p->stream);
    cudaEventRecord(ev[2], p->stream);
    rc = compact_bitmap(p, d_out_codes, capacity);
    cudaEventRecord(ev[3], p->stream);
    if (rc) return rc;
  } else {
    cudaEvent_t* ev = next_event_quad(p);
    if (!ev) return MOTIF_ERR_CUDA;
    cudaEventRecord(ev[0], p->stream);
    rc = enqueue_search(p, d_out_codes, (uint64_t)capacity, false);
    if (rc) return rc;
    cudaEventRecord(ev[1], p->stream);
    cudaEventRecord(ev[2], p->stream);
    rc = ensure_sort_graph(p, d_out_codes, capacity, p->d_sort);  // sized for capacity above
    if (rc) return rc;
    cudaError_t e = cudaGraphLaunch(p->g_sort, p->stream);
    note_launches(1);
    cudaEventRecord(ev[3], p->stream);
    if (e != cudaSuccess) return status_from_cuda(e);
  }
  note_launches(1);
  finalize_count_kernel<<<1, 32, 0, p->stream>>>(p->d_err, &p->d_state->out_count, d_out_count);
  return status_from_cuda(cudaGetLastError());
}

int motif_seed_count(motif_plan p, uint64_t* out) {
  if (!p || !out) return MOTIF_ERR_ARG;
  if (!p->loaded || !p->seeded) return MOTIF_ERR_STATE;
  DeviceGuard g(p->device);
  int rc = check_alphabet(p);
  if (rc) return rc;
  *out = 0;
  if (p->W <= 0 || p->hi <= p->lo) return MOTIF_OK;
  rc = plan_ensure_buffers(p);
  if (rc) return rc;
  rc = prepare_seed(p, p->stream);
  if (rc) return rc;
  unsigned long long n = 0;
  cudaError_t e = launch_bitmap_count(p->d_seed, p->seed_words, p->d_seed_scratch,
                                      p->d_seed_count, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&n, p->d_seed_count, sizeof(n), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return status_from_cuda(e);
  *out = n;
  return MOTIF_OK;
}

int motif_count_compares(motif_plan p, uint64_t* out) {
  if (!p || !out) return MOTIF_ERR_ARG;
  if (!p->loaded) return MOTIF_ERR_STATE;
  DeviceGuard g(p->device);
  int rc = check_alphabet(p);
  if (rc) return rc;
  *out = 0;
  if (p->W <= 0 || p->hi <= p->lo) return MOTIF_OK;
  JobDesc jd;
  fill_desc(p, &jd, p->d_out, p->out_cap);
  unsigned long long total = 0;
  cudaError_t e = cudaMemcpyAsync(p->d_job, &jd, sizeof(jd), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_total, 0, sizeof(unsigned long long), p->stream);
  if (e == cudaSuccess) e = launch_count(p->d_job, p->d_total, p->sms * 8, 256, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&total, p->d_total, sizeof(total), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return status_from_cuda(e);
  *out = total;
  p->stats.algorithmic_compares = total;
  return MOTIF_OK;
}

int motif_count_work(motif_plan p, uint64_t* compares, uint64_t* unit_steps) {
  if (!p) return MOTIF_ERR_ARG;
  if (!p->loaded) return MOTIF_ERR_STATE;
  DeviceGuard g(p->device);
  uint64_t c = 0;
  int rc = motif_count_compares(p, &c);
  if (rc) return rc;
  if (compares) *compares = c;
  if (!unit_steps) return MOTIF_OK;
  if (cand_like(p->kind) || p->W <= 0 || p->hi <= p->lo) {
    *unit_steps = cand_like(p->kind) ? c : 0;
    return MOTIF_OK;
  }
  JobDesc jd;
  fill_desc(p, &jd, p->d_out, p->out_cap);
  unsigned long long total = 0;
  cudaError_t e = cudaMemcpyAsync(p->d_job, &jd, sizeof(jd), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->d_total, 0, sizeof(unsigned long long), p->stream);
  if (e == cudaSuccess) e = launch_count_group(p->d_job, p->p, p->d_total, p->sms * 8, 256, p->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&total, p->d_total, sizeof(total), cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return status_from_cuda(e);
  *unit_steps = total;
  return MOTIF_OK;
}

int motif_count_tiled_work(motif_plan p, uint64_t* units) {
  if (!p || !units) return MOTIF_ERR_ARG;
  if (!p->loaded) return MOTIF_ERR_STATE;
  if (p->lkind != kKindTiled) return MOTIF_ERR_STATE;  // a plan that runs the whole-tile pass
  DeviceGuard g(p->device);
  int rc = check_alphabet(p);
  if (rc) return rc;
  for (int i = 0; i < kTiledUnits; ++i) units[i] = 0;
  if (p->W <= 0 || p->hi <= p->lo || p->nchunks == 0 || p->empty_row) return MOTIF_OK;
  rc = plan_ensure_buffers(p);
  if (rc) return rc;
  // One search by the counting instantiation of the tiled kernel, from its own descriptor (the
  // plan's uploaded one stays as it is), into the plan's output buffers.
  const size_t bytes = sizeof(JobDesc) + 16 * kTiledUnits;
  char* scratch = (char*)plan_alloc(p, bytes);
  if (!scratch) return MOTIF_ERR_OOM;
  JobDesc* d_jd = reinterpret_cast<JobDesc*>(scratch);
  unsigned long long* d_units = reinterpret_cast<unsigned long long*>(scratch + sizeof(JobDesc));
  JobDesc jd;
  fill_desc(p, &jd, p->d_out, (uint64_t)p->out_cap);
  jd.units = d_units;
  unsigned long long h[kTiledUnits] = {};
  cudaError_t e = cudaMemcpyAsync(d_jd, &jd, sizeof(jd), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_units, 0, 8 * kTiledUnits, p->stream);
  if (e == cudaSuccess && p->bitmap) e = cudaMemsetAsync(p->d_bitmap, 0, p->bm_words * 4, p->stream);
  if (e == cudaSuccess) e = step_kernel_attrs(kKindTiledCount, p->p, p->smem);
  if (e == cudaSuccess) e = launch_init_steps(p->d_state, 1, p->d_ctl, 0, 0, 0, p->stream);
  if (e == cudaSuccess) {
    rc = run_steps(kKindTiledCount, p->p, d_jd, p->d_state, 1, p->d_ctl, p->grid, p->block,
                   p->smem, max_steps_of(p), true, timeout_of(p), p->stream, nullptr);
    if (rc == MOTIF_OK)
      e = cudaMemcpyAsync(h, d_units, sizeof(h), cudaMemcpyDeviceToHost, p->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  plan_free(p, scratch, bytes);
  if (e != cudaSuccess) return status_from_cuda(e);
  if (rc) return rc;
  for (int i = 0; i < kTiledUnits; ++i) units[i] = h[i];
  return MOTIF_OK;
}

int motif_stats(motif_plan p, motif_stats_t* s) {
  if (!p || !s) return MOTIF_ERR_ARG;
  DeviceGuard g(p->device);
  int rc = fold_event_quads(p);
  *s = p->stats;
  s->device_bytes = p->device_bytes;
  s->search_ms_sum = p->sum_search_ms;
  s->sort_ms_sum = p->sum_sort_ms;
  s->searches = p->sum_searches;
  p->sum_search_ms = p->sum_sort_ms = 0;
  p->sum_searches = 0;
  return rc;
}

uint64_t motif_kernel_launches(void) { return launches_total(); }

int motif_shard_range(uint64_t total, int32_t rank, int32_t world, const double* weights,
                      uint64_t* lo, uint64_t* hi) {
  if (world < 1 || rank < 0 || rank >= world || !lo || !hi) return MOTIF_ERR_ARG;
  double sum = 0;
  for (int r = 0; r < world; ++r) {
    const double w = weights ? weights[r] : 1.0;
    if (!(w >= 0)) return MOTIF_ERR_ARG;
    sum += w;
  }
  if (!(sum > 0)) return MOTIF_ERR_ARG;
  // Boundary r at floor(total * (w_0 + ... + w_{r-1}) / sum); the last one is exactly total.
  // Equal weights: exact in 128-bit integers.  Given weights: IEEE double arithmetic, which
  // rounds alike on every host, and is monotone in r, so the ranges stay contiguous.
  auto cut = [&](int r) -> uint64_t {
    if (r >= world) return total;
    if (!weights) return (uint64_t)((unsigned __int128)total * (uint32_t)r / (uint32_t)world);
    double acc = 0;
    for (int i = 0; i < r; ++i) acc += weights[i];
    if (acc >= sum) return total;  // only zero weights follow: they get empty ranges
    const double v = (double)total * (acc / sum);
    if (!(v < 18446744073709551616.0)) return total;
    const uint64_t c = (uint64_t)v;
    return c > total ? total : c;
  };
  *lo = cut(rank);
  *hi = cut(rank + 1);
  if (*hi < *lo) *hi = *lo;
  return MOTIF_OK;
}

int motif_encode(const char* s, int32_t l, uint64_t* code) {
  if (!s || !code || l < 1 || l > kMaxL) return MOTIF_ERR_ARG;
  uint64_t c = 0;
  for (int i = 0; i < l; ++i) {
    int v;
    switch (s[i]) {
      case 'A': case 'a': v = 0; break;
      case 'C': case 'c': v = 1; break;
      case 'G': case 'g': v = 2; break;
      case 'T': case 't': v = 3; break;
      default: return MOTIF_ERR_ALPHABET;
    }
    c = (c << 2) | (uint64_t)v;
  }
  *code = c;
  return MOTIF_OK;
}

int motif_decode(uint64_t code, int32_t l, char* out) {
  if (!out || l < 1 || l > kMaxL) return MOTIF_ERR_ARG;
  if (l < 32 && (code >> (2 * l)) != 0) return MOTIF_ERR_ARG;
  static const char kB[4] = {'A', 'C', 'G', 'T'};
  for (int i = 0; i < l; ++i) out[i] = kB[(code >> (2 * (l - 1 - i))) & 3u];
  return MOTIF_OK;
}

}  // extern "C"

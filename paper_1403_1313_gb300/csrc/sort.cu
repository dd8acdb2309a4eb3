// K2: sort and de-duplicate the accepted codes.
//
// The search appends accepted codes in whatever order warps finish.  The result is returned
// ascending (which, with the code layout, is lexicographic order of the l-mers) and free of
// duplicates.  Every kernel here reads the element count from device memory, so the whole
// sequence can be enqueued without the host knowing how many codes were accepted:
//   - up to kSmallMax codes: one CTA sorts them in shared memory (bitonic network) and drops
//     repeats;
//   - above that: a stable least-significant-digit radix sort with 8-bit digits (per-CTA
//     histograms, one global digit-major scan, stable scatter ranked with warp match masks),
//     then a keep-flag compaction of repeats.
// Each path returns at once when the count belongs to the other path (or exceeds `cap`).
#include <cooperative_groups.h>

#include "motif_internal.h"

namespace cg = cooperative_groups;

namespace motif {
namespace {

constexpr int kSmallMax = 4096;
constexpr int kSmallThreads = 1024;
constexpr int kRadixThreads = 256;
constexpr int kRadixBits = 8;
constexpr int kDigits = 1 << kRadixBits;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long read_count(const unsigned long long* c) {
  return *reinterpret_cast<const volatile unsigned long long*>(c);
}

// ---- small path ----------------------------------------------------------------------------

// One CTA sorts codes[0 .. *count) in shared memory and drops repeats (a no-op unless
// 1 < *count <= min(kSmallMax, cap)).
__device__ void small_sort_block(uint64_t* codes, unsigned long long* count, long long cap,
                                 unsigned long long n) {
  __shared__ uint64_t a[kSmallMax];
  __shared__ unsigned warp_tot[kSmallThreads / 32];
  if (n <= 1 || n > (unsigned long long)kSmallMax || n > (unsigned long long)cap) return;
  int size = 2;
  while ((unsigned long long)size < n) size <<= 1;
  for (int i = threadIdx.x; i < size; i += blockDim.x) a[i] = (unsigned long long)i < n ? codes[i] : ~0ull;
  __syncthreads();
  // Bitonic sorting network over `size` (a power of two) elements.
  for (int k = 2; k <= size; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < size; i += blockDim.x) {
        const int p = i ^ j;
        if (p > i) {
          const bool up = (i & k) == 0;
          const uint64_t x = a[i], y = a[p];
          if ((x > y) == up) { a[i] = y; a[p] = x; }
        }
      }
      __syncthreads();
    }
  }
  // Keep the first of each run of equal codes: each thread owns kSmallMax/kSmallThreads slots.
  const int per = kSmallMax / kSmallThreads;
  const int first = threadIdx.x * per;
  unsigned keep = 0;
  for (int q = 0; q < per; ++q) {
    const int i = first + q;
    if ((unsigned long long)i < n && (i == 0 || a[i] != a[i - 1])) keep |= 1u << q;
  }
  const unsigned mine = __popc(keep);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned incl = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  unsigned before = 0, total = 0;
  for (int w = 0; w < kSmallThreads / 32; ++w) {
    if (w < warp) before += warp_tot[w];
    total += warp_tot[w];
  }
  unsigned pos = before + incl - mine;
  for (int q = 0; q < per; ++q)
    if (keep & (1u << q)) codes[pos++] = a[first + q];
  __syncthreads();
  if (threadIdx.x == 0) *count = total;
}

__global__ void __launch_bounds__(kSmallThreads) small_sort_kernel(uint64_t* codes,
                                                                   unsigned long long* count,
                                                                   long long cap,
                                                                   cudaGraphConditionalHandle cond,
                                                                   int use_cond) {
  const unsigned long long n = read_count(count);
  if (use_cond && threadIdx.x == 0)  // inside a graph: run the multi-CTA path only when needed
    cudaGraphSetConditional(cond, (n > (unsigned long long)kSmallMax && n <= (unsigned long long)cap) ? 1u : 0u);
  small_sort_block(codes, count, cap, n);
}

// Many jobs' small lists at once: CTA b sorts task b's codes.
__global__ void __launch_bounds__(kSmallThreads) small_sort_tasks_kernel(const SortTask* tasks) {
  const SortTask t = tasks[blockIdx.x];
  small_sort_block(t.codes, t.count, t.cap, read_count(t.count));
}

// ---- large path: LSD radix sort --------------------------------------------------------------

__device__ __forceinline__ bool large_active(unsigned long long n, long long cap) {
  return n > (unsigned long long)kSmallMax && n <= (unsigned long long)cap;
}

__device__ __forceinline__ void segment(unsigned long long n, unsigned long long& b,
                                        unsigned long long& e) {
  const unsigned long long per = (n + gridDim.x - 1) / gridDim.x;
  b = per * blockIdx.x;
  e = b + per;
  if (b > n) b = n;
  if (e > n) e = n;
}

// The radix sort's phases, as device functions of one CTA (blockIdx.x of gridDim.x CTAs, or the
// CTA alone for the scans).  The per-phase kernels below and the single cooperative kernel run
// the same phases; n is the count read at the start.

// Per-CTA digit counts of keys[segment], into hist[digit * gridDim.x + cta].
__device__ void hist_phase(const uint64_t* __restrict__ keys, unsigned long long n, int shift,
                           unsigned* __restrict__ hist) {
  __shared__ unsigned h[kDigits];
  for (int i = threadIdx.x; i < kDigits; i += blockDim.x) h[i] = 0;
  __syncthreads();
  unsigned long long b, e;
  segment(n, b, e);
  for (unsigned long long i = b + threadIdx.x; i < e; i += blockDim.x)
    atomicAdd(&h[(keys[i] >> shift) & (kDigits - 1)], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kDigits; i += blockDim.x) hist[(size_t)i * gridDim.x + blockIdx.x] = h[i];
  __syncthreads();
}

// Exclusive scan of `len` counters in place by one CTA of kRadixThreads threads.
__device__ void scan_phase(unsigned* __restrict__ v, int len) {
  __shared__ unsigned warp_tot[kRadixThreads / 32];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < len; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const unsigned x = i < len ? v[i] : 0;
    unsigned incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned before = 0, total = 0;
    for (int w = 0; w < kRadixThreads / 32; ++w) {
      if (w < warp) before += warp_tot[w];
      total += warp_tot[w];
    }
    if (i < len) v[i] = carry + before + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
}

// Exclusive scan of a digit-major histogram hist[digit * ctas + cta], taken in (digit, cta)
// order: thread `digit` sums its row, the CTA scans the row totals, and each thread rewrites its
// row as running offsets from its digit's base.  One CTA of kDigits threads.
__device__ void hist_scan_phase(unsigned* __restrict__ hist, int ctas) {
  __shared__ unsigned warp_tot[kDigits / 32];
  const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
  unsigned* row = hist + (size_t)d * ctas;
  unsigned tot = 0;
#pragma unroll 8
  for (int c = 0; c < ctas; ++c) tot += row[c];
  unsigned incl = tot;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  unsigned run = incl - tot;
  for (int w = 0; w < warp; ++w) run += warp_tot[w];
#pragma unroll 8
  for (int c = 0; c < ctas; ++c) {
    const unsigned x = row[c];
    row[c] = run;
    run += x;
  }
  __syncthreads();
}

// Stable scatter of keys[segment] by digit, from the CTA's scanned histogram column.
__device__ void scatter_phase(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst,
                              unsigned long long n, int shift,
                              const unsigned* __restrict__ offsets) {
  constexpr int kWarps = kRadixThreads / 32;
  __shared__ unsigned base[kDigits];
  __shared__ unsigned warp_cnt[kWarps][kDigits];
  __shared__ unsigned chunk_tot[kDigits];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offsets[(size_t)tid * gridDim.x + blockIdx.x];  // kRadixThreads == kDigits
  unsigned long long b, e;
  segment(n, b, e);
  const unsigned lt_mask = (1u << lane) - 1;
  for (unsigned long long c = b; c < e; c += kRadixThreads) {
    for (int w = 0; w < kWarps; ++w) warp_cnt[w][tid] = 0;
    __syncthreads();
    const unsigned long long i = c + tid;
    const bool valid = i < e;
    const uint64_t key = valid ? src[i] : 0;
    const unsigned digit = valid ? (unsigned)((key >> shift) & (kDigits - 1)) : kDigits;
    const unsigned peers = __match_any_sync(kFull, digit);
    const unsigned rank = __popc(peers & lt_mask);
    if (valid && rank == 0) warp_cnt[warp][digit] = __popc(peers);
    __syncthreads();
    {  // exclusive prefix over warps for digit `tid`
      unsigned acc = 0;
      for (int w = 0; w < kWarps; ++w) {
        const unsigned x = warp_cnt[w][tid];
        warp_cnt[w][tid] = acc;
        acc += x;
      }
      chunk_tot[tid] = acc;
    }
    __syncthreads();
    if (valid) dst[base[digit] + warp_cnt[warp][digit] + rank] = key;
    __syncthreads();
    base[tid] += chunk_tot[tid];
    __syncthreads();
  }
}

// Keep flags: the CTA's count of first-of-run elements.
__device__ void unique_count_phase(const uint64_t* __restrict__ keys, unsigned long long n,
                                   unsigned* __restrict__ per_cta) {
  __shared__ unsigned tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  unsigned long long b, e;
  segment(n, b, e);
  unsigned mine = 0;
  for (unsigned long long i = b + threadIdx.x; i < e; i += blockDim.x)
    mine += (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
  atomicAdd(&tot, mine);
  __syncthreads();
  if (threadIdx.x == 0) per_cta[blockIdx.x] = tot;
}

// The CTA's first-of-run elements, in order, from its scanned offset.
__device__ void unique_write_phase(const uint64_t* __restrict__ keys, uint64_t* __restrict__ dst,
                                   unsigned long long n, const unsigned* __restrict__ offsets) {
  __shared__ unsigned warp_tot[kRadixThreads / 32];
  __shared__ unsigned run;
  if (threadIdx.x == 0) run = offsets[blockIdx.x];
  __syncthreads();
  unsigned long long b, e;
  segment(n, b, e);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (unsigned long long c = b; c < e; c += blockDim.x) {
    const unsigned long long i = c + threadIdx.x;
    const bool keep = i < e && (i == 0 || keys[i] != keys[i - 1]);
    const unsigned bal = __ballot_sync(kFull, keep);
    if (lane == 0) warp_tot[warp] = __popc(bal);
    __syncthreads();
    unsigned before = 0, total = 0;
    for (int w = 0; w < kRadixThreads / 32; ++w) {
      if (w < warp) before += warp_tot[w];
      total += warp_tot[w];
    }
    if (keep) dst[run + before + __popc(bal & ((1u << lane) - 1))] = keys[i];
    __syncthreads();
    if (threadIdx.x == 0) run += total;
    __syncthreads();
  }
}

// The de-duplicated codes copied back (all CTAs, grid-stride).
__device__ void finish_copy_phase(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst,
                                  unsigned long long total) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

__global__ void __launch_bounds__(kRadixThreads) radix_hist_kernel(
    const uint64_t* __restrict__ keys, const unsigned long long* count, long long cap, int shift,
    unsigned* __restrict__ hist) {
  const unsigned long long n = read_count(count);
  if (!large_active(n, cap)) return;
  hist_phase(keys, n, shift, hist);
}

__global__ void __launch_bounds__(kRadixThreads) scan_kernel(unsigned* __restrict__ v, int len,
                                                             const unsigned long long* count,
                                                             long long cap, int need_large) {
  const unsigned long long n = read_count(count);
  if (need_large && !large_active(n, cap)) return;
  scan_phase(v, len);
}

__global__ void __launch_bounds__(kDigits) hist_scan_kernel(unsigned* __restrict__ hist,
                                                            int ctas,
                                                            const unsigned long long* count,
                                                            long long cap) {
  const unsigned long long n = read_count(count);
  if (!large_active(n, cap)) return;
  hist_scan_phase(hist, ctas);
}

__global__ void __launch_bounds__(kRadixThreads) radix_scatter_kernel(
    const uint64_t* __restrict__ src, uint64_t* __restrict__ dst, const unsigned long long* count,
    long long cap, int shift, const unsigned* __restrict__ offsets) {
  const unsigned long long n = read_count(count);
  if (!large_active(n, cap)) return;
  scatter_phase(src, dst, n, shift, offsets);
}

__global__ void __launch_bounds__(kRadixThreads) unique_count_kernel(
    const uint64_t* __restrict__ keys, const unsigned long long* count, long long cap,
    unsigned* __restrict__ per_cta) {
  const unsigned long long n = read_count(count);
  if (!large_active(n, cap)) return;
  unique_count_phase(keys, n, per_cta);
}

__global__ void __launch_bounds__(kRadixThreads) unique_write_kernel(
    const uint64_t* __restrict__ keys, uint64_t* __restrict__ dst, const unsigned long long* count,
    long long cap, const unsigned* __restrict__ offsets) {
  const unsigned long long n = read_count(count);
  if (!large_active(n, cap)) return;
  unique_write_phase(keys, dst, n, offsets);
}

// Copies the de-duplicated codes back and stores the new count.
__global__ void unique_finish_kernel(const uint64_t* __restrict__ src, uint64_t* __restrict__ dst,
                                     unsigned long long* count, long long cap,
                                     const unsigned* __restrict__ per_cta_scanned,
                                     const unsigned* __restrict__ per_cta_raw, int ctas) {
  const unsigned long long n = read_count(count);
  if (!large_active(n, cap)) return;
  finish_copy_phase(src, dst,
                    (unsigned long long)per_cta_scanned[ctas - 1] + per_cta_raw[ctas - 1]);
}

__global__ void store_count_kernel(unsigned long long* count, long long cap,
                                   const unsigned* __restrict__ per_cta_scanned,
                                   const unsigned* __restrict__ per_cta_raw, int ctas) {
  const unsigned long long n = read_count(count);
  if (!large_active(n, cap)) return;
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *count = (unsigned long long)per_cta_scanned[ctas - 1] + per_cta_raw[ctas - 1];
}

// The whole large path in one cooperative launch (every CTA resident; grid-wide barriers
// between the phases): it returns at once, from every CTA, unless the count needs it, so a
// sort graph can hold it unconditionally after the one-CTA sort.  alt, hist, raw and scanned
// are the scratch of launch_sort_unique's layout, for gridDim.x CTAs.
__global__ void __launch_bounds__(kRadixThreads) radix_sort_coop_kernel(
    uint64_t* codes, uint64_t* alt, unsigned long long* count, long long cap, int key_bits,
    unsigned* hist, unsigned* raw, unsigned* scanned) {
  static_assert(kRadixThreads == kDigits, "one thread per digit in the histogram scan");
  const unsigned long long n = read_count(count);
  if (!large_active(n, cap)) return;  // the same answer in every CTA
  cg::grid_group grid = cg::this_grid();
  uint64_t* a = codes;
  uint64_t* b = alt;
  const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kRadixBits;
    hist_phase(a, n, shift, hist);
    grid.sync();
    if (blockIdx.x == 0) hist_scan_phase(hist, gridDim.x);
    grid.sync();
    scatter_phase(a, b, n, shift, hist);
    grid.sync();
    uint64_t* t = a; a = b; b = t;
  }
  unique_count_phase(a, n, raw);
  grid.sync();
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) scanned[i] = raw[i];
    __syncthreads();
    scan_phase(scanned, gridDim.x);
  }
  grid.sync();
  unique_write_phase(a, b, n, scanned);
  grid.sync();
  const unsigned long long total =
      (unsigned long long)scanned[gridDim.x - 1] + raw[gridDim.x - 1];
  finish_copy_phase(b, codes, total);
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = total;
}

int radix_ctas(int sms) { return sms > 0 ? 2 * sms : 256; }

}  // namespace

// ---------------------------------------------------------------------------------------------
// Bitmap output: compaction of the set bits, in order, into codes.
//
// The bitmap is cut into blocks of kBmWords words, one CTA each (8 warps x 256 words).  Pass 1
// counts the set bits of every block, pass 2 scans the block counts (and stores the total), and
// pass 3 writes the codes: each warp walks its nonzero words in order and its 32 lanes write
// the set bits of one word at once, so the stores are coalesced where the bitmap is dense.

constexpr int kBmThreads = 256;
constexpr int kBmWordsPerLane = 8;
constexpr int kBmWords = kBmThreads * kBmWordsPerLane;
// Bitmaps of at most this many blocks (2^19 codes) are compacted by one CTA in one launch: the
// three launches of the multi-CTA form cost more than the one CTA's walk.
constexpr int kBmSmallBlocks = 16;

__global__ void __launch_bounds__(kBmThreads) bitmap_count_kernel(const uint32_t* __restrict__ bm,
                                                                 uint64_t nwords,
                                                                 unsigned* __restrict__ blk) {
  __shared__ unsigned warp_tot[kBmThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t w0 = (uint64_t)blockIdx.x * kBmWords;
  unsigned c = 0;
  for (int i = threadIdx.x; i < kBmWords; i += kBmThreads)
    if (w0 + i < nwords) c += __popc(bm[w0 + i]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
  if (lane == 0) warp_tot[warp] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < kBmThreads / 32; ++w) t += warp_tot[w];
    blk[blockIdx.x] = t;
  }
}

// Exclusive scan of the nblk block counts in place (one CTA); *count receives the total.
// Bitmaps hold at most 2^31 bits, so every offset fits 32 bits.
__global__ void __launch_bounds__(kBmThreads) bitmap_scan_kernel(unsigned* __restrict__ blk,
                                                                int nblk,
                                                                unsigned long long* count) {
  __shared__ unsigned warp_tot[kBmThreads / 32];
  __shared__ unsigned carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nblk; b0 += kBmThreads) {
    const int i = b0 + threadIdx.x;
    const unsigned x = i < nblk ? blk[i] : 0u;
    unsigned incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned before = 0, total = 0;
    for (int w = 0; w < kBmThreads / 32; ++w) {
      if (w < warp) before += warp_tot[w];
      total += warp_tot[w];
    }
    if (i < nblk) blk[i] = carry + before + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = carry;
}

// Writes the codes base + bit of the set bits of block `b` from offset `pos0` (at most cap codes
// in all) and returns the block's count (every thread).  Warp w of the block owns words
// [w*256, (w+1)*256) of it; lane k holds words k, k+32, ... of that range.  The CTA may call it
// again for another block once it returns.
__device__ unsigned bitmap_write_block(const uint32_t* __restrict__ bm, uint64_t nwords,
                                       uint64_t base, uint64_t b, unsigned long long pos0,
                                       uint64_t* __restrict__ out, long long cap) {
  __shared__ unsigned warp_tot[kBmThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const uint64_t wbase = b * kBmWords + (uint64_t)warp * (32 * kBmWordsPerLane);
  uint32_t x[kBmWordsPerLane];
  unsigned c = 0;
#pragma unroll
  for (int i = 0; i < kBmWordsPerLane; ++i) {
    const uint64_t w = wbase + (uint64_t)i * 32 + lane;
    x[i] = w < nwords ? bm[w] : 0u;
    c += __popc(x[i]);
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
  if (lane == 0) warp_tot[warp] = c;
  __syncthreads();
  unsigned long long pos = pos0;
  unsigned block_tot = 0;
  for (int w = 0; w < kBmThreads / 32; ++w) {
    if (w < warp) pos += warp_tot[w];
    block_tot += warp_tot[w];
  }
#pragma unroll
  for (int i = 0; i < kBmWordsPerLane; ++i) {
    const unsigned cnt = __popc(x[i]);
    unsigned excl = cnt;  // inclusive, then exclusive, prefix over the lanes' words
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, excl, o);
      if (lane >= o) excl += y;
    }
    const unsigned tot = __shfl_sync(kFull, excl, 31);
    excl -= cnt;
    unsigned nz = __ballot_sync(kFull, x[i] != 0u);
    while (nz) {  // the warp writes the set bits of one word at a time, lane = bit
      const int src = __ffs(nz) - 1;
      nz &= nz - 1;
      const uint32_t xs = __shfl_sync(kFull, x[i], src);
      const unsigned ps = __shfl_sync(kFull, excl, src);
      if ((xs >> lane) & 1u) {
        const unsigned long long q = pos + ps + __popc(xs & lt);
        if (q < (unsigned long long)cap)
          out[q] = base + ((wbase + (uint64_t)i * 32 + src) << 5) + lane;
      }
    }
    pos += tot;
  }
  __syncthreads();  // warp_tot is read by every warp before a next block overwrites it
  return block_tot;
}

__global__ void __launch_bounds__(kBmThreads) bitmap_write_kernel(const uint32_t* __restrict__ bm,
                                                                 uint64_t nwords, uint64_t base,
                                                                 const unsigned* __restrict__ blk,
                                                                 uint64_t* __restrict__ out,
                                                                 long long cap) {
  bitmap_write_block(bm, nwords, base, blockIdx.x, blk[blockIdx.x], out, cap);
}

// A small bitmap (at most kBmSmallBlocks blocks) compacted by one CTA in one launch: its blocks
// in order, each written from the running count, which *count receives at the end.
__global__ void __launch_bounds__(kBmThreads) bitmap_compact_small_kernel(
    const uint32_t* __restrict__ bm, uint64_t nwords, uint64_t base, uint64_t* __restrict__ out,
    long long cap, unsigned long long* count) {
  const uint64_t nblk = (nwords + kBmWords - 1) / kBmWords;
  unsigned long long run = 0;
  for (uint64_t b = 0; b < nblk; ++b) run += bitmap_write_block(bm, nwords, base, b, run, out, cap);
  if (threadIdx.x == 0) *count = run;
}

// ---- many jobs' bitmaps at once --------------------------------------------------------------
// The blocks of all tasks form one grid: task k owns blocks [first[k], first[k+1]).  Each CTA
// finds its task by binary search over `first` (ntasks + 1 entries).

__device__ __forceinline__ int task_of_block(const unsigned* first, int ntasks, unsigned b) {
  int lo = 0, hi = ntasks;  // first[lo] <= b < first[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (first[mid] <= b) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kBmThreads) bitmap_count_tasks_kernel(const BitmapTask* tasks,
                                                                       const unsigned* first,
                                                                       int ntasks) {
  __shared__ unsigned warp_tot[kBmThreads / 32];
  const int k = task_of_block(first, ntasks, blockIdx.x);
  const BitmapTask t = tasks[k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t w0 = (uint64_t)(blockIdx.x - first[k]) * kBmWords;
  unsigned c = 0;
  for (int i = threadIdx.x; i < kBmWords; i += kBmThreads)
    if (w0 + i < t.nwords) c += __popc(t.bm[w0 + i]);
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
  if (lane == 0) warp_tot[warp] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned tot = 0;
    for (int w = 0; w < kBmThreads / 32; ++w) tot += warp_tot[w];
    t.scratch[blockIdx.x - first[k]] = tot;
  }
}

// CTA k scans task k's block counts (as bitmap_scan_kernel does for one bitmap).
__global__ void __launch_bounds__(kBmThreads) bitmap_scan_tasks_kernel(const BitmapTask* tasks,
                                                                      const unsigned* first) {
  const int k = blockIdx.x;
  const BitmapTask t = tasks[k];
  __shared__ unsigned warp_tot[kBmThreads / 32];
  __shared__ unsigned carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nblk = (int)(first[k + 1] - first[k]);
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nblk; b0 += kBmThreads) {
    const int i = b0 + threadIdx.x;
    const unsigned x = i < nblk ? t.scratch[i] : 0u;
    unsigned incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned before = 0, total = 0;
    for (int w = 0; w < kBmThreads / 32; ++w) {
      if (w < warp) before += warp_tot[w];
      total += warp_tot[w];
    }
    if (i < nblk) t.scratch[i] = carry + before + incl - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *t.count = carry;
}

// Writes every task's codes (as bitmap_write_kernel does for one bitmap).
__global__ void __launch_bounds__(kBmThreads) bitmap_write_tasks_kernel(const BitmapTask* tasks,
                                                                       const unsigned* first,
                                                                       int ntasks) {
  const int k = task_of_block(first, ntasks, blockIdx.x);
  const BitmapTask t = tasks[k];
  const unsigned blk = blockIdx.x - first[k];
  bitmap_write_block(t.bm, t.nwords, t.base, blk, t.scratch[blk], t.out, t.cap);
}

// Scratch layout: [keys: cap u64][hist: kDigits*ctas u32][per_cta raw: ctas][per_cta scan: ctas]
size_t sort_scratch_bytes(int64_t cap, int sms) {
  const int ctas = radix_ctas(sms);
  size_t b = (size_t)(cap > 0 ? cap : 1) * 8;
  b += (size_t)kDigits * ctas * 4 + 2 * (size_t)ctas * 4 + 64;
  return b;
}

uint64_t bitmap_scratch_words(uint64_t nwords) { return (nwords + kBmWords - 1) / kBmWords + 1; }

cudaError_t launch_bitmap_count(const uint32_t* bm, uint64_t nwords, unsigned* scratch,
                                unsigned long long* count, cudaStream_t s) {
  const uint64_t nblk = (nwords + kBmWords - 1) / kBmWords;
  if (nblk == 0 || nblk > (uint64_t)INT32_MAX) return cudaErrorInvalidValue;
  bitmap_count_kernel<<<(unsigned)nblk, kBmThreads, 0, s>>>(bm, nwords, scratch);
  bitmap_scan_kernel<<<1, kBmThreads, 0, s>>>(scratch, (int)nblk, count);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_bitmap_compact(const uint32_t* bm, uint64_t nwords, uint64_t base,
                                  uint64_t* out, int64_t cap, unsigned* scratch,
                                  unsigned long long* count, cudaStream_t s) {
  const uint64_t nblk = (nwords + kBmWords - 1) / kBmWords;
  if (nblk == 0 || nblk > (uint64_t)INT32_MAX) return cudaErrorInvalidValue;
  if (nblk <= (uint64_t)kBmSmallBlocks) {  // one CTA, one launch
    bitmap_compact_small_kernel<<<1, kBmThreads, 0, s>>>(bm, nwords, base, out, (long long)cap,
                                                         count);
    note_launches(1);
    return cudaGetLastError();
  }
  bitmap_count_kernel<<<(unsigned)nblk, kBmThreads, 0, s>>>(bm, nwords, scratch);
  bitmap_scan_kernel<<<1, kBmThreads, 0, s>>>(scratch, (int)nblk, count);
  bitmap_write_kernel<<<(unsigned)nblk, kBmThreads, 0, s>>>(bm, nwords, base, scratch, out,
                                                            (long long)cap);
  note_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_small_sort_tasks(const SortTask* d_tasks, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  small_sort_tasks_kernel<<<ntasks, kSmallThreads, 0, s>>>(d_tasks);
  note_launches(1);
  return cudaGetLastError();
}

uint64_t bitmap_task_blocks(uint64_t nwords) { return (nwords + kBmWords - 1) / kBmWords; }

cudaError_t launch_bitmap_compact_tasks(const BitmapTask* d_tasks, const unsigned* d_first,
                                        int ntasks, unsigned total_blocks, cudaStream_t s) {
  if (ntasks <= 0 || total_blocks == 0) return cudaSuccess;
  bitmap_count_tasks_kernel<<<total_blocks, kBmThreads, 0, s>>>(d_tasks, d_first, ntasks);
  bitmap_scan_tasks_kernel<<<ntasks, kBmThreads, 0, s>>>(d_tasks, d_first);
  bitmap_write_tasks_kernel<<<total_blocks, kBmThreads, 0, s>>>(d_tasks, d_first, ntasks);
  note_launches(3);
  return cudaGetLastError();
}

cudaError_t launch_sort_unique(uint64_t* d_codes, unsigned long long* d_count, int64_t cap,
                               int key_bits, void* scratch, int sms, long long known_count,
                               cudaStream_t s) {
  const bool want_small = known_count < 0 || (known_count > 1 && known_count <= kSmallMax);
  const bool want_large = known_count < 0 || (known_count > kSmallMax && known_count <= cap);
  if (want_small) {
    small_sort_kernel<<<1, kSmallThreads, 0, s>>>(d_codes, d_count, cap, 0, 0);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (!want_large || cap <= kSmallMax) return cudaSuccess;
  const int ctas = radix_ctas(sms);
  uint64_t* alt = reinterpret_cast<uint64_t*>(scratch);
  unsigned* hist = reinterpret_cast<unsigned*>(alt + cap);
  unsigned* raw = hist + (size_t)kDigits * ctas;
  unsigned* scanned = raw + ctas;
  uint64_t* a = d_codes;
  uint64_t* b = alt;
  const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = pass * kRadixBits;
    radix_hist_kernel<<<ctas, kRadixThreads, 0, s>>>(a, d_count, cap, shift, hist);
    hist_scan_kernel<<<1, kDigits, 0, s>>>(hist, ctas, d_count, cap);
    radix_scatter_kernel<<<ctas, kRadixThreads, 0, s>>>(a, b, d_count, cap, shift, hist);
    uint64_t* tmp = a; a = b; b = tmp;
  }
  // Sorted keys are in `a`; compact first-of-run elements into `b`, then back to d_codes.
  unique_count_kernel<<<ctas, kRadixThreads, 0, s>>>(a, d_count, cap, raw);
  cudaMemcpyAsync(scanned, raw, sizeof(unsigned) * ctas, cudaMemcpyDeviceToDevice, s);
  scan_kernel<<<1, kRadixThreads, 0, s>>>(scanned, ctas, d_count, cap, 1);
  unique_write_kernel<<<ctas, kRadixThreads, 0, s>>>(a, b, d_count, cap, scanned);
  unique_finish_kernel<<<ctas, kRadixThreads, 0, s>>>(b, d_codes, d_count, cap, scanned, raw, ctas);
  store_count_kernel<<<1, 32, 0, s>>>(d_count, cap, scanned, raw, ctas);
  note_launches(3 * passes + 5);
  return cudaGetLastError();
}

// Graph form of launch_sort_unique: the one-CTA kernel runs unconditionally; the multi-CTA path
// follows it as one cooperative kernel node that returns at once unless the count needs it
// (a kernel node costs about 1 us where a conditional node cost about 12 us on GB300).  Where
// a cooperative node cannot be made, the one-CTA kernel sets an IF condition and the multi-CTA
// path is the body of that IF node.  *last receives the final node.
cudaError_t add_sort_nodes(cudaGraph_t g, cudaGraphNode_t dep, uint64_t* d_codes,
                           unsigned long long* d_count, int64_t cap, int key_bits, void* scratch,
                           int sms, cudaGraphNode_t* last) {
  const bool large = cap > kSmallMax && scratch != nullptr;
  cudaGraphConditionalHandle h = 0;
  cudaError_t e = cudaSuccess;
  cudaGraphNode_t small;
  {
    long long capv = cap;
    int use = 0;
    void* args[] = {(void*)&d_codes, (void*)&d_count, (void*)&capv, (void*)&h, (void*)&use};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)small_sort_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(kSmallThreads);
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(&small, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
    if (e != cudaSuccess) return e;
  }
  if (!large) {  // the count can never need the multi-CTA path
    *last = small;
    return cudaSuccess;
  }
  // The multi-CTA path as one cooperative kernel node after it: it returns at once unless the
  // count needs it, which costs a kernel node's launch instead of a conditional node's.
  {
    int dev = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, radix_sort_coop_kernel,
                                                      kRadixThreads, 0) == cudaSuccess &&
        per_sm > 0) {
      const int ctas = std::min(radix_ctas(sms), per_sm * sms);  // every CTA resident
      uint64_t* alt = reinterpret_cast<uint64_t*>(scratch);
      unsigned* hist = reinterpret_cast<unsigned*>(alt + cap);
      unsigned* raw = hist + (size_t)kDigits * radix_ctas(sms);
      unsigned* scanned = raw + radix_ctas(sms);
      long long capv = cap;
      int kb = key_bits;
      void* args[] = {(void*)&d_codes, (void*)&alt, (void*)&d_count, (void*)&capv, (void*)&kb,
                      (void*)&hist, (void*)&raw, (void*)&scanned};
      cudaKernelNodeParams kp = {};
      kp.func = (void*)radix_sort_coop_kernel;
      kp.gridDim = dim3(ctas);
      kp.blockDim = dim3(kRadixThreads);
      kp.kernelParams = args;
      cudaGraphNode_t node;
      e = cudaGraphAddKernelNode(&node, g, &small, 1, &kp);
      if (e != cudaSuccess) return e;
      cudaKernelNodeAttrValue v = {};
      v.cooperative = 1;
      if (cudaGraphKernelNodeSetAttribute(node, cudaKernelNodeAttributeCooperative, &v) ==
          cudaSuccess) {
        *last = node;
        return cudaSuccess;
      }
      cudaGetLastError();
      e = cudaGraphDestroyNode(node);  // not cooperative: the conditional form instead
      if (e != cudaSuccess) return e;
    }
    cudaGetLastError();
  }
  e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  {  // the one-CTA sort now sets the IF node's condition
    long long capv = cap;
    int use = 1;
    void* args[] = {(void*)&d_codes, (void*)&d_count, (void*)&capv, (void*)&h, (void*)&use};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)small_sort_kernel;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(kSmallThreads);
    kp.kernelParams = args;
    e = cudaGraphKernelNodeSetParams(small, &kp);
    if (e != cudaSuccess) return e;
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t ifnode;
  e = cudaGraphAddNode(&ifnode, g, &small, nullptr, 1, &cp);
  if (e != cudaSuccess) return e;
  *last = ifnode;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  const int ctas = radix_ctas(sms);
  uint64_t* alt = reinterpret_cast<uint64_t*>(scratch);
  unsigned* hist = reinterpret_cast<unsigned*>(alt + cap);
  unsigned* raw = hist + (size_t)kDigits * ctas;
  unsigned* scanned = raw + ctas;
  long long capv = cap;
  cudaGraphNode_t prev = nullptr;
  auto add = [&](void* func, int grid, int block, void** args) -> cudaError_t {
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.kernelParams = args;
    cudaGraphNode_t n;
    cudaError_t r = cudaGraphAddKernelNode(&n, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
    prev = n;
    return r;
  };
  uint64_t* a = d_codes;
  uint64_t* b = alt;
  const int passes = (key_bits + kRadixBits - 1) / kRadixBits;
  for (int pass = 0; pass < passes && e == cudaSuccess; ++pass) {
    int shift = pass * kRadixBits;
    int nctas = ctas;
    void* ha[] = {(void*)&a, (void*)&d_count, (void*)&capv, (void*)&shift, (void*)&hist};
    e = add((void*)radix_hist_kernel, ctas, kRadixThreads, ha);
    void* sa[] = {(void*)&hist, (void*)&nctas, (void*)&d_count, (void*)&capv};
    if (e == cudaSuccess) e = add((void*)hist_scan_kernel, 1, kDigits, sa);
    void* xa[] = {(void*)&a, (void*)&b, (void*)&d_count, (void*)&capv, (void*)&shift, (void*)&hist};
    if (e == cudaSuccess) e = add((void*)radix_scatter_kernel, ctas, kRadixThreads, xa);
    uint64_t* tmp = a; a = b; b = tmp;
  }
  if (e != cudaSuccess) return e;
  int ctas_i = ctas, need = 1;
  void* ua[] = {(void*)&a, (void*)&d_count, (void*)&capv, (void*)&raw};
  e = add((void*)unique_count_kernel, ctas, kRadixThreads, ua);
  if (e != cudaSuccess) return e;
  cudaGraphNode_t cpy;
  e = cudaGraphAddMemcpyNode1D(&cpy, body, &prev, 1, scanned, raw, sizeof(unsigned) * ctas,
                               cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) return e;
  prev = cpy;
  void* sa2[] = {(void*)&scanned, (void*)&ctas_i, (void*)&d_count, (void*)&capv, (void*)&need};
  e = add((void*)scan_kernel, 1, kRadixThreads, sa2);
  void* wa[] = {(void*)&a, (void*)&b, (void*)&d_count, (void*)&capv, (void*)&scanned};
  if (e == cudaSuccess) e = add((void*)unique_write_kernel, ctas, kRadixThreads, wa);
  void* fa[] = {(void*)&b, (void*)&d_codes, (void*)&d_count, (void*)&capv, (void*)&scanned,
                (void*)&raw, (void*)&ctas_i};
  if (e == cudaSuccess) e = add((void*)unique_finish_kernel, ctas, kRadixThreads, fa);
  void* ca[] = {(void*)&d_count, (void*)&capv, (void*)&scanned, (void*)&raw, (void*)&ctas_i};
  if (e == cudaSuccess) e = add((void*)store_count_kernel, 1, 32, ca);
  return e;
}

}  // namespace motif

// K1: the skip-BF search (Sec. III.A) as a multi-job, pass-structured CUDA kernel.
//
// Work is organised in *passes* over the live work units of each job:
//   FRESH — units come straight from the candidate index range of the current chunk (Sec. IV.A:
//           an l-mer is produced from its index, never stored); one lane per unit scans
//           sequences [0, span0) from shared memory;
//   QUEUE — the survivors the previous pass compacted into a ping-pong queue; one lane per
//           entry scans the next sequence from shared memory;
//   REST  — once few survivors are left, one warp per entry scans every remaining sequence:
//           the lanes split the windows and the warp combines their results.
// A unit that fails a sequence is dropped on the spot and never looks at the later sequences
// (the skip of Sec. III.A); a unit that passes the last sequence is accepted.  Between passes the
// survivors are compacted with a warp ballot / prefix sum and one atomic per warp, so the next
// pass runs full warps instead of lanes idling behind the skip.
//
// Two unit kinds share this structure:
//   CAND  — one candidate l-mer per lane (cpt of them in a fresh pass).  Per window:
//           m = (E_c ^ E_w) | (O_c ^ O_w) over the compressed bit planes (the pair-fold of the
//           XOR of the packed codes), dist = popc(m), running min; a lane stops scanning a
//           sequence once every live candidate it holds is within d of some window.
//   GROUP — one group of 4^ks candidates sharing their first l-ks bases per lane.  Per window
//           one POPC gives the prefix distance h.  When h <= d the window is recorded in a
//           per-lane hit list in shared memory; at the end of the sequence each recorded window
//           ORs in the precomputed mask of suffixes within d-h of its last ks bases (a row of
//           the Hamming-ball table).  Hamming distance is additive over positions, so each
//           candidate of the group is matched by exactly the windows the per-candidate test
//           would accept.  Deferring the rare hits keeps the scan loop free of divergent work.
//
// A launch of the step kernel advances every job in the table by one pass (or part of one,
// under a tile budget).  CTAs are persistent: each walks the jobs in table order, stages the
// windows of the pass into shared memory and pulls tiles from the job's pass cursor.  The last
// CTA to finish advances each job's state for the next launch (and, inside a CUDA graph, sets
// the while-loop condition); no CTA ever waits for another.
#include <map>
#include <mutex>
#include <tuple>

#include "motif_internal.h"

namespace motif {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxStageSeqs = 2;  // sequences of one pass staged in shared memory
constexpr int kHitCap = 12;       // GROUP: hit-list entries per lane before a flush
constexpr int kMaxBlock = 256;

enum PassMode { kFresh = 0, kQueue = 1, kRest = 2, kTiled = 3 };

__device__ __forceinline__ uint32_t compress_even(uint64_t x) {
  x &= 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
  return (uint32_t)x;
}

// Compressed planes of a packed code: E = low bit of each base, O = high bit.
__device__ __forceinline__ void code_planes(uint64_t k, uint32_t& E, uint32_t& O) {
  E = compress_even(k);
  O = compress_even(k >> 1);
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
__device__ __forceinline__ int ld_volatile(const int32_t* p) {
  return *reinterpret_cast<const volatile int32_t*>(p);
}

// Reserves `cnt` slots per lane at `counter` with one atomic per warp; returns this lane's
// first slot.  Must be called by all 32 lanes.
// Records one accepted code in the job's bitmap.
__device__ __forceinline__ void bitmap_set(const JobDesc& jd, uint64_t code) {
  const uint64_t b = code - jd.bm_base;
  atomicOr(jd.bitmap + (b >> 5), 1u << (unsigned)(b & 31));
}

__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long* counter,
                                                           unsigned cnt) {
  const int lane = threadIdx.x & 31;
  unsigned incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  const unsigned total = __shfl_sync(kFull, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total) base = atomicAdd(counter, (unsigned long long)total);
  base = __shfl_sync(kFull, base, 31);
  return base + (incl - cnt);
}


// Shape of the pass a job is in; identical in every CTA of a step.
struct Pass {
  unsigned long long work;  // items of the pass (units, or queue entries)
  uint64_t chunk_base;      // first unit of the chunk
  uint64_t chunk_units;     // units in the chunk
  int s0, s1;               // sequences [s0, s1) the pass scans
  int mode;                 // PassMode
  int qin, qout;
};

__device__ Pass make_pass(const JobDesc& jd, const JobState* st) {
  Pass p;
  const unsigned long long chunk = ld_volatile(&st->chunk);
  const int pass_seq = ld_volatile(&st->pass_seq);
  p.chunk_base = jd.unit_lo + chunk * jd.chunk_units;
  const uint64_t left = jd.unit_hi > p.chunk_base ? jd.unit_hi - p.chunk_base : 0;
  p.chunk_units = left < jd.chunk_units ? left : jd.chunk_units;
  if (pass_seq == 0) {
    p.mode = jd.tiled ? kTiled : kFresh;
    p.work = p.chunk_units;
    if (jd.tiled && jd.seq_block > 0) {  // (sequence block, tile) items, 256 groups each
      const unsigned long long tiles = (p.chunk_units + 255) / 256;
      const unsigned long long blocks = (jd.n + jd.seq_block - 1) / jd.seq_block;
      p.work = tiles * blocks * 256;
    }
    // A seeded search has already kept only candidates that match the first sequence; its
    // fresh pass scans nothing and compacts them (few per warp) into the queue, so the second
    // sequence runs on full warps.
    p.s0 = jd.seed ? 1 : 0;
    p.s1 = jd.tiled ? jd.n : jd.seed ? 1 : (jd.span0 < jd.n ? jd.span0 : jd.n);
    p.qin = 0;
    p.qout = 0;
  } else {
    p.qin = ld_volatile(&st->qsel);
    p.qout = 1 - p.qin;
    p.work = ld_volatile(&st->qcount[p.qin]);
    p.s0 = pass_seq;
    if (p.work <= jd.rest_threshold && jd.n - pass_seq >= 2) {
      p.mode = kRest;
      p.s1 = jd.n;
    } else {
      p.mode = kQueue;
      p.s1 = pass_seq + 1;
    }
  }
  return p;
}

// Items per tile: a warp takes 32*cpt fresh CAND candidates, 32 units / entries otherwise, and
// one entry per warp in a REST pass.
__device__ __forceinline__ unsigned long long tile_of(int kind, int p, int mode) {
  if (mode == kRest) return 1;
  if ((kind == MOTIF_KERNEL_CAND || kind == MOTIF_KERNEL_BITSLICE) && mode == kFresh)
    return 32ull * p;
  return 32;
}

// ---------------------------------------------------------------------------------------------
// CAND: one candidate per lane slot.

// Scans one staged sequence for up to CPT candidates; returns the subset of `alive` that has a
// window within distance d.  `w4` holds two windows (E0,O0,E1,O1) per uint4; the row is padded
// to a multiple of 8 windows.
template <int CPT>
__device__ __forceinline__ unsigned scan_cand(const uint4* __restrict__ w4, int wpad, int d,
                                              const uint32_t (&E)[CPT], const uint32_t (&O)[CPT],
                                              unsigned alive) {
  uint32_t mn[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) mn[c] = 64u;
  const int n4 = wpad >> 1;  // uint4 count
  for (int q = 0; q < n4; q += 4) {
    const uint4 a = w4[q], b = w4[q + 1], e = w4[q + 2], f = w4[q + 3];
    unsigned hit = 0;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      uint32_t m = mn[c];
      m = min(m, (uint32_t)__popc((E[c] ^ a.x) | (O[c] ^ a.y)));
      m = min(m, (uint32_t)__popc((E[c] ^ a.z) | (O[c] ^ a.w)));
      m = min(m, (uint32_t)__popc((E[c] ^ b.x) | (O[c] ^ b.y)));
      m = min(m, (uint32_t)__popc((E[c] ^ b.z) | (O[c] ^ b.w)));
      m = min(m, (uint32_t)__popc((E[c] ^ e.x) | (O[c] ^ e.y)));
      m = min(m, (uint32_t)__popc((E[c] ^ e.z) | (O[c] ^ e.w)));
      m = min(m, (uint32_t)__popc((E[c] ^ f.x) | (O[c] ^ f.y)));
      m = min(m, (uint32_t)__popc((E[c] ^ f.z) | (O[c] ^ f.w)));
      mn[c] = m;
      hit |= (m <= (uint32_t)d ? 1u : 0u) << c;
    }
    if ((hit & alive) == alive) break;  // every live candidate has matched this sequence
  }
  unsigned matched = 0;
#pragma unroll
  for (int c = 0; c < CPT; ++c) matched |= (mn[c] <= (uint32_t)d ? 1u : 0u) << c;
  return matched & alive;
}

// ---------------------------------------------------------------------------------------------
// BITSLICE: one candidate per lane slot, 128 windows per step counted bit-sliced.
//
// For each block of 32 windows and base position i the pass stages four 32-bit words, one per
// base b of the candidate: bit j of word (i, b) is set when window j's base at position i is not
// b.  The words of four neighbouring blocks sit side by side, so one 128-bit shared load gives
// a lane the mismatch bits of its candidate's base against 128 windows.  They are added into
// 3-bit saturating counters held as bit planes (c0, c1, c2 and a sticky overflow c3), seven
// positions at a time: four full adders (8 LOP3) reduce seven words to a 3-bit number, which
// one ripple adds to the counter (7 LOP3); leftover positions go three (11 LOP3) or one (5 LOP3)
// at a time -- no POPC.  Window j is within distance d when its counter is at most d (d <= 7).

// Staged words of one sequence: word (i, b, blk) at ((4 i + b) * nblkp + blk); nblkp, the block
// count rounded up to a multiple of 4, groups the blocks in fours.  One warp per block.
__device__ __forceinline__ void stage_bitslice(uint32_t* dst, const uint2* row, int W, int l,
                                               int nblkp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int blk = warp; blk < nblkp; blk += nwarps) {
    int j = blk * 32 + lane;
    if (j >= W) j = W - 1;  // past the row: a copy of its last window (matches when it does)
    const uint2 w = row[j];
    for (int i = 0; i < l; ++i) {
      const unsigned te = __ballot_sync(kFull, (w.x >> (l - 1 - i)) & 1u);
      const unsigned to = __ballot_sync(kFull, (w.y >> (l - 1 - i)) & 1u);
      if (lane < 4)
        dst[(size_t)(4 * i + lane) * nblkp + blk] =
            (te ^ ((lane & 1) ? kFull : 0u)) | (to ^ ((lane & 2) ? kFull : 0u));
    }
  }
}

// A bit-sliced counter of mismatches over 32 windows.
struct SliceCount {
  uint32_t c0, c1, c2, c3;
  __device__ __forceinline__ void clear() { c0 = c1 = c2 = c3 = 0u; }
  __device__ __forceinline__ void add1(uint32_t x) {  // + x
    const uint32_t k = c1 & c0 & x;
    c1 ^= c0 & x;
    c0 ^= x;
    c3 |= c2 & k;
    c2 ^= k;
  }
  __device__ __forceinline__ void add3(uint32_t x1, uint32_t x2, uint32_t x3) {  // + x1+x2+x3
    const uint32_t sum = x1 ^ x2 ^ x3;
    const uint32_t cy = (x1 & x2) | (x1 & x3) | (x2 & x3);
    add1(sum);
    const uint32_t v = c2 & c1 & cy;  // + 2 cy
    c2 ^= c1 & cy;
    c1 ^= cy;
    c3 |= v;
  }
  // + x1+...+x7: four full adders reduce the seven words to a 3-bit number (y0 + 2 y1 + 4 y2),
  // added with one ripple.
  __device__ __forceinline__ void add7(uint32_t x1, uint32_t x2, uint32_t x3, uint32_t x4,
                                       uint32_t x5, uint32_t x6, uint32_t x7) {
    const uint32_t s1 = x1 ^ x2 ^ x3, k1 = (x1 & x2) | (x1 & x3) | (x2 & x3);
    const uint32_t s2 = x4 ^ x5 ^ x6, k2 = (x4 & x5) | (x4 & x6) | (x5 & x6);
    const uint32_t y0 = s1 ^ s2 ^ x7, k3 = (s1 & s2) | (s1 & x7) | (s2 & x7);
    const uint32_t y1 = k1 ^ k2 ^ k3, y2 = (k1 & k2) | (k1 & k3) | (k2 & k3);
    const uint32_t r0 = c0 & y0;
    c0 ^= y0;
    const uint32_t r1 = (c1 & y1) | (c1 & r0) | (y1 & r0);
    c1 ^= y1 ^ r0;
    const uint32_t r2 = (c2 & y2) | (c2 & r1) | (y2 & r1);
    c2 ^= y2 ^ r1;
    c3 |= r2;
  }
  // Windows whose count is at most d (D0..D2: the bits of d as all-ones / all-zero masks).
  __device__ __forceinline__ uint32_t within(uint32_t D0, uint32_t D1, uint32_t D2) const {
    const uint32_t gt = (c2 & ~D2) | (~(c2 ^ D2) & ((c1 & ~D1) | (~(c1 ^ D1) & (c0 & ~D0))));
    return ~c3 & ~gt;
  }
};

// Adds positions [0, cnt) of one candidate against four blocks: `m` points at word (0, 0, first
// block) of the sub-range, `bits` holds the candidate's bases (first base in its top two bits).
__device__ __forceinline__ void bitslice_quad(const uint32_t* __restrict__ m, int nblkp,
                                              uint32_t bits, int cnt, SliceCount& a,
                                              SliceCount& b, SliceCount& c, SliceCount& e) {
  const int step = 4 * nblkp;  // words between positions
  int i = 0;
  for (; i + 7 <= cnt; i += 7) {
    uint4 x[7];
#pragma unroll
    for (int u = 0; u < 7; ++u)
      x[u] = *reinterpret_cast<const uint4*>(m + u * step + ((bits >> (30 - 2 * u)) & 3u) * nblkp);
    bits <<= 14;
    m += 7 * step;
    a.add7(x[0].x, x[1].x, x[2].x, x[3].x, x[4].x, x[5].x, x[6].x);
    b.add7(x[0].y, x[1].y, x[2].y, x[3].y, x[4].y, x[5].y, x[6].y);
    c.add7(x[0].z, x[1].z, x[2].z, x[3].z, x[4].z, x[5].z, x[6].z);
    e.add7(x[0].w, x[1].w, x[2].w, x[3].w, x[4].w, x[5].w, x[6].w);
  }
  for (; i + 3 <= cnt; i += 3) {
    const uint4 x1 = *reinterpret_cast<const uint4*>(m + (bits >> 30) * nblkp);
    const uint4 x2 = *reinterpret_cast<const uint4*>(m + step + ((bits >> 28) & 3u) * nblkp);
    const uint4 x3 = *reinterpret_cast<const uint4*>(m + 2 * step + ((bits >> 26) & 3u) * nblkp);
    bits <<= 6;
    m += 3 * step;
    a.add3(x1.x, x2.x, x3.x);
    b.add3(x1.y, x2.y, x3.y);
    c.add3(x1.z, x2.z, x3.z);
    e.add3(x1.w, x2.w, x3.w);
  }
  for (; i < cnt; ++i) {
    const uint4 x = *reinterpret_cast<const uint4*>(m + (bits >> 30) * nblkp);
    bits <<= 2;
    m += step;
    a.add1(x.x);
    b.add1(x.y);
    c.add1(x.z);
    e.add1(x.w);
  }
}

// Scans one staged sequence for up to CPT candidates (their codes); returns the subset of
// `alive` that has a window within distance d.
template <int CPT>
__device__ __forceinline__ unsigned scan_bitslice(const uint32_t* __restrict__ stage, int nblkp,
                                                  int l, int d, const uint64_t (&code)[CPT],
                                                  unsigned alive) {
  const uint32_t D0 = (d & 1) ? kFull : 0u, D1 = (d & 2) ? kFull : 0u, D2 = (d & 4) ? kFull : 0u;
  const int nh = l > 16 ? l - 16 : 0;  // positions held in the code's high word
  const int nl = l - nh;
  uint32_t hi[CPT], lo[CPT];
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    hi[c] = nh ? (uint32_t)(code[c] >> 32) << (32 - 2 * nh) : 0u;
    lo[c] = (uint32_t)code[c] << (32 - 2 * nl);
  }
  unsigned matched = 0;
  for (int bp = 0; bp < nblkp; bp += 4) {
    const uint32_t* m = stage + bp;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      if (!(alive & ~matched & (1u << c))) continue;
      SliceCount a, b, cc, e;
      a.clear();
      b.clear();
      cc.clear();
      e.clear();
      if (nh) bitslice_quad(m, nblkp, hi[c], nh, a, b, cc, e);
      bitslice_quad(m + (size_t)4 * nh * nblkp, nblkp, lo[c], nl, a, b, cc, e);
      if (a.within(D0, D1, D2) | b.within(D0, D1, D2) | cc.within(D0, D1, D2) |
          e.within(D0, D1, D2))
        matched |= 1u << c;
    }
    if ((matched & alive) == alive) break;  // every live candidate has matched this sequence
  }
  return matched & alive;
}

// Seeded FRESH tile (CAND, BITSLICE): the seed bitmap holds exactly the candidates within d of
// a window of the first sequence, so the pass scans no sequence; it compacts the seeded items of
// [base, base + 1024), 32 per lane (one seed word, read as two when the range start is not a
// multiple of 32), into the queue, or accepts them when there is no other sequence.
__device__ __noinline__ void seeded_fresh_tile(const JobDesc& jd, JobState* st, const Pass& p,
                                  unsigned long long base) {
  const int lane = threadIdx.x & 31;
  const unsigned long long item0 = base + 32ull * (unsigned)lane;
  uint32_t bits = 0;
  if (item0 < p.work) {
    // bit (code - seed_base) of the bitmap, for the codes chunk_base + item0 + 0..31; the
    // bitmap holds one word past its end, so word + 1 is always readable
    const uint64_t b = p.chunk_base + item0 - jd.seed_base;
    const uint32_t w0 = __ldg(jd.seed + (b >> 5)), w1 = __ldg(jd.seed + (b >> 5) + 1);
    bits = __funnelshift_r(w0, w1, (unsigned)(b & 31));
    const unsigned long long left = p.work - item0;
    if (left < 32) bits &= (1u << (unsigned)left) - 1u;
  }
  const unsigned cnt = __popc(bits);
  if (p.s1 >= jd.n && jd.bitmap) {
    for (uint32_t x = bits; x; x &= x - 1) bitmap_set(jd, p.chunk_base + item0 + (__ffs(x) - 1));
  } else if (p.s1 >= jd.n) {
    unsigned long long slot = warp_reserve(&st->out_count, cnt);
    for (uint32_t x = bits; x; x &= x - 1, ++slot)
      if (slot < jd.out_cap) jd.out[slot] = p.chunk_base + item0 + (__ffs(x) - 1);
  } else {
    unsigned long long slot = warp_reserve(&st->qcount[p.qout], cnt);
    for (uint32_t x = bits; x; x &= x - 1)
      jd.qidx[p.qout][slot++] = (uint32_t)(item0 + (__ffs(x) - 1));
  }
}

// FRESH / QUEUE tile: lane slot c of the warp owns item base + c*32 + lane.
template <int KIND, int CPT>
__device__ void cand_tile(const JobDesc& jd, JobState* st, const Pass& p,
                          unsigned long long base, const uint4* stage) {
  const int lane = threadIdx.x & 31;
  uint32_t E[CPT], O[CPT], off[CPT];
  unsigned alive = 0;
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const unsigned long long item = base + (unsigned long long)c * 32 + lane;
    off[c] = 0;
    E[c] = O[c] = 0;
    if (item < p.work) {
      off[c] = p.mode == kFresh ? (uint32_t)item : jd.qidx[p.qin][item];
      code_planes(p.chunk_base + off[c], E[c], O[c]);
      alive |= 1u << c;
    }
  }
  const int wpad = jd.wstride;
  if (KIND == MOTIF_KERNEL_BITSLICE) {
    uint64_t code[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) code[c] = p.chunk_base + off[c];
    const int nblkp = ((jd.W + 127) >> 7) << 2;  // blocks of 32 windows, a multiple of 4
    const uint32_t* words = reinterpret_cast<const uint32_t*>(stage);
    for (int s = p.s0; s < p.s1 && alive; ++s)
      alive = scan_bitslice<CPT>(words + (size_t)(s - p.s0) * nblkp * 4 * jd.l, nblkp, jd.l,
                                 jd.d, code, alive);
  } else {
    for (int s = p.s0; s < p.s1 && alive; ++s)
      alive = scan_cand<CPT>(stage + (size_t)(s - p.s0) * (wpad >> 1), wpad, jd.d, E, O, alive);
  }
  __syncwarp();
  const unsigned cnt = __popc(alive);
  if (p.s1 >= jd.n && jd.bitmap) {
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (alive & (1u << c)) bitmap_set(jd, p.chunk_base + off[c]);
  } else if (p.s1 >= jd.n) {
    unsigned long long slot = warp_reserve(&st->out_count, cnt);
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (alive & (1u << c)) {
        if (slot < jd.out_cap) jd.out[slot] = p.chunk_base + off[c];
        ++slot;
      }
  } else {
    unsigned long long slot = warp_reserve(&st->qcount[p.qout], cnt);
#pragma unroll
    for (int c = 0; c < CPT; ++c)
      if (alive & (1u << c)) jd.qidx[p.qout][slot++] = off[c];
  }
}

// REST: the warp owns one queue entry and scans every remaining sequence, lanes striding over
// the windows of global memory.
__device__ void cand_rest(const JobDesc& jd, JobState* st, const Pass& p,
                          unsigned long long item) {
  const int lane = threadIdx.x & 31;
  const uint64_t k = p.chunk_base + jd.qidx[p.qin][item];
  uint32_t E, O;
  code_planes(k, E, O);
  for (int s = p.s0; s < jd.n; ++s) {
    const uint2* row = jd.planes + (size_t)s * jd.wstride;
    bool matched = false;
    for (int b = 0; b < jd.W; b += 64) {  // two loads in flight per lane
      const int j0 = b + lane, j1 = b + 32 + lane;
      const uint2 w0 = j0 < jd.W ? __ldg(row + j0) : make_uint2(~E, ~O);
      const uint2 w1 = j1 < jd.W ? __ldg(row + j1) : make_uint2(~E, ~O);
      const bool hit = (j0 < jd.W && __popc((E ^ w0.x) | (O ^ w0.y)) <= jd.d) ||
                       (j1 < jd.W && __popc((E ^ w1.x) | (O ^ w1.y)) <= jd.d);
      if (__any_sync(kFull, hit)) {
        matched = true;
        break;
      }
    }
    if (!matched) return;  // the skip: no window of sequence s is within d
  }
  if (lane == 0 && jd.bitmap) {
    bitmap_set(jd, k);
  } else if (lane == 0) {
    const unsigned long long slot = atomicAdd(&st->out_count, 1ull);
    if (slot < jd.out_cap) jd.out[slot] = k;
  }
}

// ---------------------------------------------------------------------------------------------
// GROUP: 4^KS candidates sharing their first l-KS bases per lane.

template <int KS>
struct GroupMask {
  static constexpr int NW = (KS <= 3) ? 1 : (1 << (2 * KS - 6));
  uint64_t w[NW];
};

// Marks, in `matched`, the suffixes within r of suffix value v (ball table row).
template <int KS, bool GLOBAL>
__device__ __forceinline__ void or_ball(GroupMask<KS>& matched, const uint64_t* ball, int v,
                                        int r) {
  constexpr int NW = GroupMask<KS>::NW;
  const uint64_t* row = ball + ((size_t)v * (KS + 1) + r) * NW;
  if constexpr (GLOBAL && NW == 4) {  // 32-byte row: two 128-bit read-only loads
    const ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2*>(row));
    const ulonglong2 y = __ldg(reinterpret_cast<const ulonglong2*>(row) + 1);
    matched.w[0] |= x.x;
    matched.w[1 % NW] |= x.y;
    matched.w[2 % NW] |= y.x;
    matched.w[3 % NW] |= y.y;
  } else {
#pragma unroll
    for (int i = 0; i < NW; ++i) matched.w[i] |= GLOBAL ? __ldg(row + i) : row[i];
  }
}

template <int KS>
__device__ __forceinline__ bool covers(const GroupMask<KS>& matched, const GroupMask<KS>& alive) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < GroupMask<KS>::NW; ++i) ok &= (matched.w[i] & alive.w[i]) == alive.w[i];
  return ok;
}

template <int KS>
__device__ __forceinline__ bool any_set(const GroupMask<KS>& m) {
  uint64_t o = 0;
#pragma unroll
  for (int i = 0; i < GroupMask<KS>::NW; ++i) o |= m.w[i];
  return o != 0;
}

// One window with prefix distance h (already known <= d): or in the ball of its suffix.
template <int KS, bool GLOBAL>
__device__ __forceinline__ void group_hit(GroupMask<KS>& matched, const uint64_t* ball, int d,
                                          int h, int v) {
  int r = d - h;
  r = r < KS ? r : KS;
  or_ball<KS, GLOBAL>(matched, ball, v, r);
}

// ORs the recorded hits (window j << 3 | radius) of this lane into `matched`.
template <int KS>
__device__ __forceinline__ void flush_hits(GroupMask<KS>& matched, const uint32_t* hl, int hstride,
                                           int cnt, const uint16_t* __restrict__ sfx,
                                           const uint64_t* ball) {
  for (int i = 0; i < cnt; ++i) {
    const uint32_t e = hl[i * hstride];
    or_ball<KS, true>(matched, ball, sfx[e >> 3], (int)(e & 7u));
  }
}

// Staged scan of one sequence: wp4 holds two prefix-plane windows per uint4, sfx the suffix
// value of each window; hl is this lane's hit list (stride hstride words).
template <int KS>
__device__ __forceinline__ void scan_group_staged(const uint4* __restrict__ wp4,
                                                  const uint16_t* __restrict__ sfx, int wpad,
                                                  int d, uint32_t Ep, uint32_t Op,
                                                  const uint64_t* ball, uint32_t* hl, int hstride,
                                                  GroupMask<KS>& alive) {
  GroupMask<KS> matched;
#pragma unroll
  for (int i = 0; i < GroupMask<KS>::NW; ++i) matched.w[i] = 0;
  const int n4 = wpad >> 1;
  int cnt = 0;
  for (int q = 0; q < n4; q += 4) {  // 8 windows per iteration (rows are padded to 8)
    const uint4 a = wp4[q], b = wp4[q + 1], c = wp4[q + 2], e = wp4[q + 3];
    int h[8];
    h[0] = __popc((Ep ^ a.x) | (Op ^ a.y));
    h[1] = __popc((Ep ^ a.z) | (Op ^ a.w));
    h[2] = __popc((Ep ^ b.x) | (Op ^ b.y));
    h[3] = __popc((Ep ^ b.z) | (Op ^ b.w));
    h[4] = __popc((Ep ^ c.x) | (Op ^ c.y));
    h[5] = __popc((Ep ^ c.z) | (Op ^ c.w));
    h[6] = __popc((Ep ^ e.x) | (Op ^ e.y));
    h[7] = __popc((Ep ^ e.z) | (Op ^ e.w));
    const int m = min(min(min(h[0], h[1]), min(h[2], h[3])), min(min(h[4], h[5]), min(h[6], h[7])));
    if (m <= d) {
      const uint32_t j = (uint32_t)q * 2u;
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (h[i] <= d) {
          hl[cnt * hstride] = ((j + i) << 3) | (uint32_t)min(d - h[i], KS);
          ++cnt;
        }
      if (cnt > kHitCap - 8) {
        flush_hits<KS>(matched, hl, hstride, cnt, sfx, ball);
        cnt = 0;
        if (covers<KS>(matched, alive)) break;  // every live candidate matched this sequence
      }
    }
  }
  flush_hits<KS>(matched, hl, hstride, cnt, sfx, ball);
#pragma unroll
  for (int i = 0; i < GroupMask<KS>::NW; ++i) alive.w[i] &= matched.w[i];
}

// Initial alive mask of group g: the suffixes s with lo <= (g << 2KS) + s < hi.
template <int KS>
__device__ __forceinline__ void range_mask(uint64_t g, uint64_t lo, uint64_t hi,
                                           GroupMask<KS>& m) {
  constexpr int NW = GroupMask<KS>::NW;
  constexpr int BITS = 1 << (2 * KS);
  const uint64_t first = g << (2 * KS);
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    const int wbits = BITS < 64 ? BITS : 64;
    uint64_t word = wbits == 64 ? ~0ull : ((1ull << wbits) - 1);
    const uint64_t wlo = first + (uint64_t)i * 64;  // code of bit 0 of this word
    if (lo > wlo) {  // clear bits below lo
      const uint64_t k = lo - wlo;
      word = k >= 64 ? 0 : (word & (~0ull << k));
    }
    if (hi < wlo + (uint64_t)wbits) {  // clear bits at or above hi
      const uint64_t k = hi > wlo ? hi - wlo : 0;
      word = k == 0 ? 0 : (word & (~0ull >> (64 - k)));
    }
    m.w[i] = word;
  }
}

// Appends the accepted codes of `alive` (group g) to the output; all 32 lanes call it.
template <int KS>
__device__ __forceinline__ void group_output(const JobDesc& jd, JobState* st, uint64_t g,
                                             const GroupMask<KS>& alive) {
  constexpr int NW = GroupMask<KS>::NW;
  const uint64_t first = g << (2 * KS);
  if (jd.bitmap) {  // group bits are contiguous codes: OR the mask words in (first - bm_base is
                    // a multiple of 64 for KS >= 3, of the 4 or 16 mask bits below that)
    const uint64_t b = first - jd.bm_base;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      if (!alive.w[i]) continue;
      if (KS >= 3)
        atomicOr(reinterpret_cast<unsigned long long*>(jd.bitmap + ((b >> 5) + 2 * i)),
                 (unsigned long long)alive.w[i]);
      else
        atomicOr(jd.bitmap + (b >> 5), (uint32_t)alive.w[i] << (unsigned)(b & 31));
    }
    return;
  }
  unsigned cnt = 0;
#pragma unroll
  for (int i = 0; i < NW; ++i) cnt += __popcll(alive.w[i]);
  unsigned long long slot = warp_reserve(&st->out_count, cnt);
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    uint64_t w = alive.w[i];
    while (w) {
      const int b = __ffsll((long long)w) - 1;
      w &= w - 1;
      if (slot < jd.out_cap) jd.out[slot] = first + (uint64_t)i * 64 + b;
      ++slot;
    }
  }
}

template <int KS>
__device__ void group_tile(const JobDesc& jd, JobState* st, const Pass& p,
                           unsigned long long base, const uint4* stage_wp,
                           const uint16_t* stage_sfx, const uint64_t* stage_ball, uint32_t* hl) {
  constexpr int NW = GroupMask<KS>::NW;
  const int lane = threadIdx.x & 31;
  const unsigned long long item = base + lane;
  GroupMask<KS> alive;
  uint32_t off = 0, Ep = 0, Op = 0;
#pragma unroll
  for (int i = 0; i < NW; ++i) alive.w[i] = 0;
  if (item < p.work) {
    if (p.mode == kFresh) {
      off = (uint32_t)item;
      range_mask<KS>(p.chunk_base + off, jd.lo, jd.hi, alive);
    } else {
      off = jd.qidx[p.qin][item];
      const uint64_t* src = jd.qmask[p.qin] + item * NW;
#pragma unroll
      for (int i = 0; i < NW; ++i) alive.w[i] = src[i];
    }
    code_planes(p.chunk_base + off, Ep, Op);  // prefix planes of the group (l-KS bases)
  }
  const int wpad = jd.wstride;
  for (int s = p.s0; s < p.s1 && any_set<KS>(alive); ++s) {
    const int r = s - p.s0;
    scan_group_staged<KS>(stage_wp + (size_t)r * (wpad >> 1), stage_sfx + (size_t)r * wpad, wpad,
                          jd.d, Ep, Op, stage_ball, hl, blockDim.x, alive);
  }
  __syncwarp();
  if (p.s1 >= jd.n) {
    group_output<KS>(jd, st, p.chunk_base + off, alive);
  } else {
    const unsigned cnt = any_set<KS>(alive) ? 1u : 0u;
    const unsigned long long slot = warp_reserve(&st->qcount[p.qout], cnt);
    if (cnt) {
      jd.qidx[p.qout][slot] = off;
      uint64_t* dst = jd.qmask[p.qout] + slot * NW;
#pragma unroll
      for (int i = 0; i < NW; ++i) dst[i] = alive.w[i];
    }
  }
}

// REST: the warp owns one queue entry; lanes stride over each remaining sequence's windows in
// global memory, OR their hits locally, and the warp combines the masks.
template <int KS>
__device__ void group_rest(const JobDesc& jd, JobState* st, const Pass& p, unsigned long long item,
                           const uint64_t* stage_ball) {
  constexpr int NW = GroupMask<KS>::NW;
  const int lane = threadIdx.x & 31;
  const uint32_t off = jd.qidx[p.qin][item];
  const uint64_t g = p.chunk_base + off;
  GroupMask<KS> alive;
  const uint64_t* src = jd.qmask[p.qin] + item * NW;
#pragma unroll
  for (int i = 0; i < NW; ++i) alive.w[i] = src[i];
  uint32_t Ep, Op;
  code_planes(g, Ep, Op);
  const uint64_t smask = (1ull << (2 * KS)) - 1;
  for (int s = p.s0; s < jd.n && any_set<KS>(alive); ++s) {
    const uint2* row = jd.planes + (size_t)s * jd.wstride;
    const uint64_t* crow = jd.codes + (size_t)s * jd.wstride;
    GroupMask<KS> matched;
#pragma unroll
    for (int i = 0; i < NW; ++i) matched.w[i] = 0;
    for (int j = lane; j < jd.W; j += 32) {
      const uint2 w = __ldg(row + j);
      const int h = __popc((Ep ^ (w.x >> KS)) | (Op ^ (w.y >> KS)));
      if (h <= jd.d)
        group_hit<KS, true>(matched, stage_ball, jd.d, h, (int)(__ldg(crow + j) & smask));
    }
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      uint64_t v = matched.w[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(kFull, v, o);
      alive.w[i] &= v;
    }
  }
  if (lane != 0) {
#pragma unroll
    for (int i = 0; i < NW; ++i) alive.w[i] = 0;
  }
  group_output<KS>(jd, st, g, alive);
}

// ---------------------------------------------------------------------------------------------
// GROUP, prefix-tiled (k = 4, 256 lanes per CTA).
//
// The CTA owns 256 consecutive groups g = T*256 + lane: they share the first l-8 bases (P1)
// and differ in the last 4 prefix bases (P2 = the lane index as a 4-base code); each lane
// carries the 256 suffixes of its group.  Since Ham = Ham(P1) + Ham(P2) + Ham(suffix), per
// sequence:
//   1. filter: the CTA computes h1 = Ham(P1, window) once per window; only windows with
//      h1 <= d can match any of the tile's 65536 candidates.  A window with h1 = d matches
//      exactly one of them (its own last 8 bases), so its lane sets that bit in a 65536-bit map
//      of the tile in shared memory.  The other windows are compacted into a list of head words
//      (r1 = d - h1, the window's P2 and suffix codes).  For l <= 16 a lane filters four
//      windows at once (filter_packed4), otherwise one;
//   2. after one barrier each lane ORs its 256 bits of the map into its matched mask and clears
//      them; then, 32 listed entries at a time, each warp loads its 32-bit word of each entry's
//      4-base ball-table row (the P2 values within min(r1, 4) of the window's) and transposes
//      the 32 words into one 32-bit mask per lane of the entries it hits (no POPC in this loop);
//   3. hits: per hit entry the lane computes h2 = Ham(P2, window) and ORs in the suffixes
//      within r1 - h2 of the window's last 4 bases.
// A lane with no live candidate left skips its hits; a warp with none skips the scan; the CTA
// stops when no lane has a live candidate (the skip).  Every sequence is handled inside the
// tile, so this pass accepts its survivors directly.

// One hit of the lane whose P2 code is p2 on a listed entry with head word e: OR in the
// suffixes within r1 - h2 of the window's last 4 bases.
__device__ __forceinline__ void tiled_hit(GroupMask<4>& matched, uint32_t e, uint32_t p2,
                                          const uint64_t* ball) {
  const uint32_t x = ((e >> 12) ^ p2) & 0xFFu;  // the window's P2 code against the lane's
  int r = (int)(e & 15u) - __popc((x | (x >> 1)) & 0x55u);
  r = r < 4 ? r : 4;
  or_ball<4, true>(matched, ball, (int)((e >> 4) & 0xFFu), r);
}

// 32x32 bit-matrix transpose across the warp: on entry lane i holds row i; on exit lane j holds
// column j (bit i of lane j's result = bit j of lane i's input).
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int sh = 16 >> i;
    const uint32_t y = __shfl_xor_sync(kFull, x, sh);
    const bool up = (lane & sh) == 0;
    const uint32_t keep = up ? masks[i] : ~masks[i];
    const uint32_t t = up ? (y << sh) : (y >> sh);
    x = (x & keep) | (t & ~keep);
  }
  return x;
}

// Head word of a listed window: bits 0-3 r1 = d - h1 (clamped to 15), bits 4-11 the suffix
// code, bits 12-19 the P2 code.
// ANDs the survivors of one (tile, sequence block) item into the bitmap, one 64-bit word per
// 64 codes; a group's words all lie inside the bitmap, which covers whole groups of the range.
__device__ __forceinline__ void group_and_bitmap(const JobDesc& jd, uint64_t g,
                                                 const GroupMask<4>& alive) {
  unsigned long long* w =
      reinterpret_cast<unsigned long long*>(jd.bitmap) + (((g << 8) - jd.bm_base) >> 6);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (~alive.w[i]) atomicAnd(w + i, (unsigned long long)alive.w[i]);
}

// Phase 1 of the tiled pass for l <= 16, four windows per lane: the first l - 8 bases of a
// window are byte 1 of its planes, so the lane packs the prefix planes of windows j0..j0+3 into
// one byte each and counts the mismatches with the tile's prefix for all four at once (a
// byte-wise popcount).  Windows within d - 1 are listed, windows at exactly d mark the map, as
// in the one-window form.  Every slot below the row stride holds a window of the row (padding
// repeats one), so the last lane group reads no further than the stride and a repeated window
// only repeats an entry.  P1E4 / P1O4: the tile's prefix planes in every byte.
__device__ __forceinline__ void filter_packed4(const uint2* __restrict__ row,
                                               const uint64_t* __restrict__ crow, int W, int d,
                                               uint32_t P1E4, uint32_t P1O4, uint32_t* head,
                                               uint32_t* map, unsigned* cnt, int tid) {
  const int lane = tid & 31;
  const uint4* row4 = reinterpret_cast<const uint4*>(row);
  const uint32_t over_d = (0x7Fu - (uint32_t)d) * 0x01010101u;  // bit 7 of a byte: count > d
  const uint32_t at_d = (0x80u - (uint32_t)d) * 0x01010101u;     // bit 7 of a byte: count >= d
  const unsigned lt = (1u << lane) - 1u;
  for (int b = 0; b < W; b += 1024) {
    const int j0 = b + 4 * tid;
    uint32_t pass = 0, cnt4 = 0;
    if (j0 < W) {
      const uint4 a = __ldg(row4 + (j0 >> 1));      // windows j0, j0+1: E, O, E, O
      const uint4 c = __ldg(row4 + (j0 >> 1) + 1);  // windows j0+2, j0+3
      const uint32_t e4 = __byte_perm(__byte_perm(a.x, a.z, 0x0051u),
                                      __byte_perm(c.x, c.z, 0x0051u), 0x5410u);
      const uint32_t o4 = __byte_perm(__byte_perm(a.y, a.w, 0x0051u),
                                      __byte_perm(c.y, c.w, 0x0051u), 0x5410u);
      uint32_t x = (e4 ^ P1E4) | (o4 ^ P1O4);  // byte k: the mismatch mask of window j0+k
      x = x - ((x >> 1) & 0x55555555u);
      x = (x & 0x33333333u) + ((x >> 2) & 0x33333333u);
      cnt4 = (x + (x >> 4)) & 0x0F0F0F0Fu;     // byte k: its mismatch count (at most 8)
      pass = ~(cnt4 + over_d) & 0x80808080u;  // count <= d
    }
    const uint32_t keep = pass & ~(cnt4 + at_d);  // count < d: r1 > 0, listed
    const int nk = __popc(keep);
    // exclusive prefix of the lanes' listed counts (0..4) from the three bits of each count
    const unsigned b0 = __ballot_sync(kFull, nk & 1), b1 = __ballot_sync(kFull, nk & 2),
                   b2 = __ballot_sync(kFull, nk & 4);
    const int total = __popc(b0) + 2 * __popc(b1) + 4 * __popc(b2);
    unsigned wb = 0;
    if (lane == 0 && total) wb = atomicAdd(cnt, (unsigned)total);
    unsigned slot = __shfl_sync(kFull, wb, 0) + __popc(b0 & lt) + 2 * __popc(b1 & lt) +
                    4 * __popc(b2 & lt);
    while (pass) {
      const int bit = __ffs(pass) - 1;
      pass &= pass - 1;
      const int k = bit >> 3;
      const uint32_t v = (uint32_t)__ldg(crow + j0 + k) & 0xFFFFu;  // P2 code << 8 | suffix
      const int r1 = d - (int)((cnt4 >> (8 * k)) & 0xFu);
      if (r1 == 0) {
        atomicOr(map + (v >> 5), 1u << (v & 31u));  // one candidate
      } else {
        head[slot++] = (uint32_t)(r1 < 15 ? r1 : 15) | (v << 4);
      }
    }
  }
}

// One item of the tiled pass.  SPLIT = false: the tile at group offset tbase, walked through
// every sequence, its survivors appended (or ORed into the bitmap).  SPLIT = true: the tile and
// the sequences [s_begin, s_end), its survivors ANDed into the bitmap.
// COUNT (counting launches, motif_count_tiled_work): the same pass also adds its unit counts to
// jd.units, see kTiledUnits.
template <bool SPLIT, bool COUNT = false>
__device__ void group_tiled(const JobDesc& jd, JobState* st, const Pass& p,
                            unsigned long long tbase, int s_begin, int s_end, uint32_t* head,
                            uint32_t* map, unsigned* s_cnt /* [2] */) {
  constexpr int KS = 4;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wcap = jd.wstride;
  const unsigned long long item = tbase + tid;
  // (a whole-tile pass has work == chunk_units; the loop bound of a whole tile is read from the
  // descriptor each time, which keeps one register free in the hot loop)
  const bool in_chunk = item < (SPLIT ? p.chunk_units : p.work);
  const uint64_t g = p.chunk_base + item;
  GroupMask<KS> alive;
#pragma unroll
  for (int i = 0; i < 4; ++i) alive.w[i] = 0;
  if (in_chunk) range_mask<KS>(g, jd.lo, jd.hi, alive);
  uint32_t E, O;
  code_planes(g, E, O);  // prefix planes (l-4 bases); the lane's P2 code is tid
  const uint32_t P1E = E >> 4, P1O = O >> 4;  // identical in every lane of the tile
  if (tid == 0) s_cnt[SPLIT ? (s_begin & 1) : 0] = 0;
  unsigned long long u_visits = 0, u_marks = 0, u_rounds = 0, u_witer = 0, u_hits = 0, u_list = 0;
  int live = __syncthreads_or(any_set<KS>(alive) ? 1 : 0);
  for (int s = SPLIT ? s_begin : 0; s < (SPLIT ? s_end : jd.n) && live; ++s) {
    unsigned* cnt = s_cnt + (s & 1);
    if (COUNT) ++u_visits;
    // 1. filter the windows by the shared prefix (the list count was zeroed before the
    //    barrier that precedes this phase)
    const uint2* row = jd.planes + (size_t)s * wcap;
    const uint64_t* crow = jd.codes + (size_t)s * wcap;
    if (jd.l <= 16) {
      filter_packed4(row, crow, jd.W, jd.d, P1E * 0x01010101u, P1O * 0x01010101u, head, map,
                     cnt, tid);
    } else {  // one window per lane
      for (int b = 0; b < jd.W; b += 256) {
        const int j = b + tid;
        bool keep = false;
        uint32_t e = 0;
        if (j < jd.W) {
          const uint2 w = __ldg(row + j);
          const int r1 = jd.d - __popc(((w.x >> 8) ^ P1E) | ((w.y >> 8) ^ P1O));
          if (r1 >= 0) {
            const uint32_t v = (uint32_t)__ldg(crow + j) & 0xFFFFu;  // P2 code << 8 | suffix
            if (r1 == 0) atomicOr(map + (v >> 5), 1u << (v & 31u));   // one candidate
            keep = r1 > 0;
            e = (uint32_t)(r1 < 15 ? r1 : 15) | (v << 4);
          }
        }
        const unsigned bal = __ballot_sync(kFull, keep);
        unsigned wb = 0;
        if (lane == 0 && bal) wb = atomicAdd(cnt, (unsigned)__popc(bal));
        wb = __shfl_sync(kFull, wb, 0);
        if (keep) head[wb + __popc(bal & ((1u << lane) - 1u))] = e;
      }
    }
    if (tid == 0) s_cnt[(s + 1) & 1] = 0;  // the next sequence's list count
    __syncthreads();
    const int K = (int)*cnt;
    const bool lane_live = any_set<KS>(alive);
    if (COUNT) {
      u_list += (unsigned long long)K;
      // the tile map's bits are the windows at prefix distance d (one candidate each); read
      // here before this lane clears its bits
      const uint4* own = reinterpret_cast<const uint4*>(map) + 2 * tid;
      const uint4 m0 = own[0], m1 = own[1];
      u_marks += __popc(m0.x) + __popc(m0.y) + __popc(m0.z) + __popc(m0.w) + __popc(m1.x) +
                 __popc(m1.y) + __popc(m1.z) + __popc(m1.w);
    }
    // 2. take this lane's bits of the map (the P2 code of lane tid is tid) and clear them;
    //    then scan 32 listed entries at a time: a warp transpose turns the entries' words for
    //    this warp's 32 lanes into one 32-bit hit mask per lane.  3. OR in each hit's suffix ball.
    GroupMask<KS> matched;
    {
      uint4* own = reinterpret_cast<uint4*>(map) + 2 * tid;
      const uint4 m0 = own[0], m1 = own[1];
      matched.w[0] = (uint64_t)m0.x | ((uint64_t)m0.y << 32);
      matched.w[1] = (uint64_t)m0.z | ((uint64_t)m0.w << 32);
      matched.w[2] = (uint64_t)m1.x | ((uint64_t)m1.y << 32);
      matched.w[3] = (uint64_t)m1.z | ((uint64_t)m1.w << 32);
      own[0] = make_uint4(0u, 0u, 0u, 0u);
      own[1] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (__any_sync(kFull, lane_live)) {
      const uint32_t* ball32 = reinterpret_cast<const uint32_t*>(jd.ball);
      for (int k = 0; k < K; k += 32) {
        // this warp's word (its 32 lanes) of the ball row (P2_w, min(r1, 4)) of entry k+lane
        uint32_t x = 0;
        if (k + lane < K) {
          const uint32_t e = head[k + lane];
          const uint32_t r1 = e & 15u;
          x = __ldg(ball32 + (((e >> 12) & 0xFFu) * (KS + 1) + (r1 < 4u ? r1 : 4u)) * 8u + warp);
        }
        x = warp_transpose32(x, lane);
        if (!lane_live) x = 0;
        if (COUNT) {
          ++u_rounds;
          u_hits += __popc(x);
          u_witer += __reduce_max_sync(kFull, (unsigned)__popc(x));
        }
        while (x) {
          const int i = __ffs(x) - 1;
          x &= x - 1;
          tiled_hit(matched, head[k + i], (uint32_t)tid, jd.ball);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) alive.w[i] &= matched.w[i];
    // One barrier: the list may be rebuilt, and the tile stops once no lane has a live candidate.
    live = __syncthreads_or(any_set<KS>(alive) ? 1 : 0);
  }
  if (COUNT) {
    // per tile: visits, windows filtered, listed and map marks once (thread 0 / summed map
    // bits); scan rounds and warp hit iterations once per warp; hits of every lane
    for (int o = 16; o > 0; o >>= 1) {
      u_marks += __shfl_down_sync(kFull, u_marks, o);
      u_hits += __shfl_down_sync(kFull, u_hits, o);
    }
    if (tid == 0) {
      atomicAdd(jd.units + 0, u_visits);
      atomicAdd(jd.units + 1, u_visits * (unsigned long long)jd.W);
      atomicAdd(jd.units + 3, u_list);
    }
    if (lane == 0) {
      atomicAdd(jd.units + 2, u_marks);
      atomicAdd(jd.units + 4, u_rounds);
      atomicAdd(jd.units + 5, u_witer);
      atomicAdd(jd.units + 6, u_hits);
    }
  }
  if (SPLIT) {
    if (in_chunk) group_and_bitmap(jd, g, alive);
  } else {
    group_output<KS>(jd, st, g, alive);
  }
}

// ---------------------------------------------------------------------------------------------
// End of a step, shared by every step-kernel variant: the last CTA to finish advances every job
// to its next pass (and, inside a graph's while loop, sets the loop condition).  All threads of
// the CTA call it.
__device__ void finish_step(const JobDesc* __restrict__ jobs, JobState* states, int njobs,
                            StepCtl* ctl, cudaGraphConditionalHandle cond, int use_cond,
                            int* s_last, unsigned* s_act) {
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->ctas_done, 1u);
    *s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (!*s_last) return;
  __threadfence();
  unsigned active = 0;
  for (int j = tid; j < njobs; j += blockDim.x) {
    JobState* st = &states[j];
    if (ld_volatile(&st->done)) continue;
    const JobDesc jd = jobs[j];
    const Pass p = make_pass(jd, st);
    const unsigned long long cur = ld_volatile(&st->cursor);
    if (cur > 0 || p.work == 0) st->steps += 1;
    if (cur >= p.work) {  // the pass is complete
      st->cursor = 0;
      const bool chunk_done = p.s1 >= jd.n || ld_volatile(&st->qcount[p.qout]) == 0;
      if (chunk_done) {
        const unsigned long long next = ld_volatile(&st->chunk) + 1;
        st->chunk = next;
        st->pass_seq = 0;
        st->qcount[0] = 0;
        if (next >= jd.nchunks) st->done = 1;
      } else {
        st->pass_seq = p.s1;
        st->qsel = p.qout;
        st->qcount[1 - p.qout] = 0;
      }
    }
    if (!ld_volatile(&st->done)) ++active;
  }
  for (int o = 16; o > 0; o >>= 1) active += __shfl_down_sync(kFull, active, o);
  if (lane == 0) s_act[tid >> 5] = active;
  __syncthreads();
  if (tid == 0) {
    unsigned tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_act[w];
    const unsigned steps = ctl->steps + 1;
    ctl->active_jobs = tot;
    ctl->steps = steps;
    __threadfence();
    ctl->ctas_done = 0;
    if (use_cond) {
      // Inside a graph's while loop: run another step while work remains, never beyond the
      // step bound (which ends the loop even if a job failed to complete).
      const bool more = tot > 0 && (ctl->max_steps == 0 || steps < ctl->max_steps);
      cudaGraphSetConditional(cond, more ? 1u : 0u);
    }
  }
}

// ---------------------------------------------------------------------------------------------
// The step kernel.

// KIND = MOTIF_KERNEL_CAND with P = candidates per lane, or MOTIF_KERNEL_GROUP with P = ks.
// SPLIT (GROUP, P = 4 only): the tiled pass also runs jobs split into (tile, sequence block)
// items; without it the whole-tile loop carries none of that code.
// Shared memory: staged windows of the pass (CAND: planes; GROUP: prefix planes, suffix values
// and one hit list per thread).
template <int KIND, int P, bool SPLIT>
__global__ void __launch_bounds__(kMaxBlock) step_kernel(const JobDesc* __restrict__ jobs,
                                                         JobState* states, int njobs,
                                                         StepCtl* ctl,
                                                         cudaGraphConditionalHandle cond,
                                                         int use_cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ JobDesc s_jd;
  __shared__ Pass s_pass;
  __shared__ int s_skip;
  __shared__ unsigned s_tiles;
  __shared__ int s_last;
  __shared__ unsigned s_act[kMaxBlock / 32];
  __shared__ unsigned long long s_tbase;
  __shared__ unsigned s_tcnt[2];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const unsigned budget = ctl->tiles_per_warp * (blockDim.x >> 5);
  const int first = ctl->rotate ? (int)(blockIdx.x % (unsigned)njobs) : 0;
  if (tid == 0) s_tiles = 0;

  for (int jj = 0; jj < njobs; ++jj) {
    int j = first + jj;
    if (j >= njobs) j -= njobs;
    __syncthreads();
    if (tid == 0) {
      int skip = 1;
      if (!ld_volatile(&states[j].done) && (budget == 0 || s_tiles < budget)) {
        s_jd = jobs[j];
        s_pass = make_pass(s_jd, &states[j]);
        skip = ld_volatile(&states[j].cursor) >= s_pass.work;
      }
      s_skip = skip;
    }
    __syncthreads();
    if (s_skip) continue;
    const JobDesc& jd = s_jd;
    const Pass p = s_pass;
    JobState* st = &states[j];
    const int wpad = jd.wstride;
    const int nst = (p.mode == kRest || p.mode == kTiled) ? 0 : p.s1 - p.s0;

    // Stage the windows of the pass (and, for GROUP, the ball table) in shared memory.
    const uint4* stage4 = reinterpret_cast<const uint4*>(smem);
    const uint16_t* stage_sfx = nullptr;
    const uint64_t* stage_ball = nullptr;
    uint32_t* hits = nullptr;
    if (KIND == MOTIF_KERNEL_CAND) {
      uint4* dst = reinterpret_cast<uint4*>(smem);
      const uint4* src = reinterpret_cast<const uint4*>(jd.planes + (size_t)p.s0 * wpad);
      for (int i = tid; i < nst * (wpad >> 1); i += blockDim.x) dst[i] = src[i];
    } else if (KIND == MOTIF_KERNEL_BITSLICE) {
      const int nblkp = ((jd.W + 127) >> 7) << 2;
      for (int q = 0; q < nst; ++q)
        stage_bitslice(reinterpret_cast<uint32_t*>(smem) + (size_t)q * nblkp * 4 * jd.l,
                       jd.planes + (size_t)(p.s0 + q) * wpad, jd.W, jd.l, nblkp);
    } else {
      // The ball table stays in global memory (read through L1 only for the rare hits);
      // shared memory holds the staged prefix planes, suffix values and the hit lists.
      const size_t wp_bytes = (size_t)kMaxStageSeqs * wpad * 8;
      size_t hit_off = wp_bytes + (size_t)kMaxStageSeqs * wpad * 2;
      hit_off += 16 - hit_off % 16;
      uint2* dwp = reinterpret_cast<uint2*>(smem);
      uint16_t* dsfx = reinterpret_cast<uint16_t*>(smem + wp_bytes);
      const uint64_t smask = (1ull << (2 * P)) - 1;
      for (int i = tid; i < nst * wpad; i += blockDim.x) {
        const uint2 pl = jd.planes[(size_t)p.s0 * wpad + i];
        dwp[i] = make_uint2(pl.x >> P, pl.y >> P);
        dsfx[i] = (uint16_t)(jd.codes[(size_t)p.s0 * wpad + i] & smask);
      }
      stage_sfx = dsfx;
      stage_ball = jd.ball;
      hits = reinterpret_cast<uint32_t*>(smem + hit_off) + tid;
    }
    __syncthreads();

    if (KIND == MOTIF_KERNEL_GROUP && P == 4 && p.mode == kTiled) {
      // CTA-wide tiles of 256 groups: the tile map of single-candidate windows (8 KB; it starts
      // cleared and every tile leaves it cleared), then the list heads.
      uint32_t* map = reinterpret_cast<uint32_t*>(smem);
      uint32_t* head = map + 2048;
      for (int i = tid; i < 2048; i += blockDim.x) map[i] = 0u;
      for (;;) {
        __syncthreads();
        if (tid == 0) {
          unsigned long long b = ~0ull;
          if (budget == 0 || atomicAdd(&s_tiles, blockDim.x >> 5) < budget)
            b = atomicAdd(&st->cursor, (unsigned long long)blockDim.x);
          s_tbase = b;
        }
        __syncthreads();
        const unsigned long long b = s_tbase;
        if (b >= p.work) break;
        if constexpr (SPLIT) {
          if (jd.seq_block > 0) {  // item b / 256 = (sequence block, tile), blocks outermost
            const unsigned long long tiles = (p.chunk_units + 255) / 256, u = b >> 8;
            const int s0 = (int)(u / tiles) * jd.seq_block;
            const int s1 = s0 + jd.seq_block < jd.n ? s0 + jd.seq_block : jd.n;
            group_tiled<true>(jd, st, p, (u % tiles) << 8, s0, s1, head, map, s_tcnt);
            continue;
          }
        }
        group_tiled<false>(jd, st, p, b, 0, 0, head, map, s_tcnt);
      }
      continue;
    }
    // Pull tiles until the pass is exhausted (or the step's tile budget is spent).
    const bool seeded_fresh = KIND != MOTIF_KERNEL_GROUP && p.mode == kFresh && jd.seed;
    const unsigned long long tile = seeded_fresh ? 1024 : tile_of(KIND, P, p.mode);
    for (;;) {
      unsigned long long base = 0;
      int stop = 0;
      if (lane == 0) {
        if (budget != 0 && atomicAdd(&s_tiles, 1u) >= budget) {
          stop = 1;
        } else {
          base = atomicAdd(&st->cursor, tile);
          stop = base >= p.work;
        }
      }
      stop = __shfl_sync(kFull, stop, 0);
      if (stop) break;
      base = __shfl_sync(kFull, base, 0);
      if (KIND == MOTIF_KERNEL_CAND || KIND == MOTIF_KERNEL_BITSLICE) {
        if (p.mode == kRest) cand_rest(jd, st, p, base);
        else if (seeded_fresh) seeded_fresh_tile(jd, st, p, base);
        else if (p.mode == kFresh) cand_tile<KIND, P>(jd, st, p, base, stage4);
        else cand_tile<KIND, 1>(jd, st, p, base, stage4);
      } else {
        if (p.mode == kRest) group_rest<P>(jd, st, p, base, stage_ball);
        else group_tile<P>(jd, st, p, base, stage4, stage_sfx, stage_ball, hits);
      }
    }
  }

  finish_step(jobs, states, njobs, ctl, cond, use_cond, &s_last, s_act);
}

// Resets the states of a job table and its step control block.
__global__ void init_steps_kernel(JobState* states, int njobs, StepCtl* ctl, unsigned max_steps,
                                  unsigned tiles_per_warp, unsigned rotate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < njobs) {
    unsigned long long* w = reinterpret_cast<unsigned long long*>(&states[i]);
    for (int k = 0; k < (int)(sizeof(JobState) / 8); ++k) w[k] = 0;
  }
  if (i == 0) {
    ctl->ctas_done = 0;
    ctl->tiles_per_warp = tiles_per_warp;
    ctl->active_jobs = (unsigned)njobs;
    ctl->steps = 0;
    ctl->max_steps = max_steps;
    ctl->rotate = rotate;
  }
}

// ---------------------------------------------------------------------------------------------
// Counting kernel: the canonical algorithmic window-compare tally (per candidate, sequences in
// input order, windows left to right up to the first match, W for a sequence without one, and
// nothing after it).

__global__ void __launch_bounds__(256) count_kernel(const JobDesc* __restrict__ job,
                                                    unsigned long long* total) {
  const JobDesc jd = *job;
  unsigned long long local = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = jd.lo + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < jd.hi;
       k += stride) {
    uint32_t E, O;
    code_planes(k, E, O);
    for (int s = 0; s < jd.n; ++s) {
      // Ragged or masked rows: this row's own window count, and only valid windows match.
      const uint2* row = jd.planes + (size_t)s * jd.wstride;
      const uint8_t* ok = jd.valid ? jd.valid + (size_t)s * jd.wstride : nullptr;
      const int W = jd.wrow ? jd.wrow[s] : jd.W;
      int j = 0;
      for (; j < W; ++j) {
        const uint2 w = __ldg(row + j);
        if (__popc((E ^ w.x) | (O ^ w.y)) <= jd.d && (!ok || ok[j])) break;
      }
      if (j < W) {
        local += (unsigned long long)(j + 1);
      } else {
        local += (unsigned long long)W;
        break;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(kFull, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(total, local);
}

// Canonical (group, window) prefix-compare tally of the GROUP formulation: per group,
// sequences in input order, windows left to right up to and including the first window after
// which every live candidate of the group has matched (W when some live candidate has no window
// within d); live candidates that found no window are dropped; a group with none left stops.
template <int KS>
__global__ void __launch_bounds__(256) count_group_kernel(const JobDesc* __restrict__ job,
                                                          unsigned long long* total) {
  const JobDesc jd = *job;
  const uint64_t smask = (1ull << (2 * KS)) - 1;
  unsigned long long local = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = jd.unit_lo + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < jd.unit_hi;
       g += stride) {
    GroupMask<KS> alive;
    range_mask<KS>(g, jd.lo, jd.hi, alive);
    uint32_t Ep, Op;
    code_planes(g, Ep, Op);
    for (int s = 0; s < jd.n && any_set<KS>(alive); ++s) {
      GroupMask<KS> matched;
#pragma unroll
      for (int i = 0; i < GroupMask<KS>::NW; ++i) matched.w[i] = 0;
      const uint2* row = jd.planes + (size_t)s * jd.wstride;
      const uint64_t* crow = jd.codes + (size_t)s * jd.wstride;
      int scanned = jd.W;
      for (int j = 0; j < jd.W; ++j) {
        const uint2 w = __ldg(row + j);
        const int h = __popc((Ep ^ (w.x >> KS)) | (Op ^ (w.y >> KS)));
        if (h <= jd.d) {
          group_hit<KS, true>(matched, jd.ball, jd.d, h, (int)(__ldg(crow + j) & smask));
          if (covers<KS>(matched, alive)) {
            scanned = j + 1;
            break;
          }
        }
      }
      local += (unsigned long long)scanned;
#pragma unroll
      for (int i = 0; i < GroupMask<KS>::NW; ++i) alive.w[i] &= matched.w[i];
    }
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(kFull, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(total, local);
}

// Ball tables for ks = 1..kMaxKs: entry (v, r) = suffixes within distance r of v.
__global__ void seed_kernel(const uint64_t* __restrict__ codes0, int W,
                            const uint64_t* __restrict__ pat, uint64_t npat, uint64_t lo,
                            uint64_t hi, uint32_t* seed, uint64_t base) {
  const uint64_t total = (uint64_t)W * npat;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = i / npat;
    const uint64_t c = __ldg(codes0 + j) ^ __ldg(pat + (i - j * npat));
    if (c >= lo && c < hi) {
      const uint64_t b = c - base;
      atomicOr(seed + (b >> 5), 1u << (unsigned)(b & 31));
    }
  }
}

// ---------------------------------------------------------------------------------------------
// The step kernel of launches whose every job runs the whole-tile prefix-tiled pass (GROUP,
// k = 4, JobDesc::tiled, no sequence blocks).  Same job walk, tile claiming and end of step as
// step_kernel, with the per-group passes left out: compiled for kTiledMinBlocks resident CTAs per
// SM (48 registers, no spills), against 64 registers and 4 CTAs for step_kernel<GROUP, 4>, and the
// extra warps hide more of the tiled pass's latency.  Shared memory: the 8 KB tile map, then the
// list heads.
constexpr int kTiledMinBlocks = 5;

template <bool COUNT>
__global__ void __launch_bounds__(kMaxBlock, kTiledMinBlocks)
tiled_kernel(const JobDesc* __restrict__ jobs, JobState* states, int njobs, StepCtl* ctl,
             cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ JobDesc s_jd;
  __shared__ Pass s_pass;
  __shared__ int s_skip;
  __shared__ unsigned s_tiles;
  __shared__ int s_last;
  __shared__ unsigned s_act[kMaxBlock / 32];
  __shared__ unsigned long long s_tbase;
  __shared__ unsigned s_tcnt[2];
  const int tid = threadIdx.x;
  const unsigned budget = ctl->tiles_per_warp * (blockDim.x >> 5);
  const int first = ctl->rotate ? (int)(blockIdx.x % (unsigned)njobs) : 0;
  if (tid == 0) s_tiles = 0;
  uint32_t* map = reinterpret_cast<uint32_t*>(smem);
  uint32_t* head = map + 2048;
  for (int i = tid; i < 2048; i += blockDim.x) map[i] = 0u;  // every tile leaves it cleared
  for (int jj = 0; jj < njobs; ++jj) {
    int j = first + jj;
    if (j >= njobs) j -= njobs;
    __syncthreads();
    if (tid == 0) {
      int skip = 1;
      if (!ld_volatile(&states[j].done) && (budget == 0 || s_tiles < budget)) {
        s_jd = jobs[j];
        s_pass = make_pass(s_jd, &states[j]);
        // only whole-tile tiled passes run here (the host routes no other job to this kernel)
        skip = s_pass.mode != kTiled || s_jd.seq_block > 0 ||
               ld_volatile(&states[j].cursor) >= s_pass.work;
      }
      s_skip = skip;
    }
    __syncthreads();
    if (s_skip) continue;
    const JobDesc& jd = s_jd;
    const Pass p = s_pass;
    JobState* st = &states[j];
    for (;;) {
      __syncthreads();
      if (tid == 0) {
        unsigned long long b = ~0ull;
        if (budget == 0 || atomicAdd(&s_tiles, blockDim.x >> 5) < budget)
          b = atomicAdd(&st->cursor, (unsigned long long)blockDim.x);
        s_tbase = b;
      }
      __syncthreads();
      const unsigned long long b = s_tbase;
      if (b >= p.work) break;
      group_tiled<false, COUNT>(jd, st, p, b, 0, 0, head, map, s_tcnt);
    }
  }
  finish_step(jobs, states, njobs, ctl, cond, use_cond, &s_last, s_act);
}

__global__ void ball_kernel(uint64_t* table, int ks) {
  const int nv = 1 << (2 * ks);
  const int nw = mask_words(ks);
  const int entries = nv * (ks + 1) * nw;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < entries; e += gridDim.x * blockDim.x) {
    const int w = e % nw;
    const int r = (e / nw) % (ks + 1);
    const int v = e / (nw * (ks + 1));
    uint64_t word = 0;
    for (int b = 0; b < 64; ++b) {
      const int s = w * 64 + b;
      if (s >= nv) break;
      const uint32_t x = (uint32_t)(s ^ v);
      const int dist = __popc((x | (x >> 1)) & 0x55555555u);
      if (dist <= r) word |= 1ull << b;
    }
    table[e] = word;
  }
}


template <int KIND, int P, bool SPLIT = false>
const void* step_fn() {
  return reinterpret_cast<const void*>(&step_kernel<KIND, P, SPLIT>);
}

const void* step_function(int kind, int p) {
  if (kind == kKindTiledSplit) return p == 4 ? step_fn<MOTIF_KERNEL_GROUP, 4, true>() : nullptr;
  if (kind == kKindTiled)
    return p == 4 ? reinterpret_cast<const void*>(&tiled_kernel<false>) : nullptr;
  if (kind == kKindTiledCount)
    return p == 4 ? reinterpret_cast<const void*>(&tiled_kernel<true>) : nullptr;
  if (kind == MOTIF_KERNEL_CAND) {
    switch (p) {
      case 1: return step_fn<MOTIF_KERNEL_CAND, 1>();
      case 2: return step_fn<MOTIF_KERNEL_CAND, 2>();
      case 4: return step_fn<MOTIF_KERNEL_CAND, 4>();
    }
  } else if (kind == MOTIF_KERNEL_BITSLICE) {
    switch (p) {
      case 1: return step_fn<MOTIF_KERNEL_BITSLICE, 1>();
      case 2: return step_fn<MOTIF_KERNEL_BITSLICE, 2>();
      case 4: return step_fn<MOTIF_KERNEL_BITSLICE, 4>();
    }
  } else if (kind == MOTIF_KERNEL_GROUP) {
    switch (p) {
      case 1: return step_fn<MOTIF_KERNEL_GROUP, 1>();
      case 2: return step_fn<MOTIF_KERNEL_GROUP, 2>();
      case 3: return step_fn<MOTIF_KERNEL_GROUP, 3>();
      case 4: return step_fn<MOTIF_KERNEL_GROUP, 4>();
    }
  }
  return nullptr;
}

}  // namespace

size_t step_smem_bytes(int kind, int p, int wstride, int block) {
  if (kind == kKindTiled || kind == kKindTiledCount)  // the tile map, the list heads
    return 8192 + (size_t)wstride * 4;
  if (kind == kKindTiledSplit) kind = MOTIF_KERNEL_GROUP;
  if (kind == MOTIF_KERNEL_CAND) return (size_t)kMaxStageSeqs * wstride * 8;
  if (kind == MOTIF_KERNEL_BITSLICE)  // 4 words per base position (l <= 32) per 32 windows,
                                      // blocks in fours
    return (size_t)kMaxStageSeqs * (((wstride + 127) / 128) * 4) * 4 * 32 * 4;
  size_t b = (size_t)kMaxStageSeqs * wstride * 10;
  b += 16 - b % 16;
  b += (size_t)kHitCap * block * 4;
  if (p == 4) {  // the prefix-tiled pass: the 8 KB map of single-candidate windows and the
                 // list heads
    const size_t t = 8192 + (size_t)wstride * 4;
    if (t > b) b = t;
  }
  return b;
}

// Raises (never lowers) a variant's dynamic shared memory limit: plans, batches and the server
// share the kernels, and one caller's smaller request must not break another's launch.
cudaError_t step_kernel_attrs(int kind, int p, size_t smem) {
  static std::mutex mu;
  static size_t set[64][kLaunchKinds][kMaxKs + 1] = {};  // per device
  const void* f = step_function(kind, p);
  if (!f || kind < 1 || kind >= kLaunchKinds || p < 1 || p > kMaxKs)
    return cudaErrorInvalidValue;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(mu);
  if (smem <= set[dev][kind][p]) return cudaSuccess;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) set[dev][kind][p] = smem;
  return e;
}

int step_max_ctas_per_sm(int kind, int p, int block, size_t smem) {
  // The occupancy query is asked again for every plan configured: its answers are kept, per
  // device (the same kernel can differ in resident CTAs on another device).
  static std::mutex mu;
  static std::map<std::tuple<int, int, int, int, size_t>, int> known;
  const void* f = step_function(kind, p);
  int dev = 0;
  if (!f || cudaGetDevice(&dev) != cudaSuccess) return 0;
  const auto key = std::make_tuple(dev, kind, p, block, smem);
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = known.find(key);
    if (it != known.end()) return it->second;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, block, smem) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> g(mu);
  known[key] = n;
  return n;
}

cudaError_t launch_step(int kind, int p, const JobDesc* d_jobs, JobState* d_states, int njobs,
                        StepCtl* d_ctl, int grid, int block, size_t smem, cudaStream_t s) {
  const void* f = step_function(kind, p);
  if (!f) return cudaErrorInvalidValue;
  cudaGraphConditionalHandle none = 0;
  int use_cond = 0;
  void* args[] = {(void*)&d_jobs, (void*)&d_states, (void*)&njobs, (void*)&d_ctl, (void*)&none,
                  (void*)&use_cond};
  note_launches(1);
  return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, s);
}

cudaError_t add_step_node(cudaGraph_t g, int kind, int p, const JobDesc* d_jobs,
                          JobState* d_states, int njobs, StepCtl* d_ctl, int grid, int block,
                          size_t smem, cudaGraphConditionalHandle cond, int use_cond,
                          cudaGraphNode_t* node) {
  const void* f = step_function(kind, p);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {(void*)&d_jobs, (void*)&d_states, (void*)&njobs, (void*)&d_ctl, (void*)&cond,
                  (void*)&use_cond};
  cudaKernelNodeParams kp = {};
  kp.func = const_cast<void*>(f);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, nullptr, 0, &kp);
}

cudaError_t launch_init_steps(JobState* d_states, int njobs, StepCtl* d_ctl, unsigned max_steps,
                              unsigned tiles_per_warp, unsigned rotate, cudaStream_t s) {
  init_steps_kernel<<<(njobs + 255) / 256, 256, 0, s>>>(d_states, njobs, d_ctl, max_steps,
                                                        tiles_per_warp, rotate);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t add_init_node(cudaGraph_t g, JobState* d_states, int njobs, StepCtl* d_ctl,
                          unsigned max_steps, unsigned tiles_per_warp, unsigned rotate,
                          cudaGraphNode_t* node) {
  void* args[] = {(void*)&d_states, (void*)&njobs, (void*)&d_ctl, (void*)&max_steps,
                  (void*)&tiles_per_warp, (void*)&rotate};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)init_steps_kernel;
  kp.gridDim = dim3((njobs + 255) / 256);
  kp.blockDim = dim3(256);
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, nullptr, 0, &kp);
}

cudaError_t build_step_graph(int kind, int p, const JobDesc* d_jobs, JobState* d_states,
                             int njobs, StepCtl* d_ctl, int grid, int block, size_t smem,
                             unsigned max_steps, unsigned rotate, cudaGraphExec_t* exec,
                             bool one_step) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphNode_t init;
  e = add_init_node(g, d_states, njobs, d_ctl, max_steps, 0, rotate, &init);
  if (one_step) {  // init -> step: the conditional loop node costs about 15 us per launch
    cudaGraphNode_t step;
    if (e == cudaSuccess)
      e = add_step_node(g, kind, p, d_jobs, d_states, njobs, d_ctl, grid, block, smem, 0, 0,
                        &step);
    if (e == cudaSuccess) e = cudaGraphAddDependencies(g, &init, &step, nullptr, 1);
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return e;
  }
  cudaGraphConditionalHandle h;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t loop;
  if (e == cudaSuccess) e = cudaGraphAddNode(&loop, g, &init, nullptr, 1, &cp);
  cudaGraphNode_t step;
  if (e == cudaSuccess)
    e = add_step_node(cp.conditional.phGraph_out[0], kind, p, d_jobs, d_states, njobs, d_ctl, grid,
                      block, smem, h, 1, &step);
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return e;
}

cudaError_t launch_count(const JobDesc* d_job, unsigned long long* d_total, int grid, int block,
                         cudaStream_t s) {
  count_kernel<<<grid, block, 0, s>>>(d_job, d_total);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_count_group(const JobDesc* d_job, int ks, unsigned long long* d_total, int grid,
                               int block, cudaStream_t s) {
  switch (ks) {
    case 1: count_group_kernel<1><<<grid, block, 0, s>>>(d_job, d_total); break;
    case 2: count_group_kernel<2><<<grid, block, 0, s>>>(d_job, d_total); break;
    case 3: count_group_kernel<3><<<grid, block, 0, s>>>(d_job, d_total); break;
    case 4: count_group_kernel<4><<<grid, block, 0, s>>>(d_job, d_total); break;
    default: return cudaErrorInvalidValue;
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_seed_scatter(const uint64_t* codes0, int W, const uint64_t* pat,
                                uint64_t npat, uint64_t lo, uint64_t hi, uint32_t* seed,
                                uint64_t base, cudaStream_t s) {
  if (W <= 0 || npat == 0) return cudaSuccess;
  const uint64_t total = (uint64_t)W * npat;
  const uint64_t blocks = (total + 255) / 256;
  seed_kernel<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, s>>>(codes0, W, pat, npat,
                                                                         lo, hi, seed, base);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_ball_table(uint64_t* table, int ks, cudaStream_t s) {
  const int entries = ball_table_words(ks);
  ball_kernel<<<(entries + 255) / 256, 256, 0, s>>>(table, ks);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace motif

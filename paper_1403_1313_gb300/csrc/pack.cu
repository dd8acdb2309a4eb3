// K0: window extraction (Sec. IV.A: every window is extracted before the search starts).
//
// Each thread turns one length-l window of one sequence into
//   - its packed 2l-bit code: base i (0 = leftmost) in bits [2(l-1-i), 2(l-1-i)+1], A=0 C=1 G=2
//     T=3, so the code of a window equals the index of the identical candidate l-mer;
//   - its two compressed bit planes: E holds the low bit of every base, O the high bit, base i
//     at plane bit (l-1-i).  Two l-mers differ at base i exactly when E or O differs at bit
//     l-1-i, so their Hamming distance is popc((E1 ^ E2) | (O1 ^ O2)) for every l <= 32.
// Rows are padded to `wstride` windows by repeating the last window: a repeated window
// matches exactly when the original does, so scans may run over the padding unguarded.
#include "motif_internal.h"

namespace motif {
namespace {

__device__ __forceinline__ int base_code(char ch) {
  switch (ch) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
  }
}

__global__ void validate_kernel(const char* __restrict__ chars, int64_t stride, int n, int t,
                                int* err) {
  const int64_t total = (int64_t)n * t;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / t, c = i - r * t;
    if (base_code(chars[r * stride + c]) < 0) atomicOr(err, 1);
  }
}

// Packs every window and, when err is given, validates the characters on the way: with t >= l
// the windows cover every character of every row.
__global__ void pack_kernel(const char* __restrict__ chars, int64_t stride, int n, int t, int l,
                            int wstride, uint2* __restrict__ planes,
                            uint64_t* __restrict__ codes, int* err) {
  const int W = t - l + 1;
  const int64_t total = (int64_t)n * wstride;
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / wstride);
    int j = (int)(i - (int64_t)s * wstride);
    if (j >= W) j = W - 1;  // padding repeats the last window
    const char* p = chars + (int64_t)s * stride + j;
    uint64_t code = 0;
    uint32_t E = 0, O = 0;
    for (int b = 0; b < l; ++b) {
      int v = base_code(p[b]);
      bad |= v < 0;
      v = v < 0 ? 0 : v;
      code = (code << 2) | (uint64_t)v;
      E = (E << 1) | (uint32_t)(v & 1);
      O = (O << 1) | (uint32_t)(v >> 1);
    }
    planes[i] = make_uint2(E, O);
    codes[i] = code;
  }
  if (err && bad) atomicOr(err, 1);
}

// Ragged rows: row s holds lens[s] characters.  A window is valid when it lies inside its row
// and, with masking, contains only ACGTacgt; its code and planes are written as above and its
// flag to valid[].  Invalid positions (masked windows, windows past the row's end, padding) are
// overwritten afterwards by fill_rows_kernel.
__global__ void pack_var_kernel(const char* __restrict__ chars, int64_t stride, int n, int l,
                                int wstride, const int32_t* __restrict__ lens, int mask_unknown,
                                uint2* __restrict__ planes, uint64_t* __restrict__ codes,
                                uint8_t* __restrict__ valid, int* err) {
  const int64_t total = (int64_t)n * wstride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(i / wstride);
    const int j = (int)(i - (int64_t)s * wstride);
    const int W = lens[s] - l + 1;
    uint64_t code = 0;
    uint32_t E = 0, O = 0;
    bool ok = j < W;
    if (ok) {
      const char* p = chars + (int64_t)s * stride + j;
      for (int b = 0; b < l; ++b) {
        int v = base_code(p[b]);
        if (v < 0) {
          if (!mask_unknown) atomicOr(err, 1);
          ok = false;
          v = 0;
        }
        code = (code << 2) | (uint64_t)v;
        E = (E << 1) | (uint32_t)(v & 1);
        O = (O << 1) | (uint32_t)(v >> 1);
      }
    }
    planes[i] = make_uint2(E, O);
    codes[i] = code;
    valid[i] = ok ? 1 : 0;
  }
}

// One warp per row: every invalid position takes the code and planes of the nearest valid
// window before it (or of the row's first valid window when there is none before it).  A
// window that is present twice matches exactly when it matches once, so the search kernels run
// over the filled rows unchanged.  A row with no valid window sets *empty: no candidate can
// match it.
__global__ void fill_rows_kernel(int n, int wstride, const uint8_t* __restrict__ valid,
                                 uint2* __restrict__ planes, uint64_t* __restrict__ codes,
                                 int* empty) {
  const int lane = threadIdx.x & 31;
  const int s = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  if (s >= n) return;
  const uint8_t* v = valid + (int64_t)s * wstride;
  uint2* pl = planes + (int64_t)s * wstride;
  uint64_t* co = codes + (int64_t)s * wstride;
  int first = -1;
  for (int b = 0; b < wstride && first < 0; b += 32) {
    const unsigned bal = __ballot_sync(0xffffffffu, b + lane < wstride && v[b + lane]);
    if (bal) first = b + __ffs(bal) - 1;
  }
  if (first < 0) {
    if (lane == 0) atomicOr(empty, 1);
    return;
  }
  int carry = first;  // the last valid window before the current chunk
  for (int b = 0; b < wstride; b += 32) {
    const int j = b + lane;
    const bool ok = j < wstride && v[j];
    const unsigned bal = __ballot_sync(0xffffffffu, ok);
    const unsigned below = bal & ((1u << lane) - 1u);
    const int src = below ? b + 31 - __clz(below) : carry;
    if (j < wstride && !ok) {
      pl[j] = pl[src];
      co[j] = co[src];
    }
    if (bal) carry = b + 31 - __clz(bal);
  }
}

}  // namespace

cudaError_t launch_pack_var(const char* d_chars, int64_t stride, int n, int l, int wstride,
                            const int32_t* d_lens, int mask_unknown, uint2* planes,
                            uint64_t* codes, uint8_t* valid, int* d_err, int* d_empty,
                            cudaStream_t s) {
  const int block = 256;
  const int64_t wins = (int64_t)n * wstride;
  int grid = (int)((wins + block - 1) / block);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  pack_var_kernel<<<grid, block, 0, s>>>(d_chars, stride, n, l, wstride, d_lens, mask_unknown,
                                         planes, codes, valid, d_err);
  const int rows_per_block = block / 32;
  fill_rows_kernel<<<(n + rows_per_block - 1) / rows_per_block, block, 0, s>>>(
      n, wstride, valid, planes, codes, d_empty);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_pack(const char* d_chars, int64_t stride, int n, int t, int l, int wstride,
                        uint2* planes, uint64_t* codes, int* d_err, cudaStream_t s) {
  const int block = 256;
  const int64_t chars = (int64_t)n * t;
  int grid = (int)((chars + block - 1) / block);
  if (grid > 4096) grid = 4096;
  if (grid < 1) grid = 1;
  if (t < l) {  // no windows: only the characters to check
    if (d_err) {
      validate_kernel<<<grid, block, 0, s>>>(d_chars, stride, n, t, d_err);
      note_launches(1);
    }
    return cudaGetLastError();
  }
  const int64_t wins = (int64_t)n * wstride;
  grid = (int)((wins + block - 1) / block);
  if (grid > 4096) grid = 4096;
  pack_kernel<<<grid, block, 0, s>>>(d_chars, stride, n, t, l, wstride, planes, codes, d_err);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace motif

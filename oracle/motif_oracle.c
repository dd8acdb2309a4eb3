/*
 * ORACLE — test infrastructure, not part of the library.
 *
 * A plain, slow, obviously correct CPU implementation of the Skip-Brute-Force (skip-BF) motif
 * search of Perera & Ragel (Sec. III.A), written over character arrays.  It shares no code with
 * the CUDA path: no packing, no bit tricks, no tables.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * What it computes (Sec. I.A problem, Sec. III.A method):
 *   R(l,d,S) = { c in {A,C,G,T}^l : for every sequence s in S there is a window
 *                s[j .. j+l-1], 0 <= j <= t-l, with Hamming(c, window) <= d },
 * returned as ascending candidate indices.  Candidate index k encodes the l-mer whose base i
 * (0 = leftmost) is "ACGT"[(k >> 2(l-1-i)) & 3], so ascending k is lexicographic order.
 *
 * Steps, in the paper's order: generate each l-mer from its index (Sec. IV.A: l-mers are not
 * generated in advance); compare it with the windows of each sequence by counting mismatched
 * nucleotides (Sec. III.A); it matches a sequence when some window has at most d mismatches;
 * when a sequence has no matching window the l-mer is discarded and the remaining sequences
 * are skipped (Sec. III.A: the skip).  Readings where the paper is silent:
 *   - sequences are visited in input order, windows left to right;
 *   - a sequence's scan stops at its first matching window (the result set does not depend on
 *     this; the compare tally does);
 *   - counting the mismatches of one window may stop once they exceed d.
 *
 * The tally `compares` is the canonical algorithmic window-compare count: per candidate and
 * per visited sequence, j+1 for a first match at window j, or W when no window matches.
 *
 * oracle_skipbf_var takes sequences of different lengths t_s (each sequence has t_s - l + 1
 * windows, none when t_s < l) and may mask characters outside ACGTacgt: a window that contains
 * one never matches, so no l-mer over {A,C,G,T} is within d of it.  Its tally counts every
 * window position, masked or not, the same way (j+1 at the first match, else t_s - l + 1).
 *
 * oracle_skipbf_threads is the paper's multicore decomposition (Sec. IV.A, Fig. 1): the index
 * space is cut into one contiguous range per POSIX thread, each thread searches its range
 * against its own view of the windows, and the per-thread outputs are concatenated in order.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_ALPHABET (-2)
#define ORACLE_ERR_OOM (-4)

static const char kBases[4] = {'A', 'C', 'G', 'T'};

/* Upper-cases one nucleotide character; returns 0 for anything outside ACGTacgt. */
static char oracle_norm(char ch) {
  switch (ch) {
    case 'A': case 'a': return 'A';
    case 'C': case 'c': return 'C';
    case 'G': case 'g': return 'G';
    case 'T': case 't': return 'T';
    default: return 0;
  }
}

/* The l-mer with index k (Sec. IV.A: an l-mer is produced from its number). */
void oracle_lmer_from_index(uint64_t k, int l, char* out) {
  for (int i = 0; i < l; ++i) out[i] = kBases[(k >> (2 * (l - 1 - i))) & 3u];
}

/* Copies the n x t characters to a packed upper-case buffer; ORACLE_ERR_ALPHABET on a bad
 * character.  Nothing is encoded: the search below compares characters. */
static int oracle_copy_seqs(int n, int t, const char* seqs, long long stride, char* dst) {
  for (int s = 0; s < n; ++s)
    for (int j = 0; j < t; ++j) {
      char ch = oracle_norm(seqs[(long long)s * stride + j]);
      if (!ch) return ORACLE_ERR_ALPHABET;
      dst[(long long)s * t + j] = ch;
    }
  return ORACLE_OK;
}

/* Skip-BF over candidate indices [lo, hi) (Sec. III.A, range form of Sec. IV.A).
 * seqs: n rows at seqs + s*stride, already upper-case; row s has lens[s] characters (every row
 * has t when lens is NULL); a 0 character is masked (no window containing it matches).
 * Accepted indices are written ascending to out[0 .. min(count, cap)); *count receives the
 * total accepted; *compares the canonical window-compare tally. */
static void oracle_skipbf_rows(int n, long long stride, const int* lens, int t, int l, int d,
                               const char* seqs, uint64_t lo, uint64_t hi, uint64_t* out,
                               long long cap, long long* count, uint64_t* compares) {
  char lmer[64];
  long long found = 0;
  uint64_t tally = 0;
  for (uint64_t k = lo; k < hi; ++k) {
    oracle_lmer_from_index(k, l, lmer);
    int survives = 1;
    for (int s = 0; s < n && survives; ++s) {
      const char* row = seqs + (long long)s * stride;
      const int W = (lens ? lens[s] : t) - l + 1; /* windows of this sequence (Sec. III.A) */
      int matched = 0;
      for (int j = 0; j < W; ++j) {
        int mismatches = 0;
        for (int i = 0; i < l; ++i) {
          if (row[j + i] == 0) { /* a masked character: this window never matches */
            mismatches = d + 1;
            break;
          }
          if (lmer[i] != row[j + i]) {
            ++mismatches;
            if (mismatches > d) break;
          }
        }
        if (mismatches <= d) { /* window j matches: Hamming distance <= d */
          matched = 1;
          tally += (uint64_t)(j + 1);
          break;
        }
      }
      if (!matched) {       /* no window of sequence s matches: */
        if (W > 0) tally += (uint64_t)W;
        survives = 0;       /* discard the l-mer, skip the remaining sequences */
      }
    }
    if (survives) {
      if (found < cap) out[found] = k;
      ++found;
    }
  }
  *count = found;
  *compares = tally;
}

/* Equal lengths: n rows of t characters, row s at seqs + s*t. */
static void oracle_skipbf_core(int n, int t, int l, int d, const char* seqs, uint64_t lo,
                               uint64_t hi, uint64_t* out, long long cap, long long* count,
                               uint64_t* compares) {
  oracle_skipbf_rows(n, t, NULL, t, l, d, seqs, lo, hi, out, cap, count, compares);
}

static int oracle_check_args(int n, int t, int l, int d, const char* seqs, long long stride) {
  if (n < 1 || t < 1 || l < 1 || l > 31 || d < 0 || !seqs || stride < t) return ORACLE_ERR_ARG;
  return ORACLE_OK;
}

/* Single-threaded skip-BF over [lo, hi).  Returns ORACLE_OK or an error code. */
int oracle_skipbf_range(int n, int t, int l, int d, const char* seqs, long long stride,
                        uint64_t lo, uint64_t hi, uint64_t* out, long long cap,
                        long long* count, uint64_t* compares) {
  int rc = oracle_check_args(n, t, l, d, seqs, stride);
  if (rc) return rc;
  const uint64_t space = 1ull << (2 * l);
  if (hi > space || lo > hi || (cap > 0 && !out) || !count || !compares) return ORACLE_ERR_ARG;
  char* buf = (char*)malloc((size_t)n * (size_t)t);
  if (!buf) return ORACLE_ERR_OOM;
  rc = oracle_copy_seqs(n, t, seqs, stride, buf);
  if (rc == ORACLE_OK) oracle_skipbf_core(n, t, l, d, buf, lo, hi, out, cap, count, compares);
  free(buf);
  return rc;
}

/* Single-threaded skip-BF over [lo, hi) for sequences of different lengths: row s has
 * lens[s] >= 0 characters at seqs + s*stride.  With mask_unknown, a character outside
 * ACGTacgt masks the windows that contain it; without it, it is ORACLE_ERR_ALPHABET. */
int oracle_skipbf_var(int n, const int* lens, int l, int d, const char* seqs, long long stride,
                      int mask_unknown, uint64_t lo, uint64_t hi, uint64_t* out, long long cap,
                      long long* count, uint64_t* compares) {
  if (n < 1 || !lens || l < 1 || l > 31 || d < 0 || !seqs) return ORACLE_ERR_ARG;
  const uint64_t space = 1ull << (2 * l);
  if (hi > space || lo > hi || (cap > 0 && !out) || !count || !compares) return ORACLE_ERR_ARG;
  if (stride < 1) return ORACLE_ERR_ARG;
  for (int s = 0; s < n; ++s)
    if (lens[s] < 0 || lens[s] > stride) return ORACLE_ERR_ARG;
  char* buf = (char*)malloc((size_t)n * (size_t)stride);
  if (!buf) return ORACLE_ERR_OOM;
  int rc = ORACLE_OK;
  for (int s = 0; s < n && rc == ORACLE_OK; ++s)
    for (int j = 0; j < lens[s]; ++j) {
      const char ch = oracle_norm(seqs[(long long)s * stride + j]);
      if (!ch && !mask_unknown) { rc = ORACLE_ERR_ALPHABET; break; }
      buf[(long long)s * stride + j] = ch;
    }
  if (rc == ORACLE_OK)
    oracle_skipbf_rows(n, stride, lens, 0, l, d, buf, lo, hi, out, cap, count, compares);
  free(buf);
  return rc;
}

/* ---- the paper's POSIX-thread decomposition (Sec. IV.A, Fig. 1) ------------------------ */

typedef struct {
  int n, t, l, d;
  const char* seqs; /* this worker's copy of the windows' source characters */
  uint64_t first, last_excl;
  uint64_t* out;
  long long cap, count;
  uint64_t compares;
} oracle_worker;

static void* oracle_worker_main(void* arg) {
  oracle_worker* w = (oracle_worker*)arg;
  /* Count first, then collect: keeps the worker free of reallocation logic. */
  long long need = 0;
  uint64_t cmp = 0;
  oracle_skipbf_core(w->n, w->t, w->l, w->d, w->seqs, w->first, w->last_excl, NULL, 0, &need,
                     &cmp);
  w->compares = cmp;
  w->count = need;
  if (need > 0) {
    w->out = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)need);
    if (w->out) {
      long long again = 0;
      uint64_t cmp2 = 0;
      oracle_skipbf_core(w->n, w->t, w->l, w->d, w->seqs, w->first, w->last_excl, w->out,
                         need, &again, &cmp2);
    }
  }
  return NULL;
}

/* Multi-threaded skip-BF over [lo, hi): `threads` contiguous index ranges of (nearly) equal
 * size, one POSIX thread each, each with its own copy of the sequences; outputs concatenated
 * in range order.  Same outputs as oracle_skipbf_range. */
int oracle_skipbf_threads(int n, int t, int l, int d, const char* seqs, long long stride,
                          uint64_t lo, uint64_t hi, int threads, uint64_t* out, long long cap,
                          long long* count, uint64_t* compares) {
  int rc = oracle_check_args(n, t, l, d, seqs, stride);
  if (rc) return rc;
  const uint64_t space = 1ull << (2 * l);
  if (threads < 1 || hi > space || lo > hi || (cap > 0 && !out) || !count || !compares)
    return ORACLE_ERR_ARG;
  oracle_worker* ws = (oracle_worker*)calloc((size_t)threads, sizeof(oracle_worker));
  pthread_t* tids = (pthread_t*)calloc((size_t)threads, sizeof(pthread_t));
  char** copies = (char**)calloc((size_t)threads, sizeof(char*));
  if (!ws || !tids || !copies) { free(ws); free(tids); free(copies); return ORACLE_ERR_OOM; }
  const uint64_t total = hi - lo;
  int started = 0;
  for (int w = 0; w < threads && rc == ORACLE_OK; ++w) {
    copies[w] = (char*)malloc((size_t)n * (size_t)t);
    if (!copies[w]) { rc = ORACLE_ERR_OOM; break; }
    rc = oracle_copy_seqs(n, t, seqs, stride, copies[w]);
    if (rc) break;
    ws[w].n = n; ws[w].t = t; ws[w].l = l; ws[w].d = d;
    ws[w].seqs = copies[w];
    ws[w].first = lo + (uint64_t)((unsigned __int128)total * (unsigned)w / (unsigned)threads);
    ws[w].last_excl = lo + (uint64_t)((unsigned __int128)total * (unsigned)(w + 1) / (unsigned)threads);
  }
  if (rc == ORACLE_OK) {
    for (int w = 0; w < threads; ++w) {
      if (pthread_create(&tids[w], NULL, oracle_worker_main, &ws[w]) != 0) { rc = ORACLE_ERR_OOM; break; }
      ++started;
    }
    for (int w = 0; w < started; ++w) pthread_join(tids[w], NULL);
  }
  long long found = 0;
  uint64_t tally = 0;
  if (rc == ORACLE_OK) {
    for (int w = 0; w < threads; ++w) {
      if (ws[w].count > 0 && !ws[w].out) { rc = ORACLE_ERR_OOM; break; }
      for (long long i = 0; i < ws[w].count; ++i) {
        if (found < cap) out[found] = ws[w].out[i];
        ++found;
      }
      tally += ws[w].compares;
    }
  }
  for (int w = 0; w < threads; ++w) { free(ws[w].out); free(copies[w]); }
  free(ws); free(tids); free(copies);
  if (rc) return rc;
  *count = found;
  *compares = tally;
  return ORACLE_OK;
}

/*
 * motif.h — C ABI of the GB300 Skip-Brute-Force planted (l,d) motif search library.
 *
 * The method (Perera & Ragel, "Accelerating Motif Finding in DNA Sequences with Multicore
 * CPUs", Sec. III.A): enumerate every l-mer over {A,C,G,T}; compare it with every length-l
 * window of each input sequence by Hamming distance; an l-mer matches a sequence when some
 * window lies within distance d; an l-mer that fails to match a sequence is discarded at once
 * and the remaining sequences are skipped.  The l-mers that match every sequence form the
 * result set (Sec. I.A defines the planted (l,d) problem whose consensus is one member).
 *
 * Conventions shared by every entry point below:
 *  - Every call returns an int status (motif_status); nothing throws across the ABI.
 *  - Sequences are n rows of t characters from "ACGTacgt" (Sec. I.A: n sequences of length t).
 *    A window is a substring of length l; each sequence has W = t - l + 1 windows (Sec. III.A;
 *    the paper writes (n - l) + 1 with n standing for the sequence length there).
 *  - A candidate l-mer c = c_0 c_1 ... c_{l-1} is identified by its 2l-bit code:
 *    A=0, C=1, G=2, T=3, base c_i stored in bits [2(l-1-i), 2(l-1-i)+1].  The candidate index
 *    space [0, 4^l) is exactly the code space (Sec. IV.A: l-mers are generated from their
 *    index, never stored), so ascending codes are lexicographic order of the strings.
 *  - Results are always ascending, duplicate-free codes.
 *  - Argument rules: n >= 1, t >= 1, 1 <= l <= 31 (4^l fits in 64 bits), d >= 0.
 *    d >= l accepts every candidate; t < l yields an empty result (no windows).
 *  - The library owns each plan and every device buffer it allocates; the caller owns every
 *    buffer it passes in.  A plan is not thread-safe; motif_submit and motif_poll are.
 *  - Device work of a plan runs on its stream (motif_opts.stream, a cudaStream_t; NULL = the
 *    legacy default stream).  Pointer arguments named d_* are device pointers, all others host.
 */
#ifndef MOTIF_H_
#define MOTIF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MOTIF_OK = 0,
  MOTIF_PENDING = 1,         /* motif_poll: the job has not finished yet */
  MOTIF_ERR_ARG = -1,        /* an argument breaks the rules above */
  MOTIF_ERR_ALPHABET = -2,   /* a sequence character outside ACGTacgt */
  MOTIF_ERR_CAPACITY = -3,   /* more results than the output capacity; *out_count = required */
  MOTIF_ERR_OOM = -4,        /* a device or host allocation failed */
  MOTIF_ERR_CUDA = -5,       /* a CUDA runtime call failed (or no CUDA device is present) */
  MOTIF_ERR_TIMEOUT = -6,    /* a step loop reached its bound with work left: a polled loop
                                past motif_opts.timeout_ms, or a graph-launched loop at its
                                step bound */
  MOTIF_ERR_BUSY = -7,       /* the serving queue refused the job (queue full) */
  MOTIF_ERR_STATE = -8,      /* wrong call order, e.g. a search before sequences were loaded */
  MOTIF_ERR_NOTFOUND = -9    /* unknown job id */
} motif_status;

/* Search kernel selection. */
typedef enum {
  MOTIF_KERNEL_AUTO = 0,  /* the plan's tuned choice (TILED where it applies, else GROUP) */
  MOTIF_KERNEL_CAND = 1,  /* one candidate per lane: XOR, pair-fold, POPC, running min */
  MOTIF_KERNEL_GROUP = 2, /* one (l-k)-base prefix per lane, its 4^k suffixes as a bit mask */
  MOTIF_KERNEL_TILED = 3, /* GROUP with k = 4 whose first pass tiles 256 lanes by a shared
                             (l-8)-base prefix (needs l >= 8; falls back to GROUP otherwise) */
  MOTIF_KERNEL_BITSLICE = 4 /* CAND with the compare counted bit-sliced: 32 windows per step,
                               a saturating counter in bit planes, no POPC (needs d <= 7; falls
                               back to CAND otherwise) */
} motif_kernel;

/* Which candidates a search enumerates. */
typedef enum {
  MOTIF_SEED_ALL = 0,           /* every index of the range (Sec. IV.A) */
  MOTIF_SEED_NEIGHBOURHOOD = 1  /* only the l-mers within d of a window of the first sequence: the
                                   others cannot match it, so the result is the same.  This is
                                   the candidate pruning of Planted Motif Search, which the paper
                                   lists among the exact methods (Sec. I.A) and as future work
                                   (Sec. VI).  CAND and BITSLICE kernels; the table of difference
                                   patterns (sum over k <= d of C(l,k) 3^k entries) may hold at
                                   most 2^24 of them */
} motif_seed;

/* How a search collects the accepted codes before returning them in ascending order (not in the
 * paper, whose output is the surviving l-mers, Sec. III.A; a GPU design choice). */
typedef enum {
  MOTIF_OUTPUT_AUTO = 0,   /* BITMAP where the expected survivors are dense, else LIST */
  MOTIF_OUTPUT_LIST = 1,   /* append codes to a list, then sort and deduplicate it */
  MOTIF_OUTPUT_BITMAP = 2  /* set one bit per code of the range, then compact the set bits in
                              order; needs (range length)/8 bytes of device memory */
} motif_output;

/* How a search launches its step kernel (not in the paper; a GPU design choice). */
typedef enum {
  MOTIF_LAUNCH_GRAPH = 0,  /* one CUDA graph launch per search: an init kernel, then a
                              conditional while node whose body is the step kernel, so no host
                              round trip separates the passes */
  MOTIF_LAUNCH_DIRECT = 1  /* the step kernel launched from the host once per step (a blocking
                              search polls the job state between groups of steps; a device
                              search launches the step bound).  Same kernels, same result; it
                              lets profilers, which do not list kernels inside conditional graph
                              nodes, see every step launch.  The environment variable
                              MOTIF_NO_GRAPH, set at the first search of a process, selects it
                              for every plan */
} motif_launch;

typedef struct motif_plan_s* motif_plan;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc returns a device
 * pointer of at least `bytes` bytes, usable on `stream`, or NULL on failure. */
typedef void* (*motif_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*motif_free_fn)(void* ptr, void* stream, void* ctx);

typedef struct {
  void* stream;             /* cudaStream_t for all device work of the plan; NULL = default */
  int32_t kernel;           /* motif_kernel */
  int32_t block;            /* threads per CTA; 0 = tuned */
  int32_t ctas_per_sm;      /* resident CTAs per SM of the persistent grid; 0 = tuned */
  int32_t cands_per_thread; /* CAND kernel: candidates a lane carries per fresh tile; 0 = tuned */
  int32_t compact_levels;   /* CAND kernel: sequences with a survivor queue; 0 = tuned */
  int32_t suffix_bases;     /* GROUP kernel: k, suffix bases enumerated in one lane; 0 = tuned */
  int32_t timeout_ms;       /* bound on a polled step loop (batches without a graph, and the
                               profiling mode that launches steps without one): past it the
                               call returns MOTIF_ERR_TIMEOUT with nothing left in flight;
                               0 = 60000.  A graph-launched search ends after its step bound
                               (every chunk needs at most n passes) instead. */
  int32_t output;           /* motif_output */
  motif_alloc_fn alloc;     /* NULL = cudaMallocAsync / cudaFreeAsync on the plan's stream */
  motif_free_fn free;
  void* alloc_ctx;
  uint64_t range_lo;        /* candidate sub-range [range_lo, range_hi) of [0, 4^l), the */
  uint64_t range_hi;        /* per-worker index range of Sec. IV.A; range_hi == 0: all */
  int32_t seed;             /* motif_seed */
  int32_t seq_block;        /* prefix-tiled pass with BITMAP output: sequences per work item
                               (a tile and a block of sequences, ANDed into the bitmap); 0 =
                               chosen so the items fill the GPU, -1 = one item walks a tile
                               through every sequence */
  int32_t launch;           /* motif_launch (searches of this plan alone; a batch or a server
                               launches its own graphs) */
} motif_opts;

typedef struct {
  uint64_t candidates;           /* candidates in the searched range */
  uint64_t survivors;            /* codes accepted by the last search */
  uint64_t algorithmic_compares; /* canonical window-compare count (motif_count_compares) */
  double search_ms;              /* device time of the search kernel, last search */
  double sort_ms;                /* device time of sort/dedup, last search */
  double total_ms;               /* host wall time of the last motif_search or served job */
  double queue_ms;               /* served job: submit -> admission; batched job: the part of its
                                    batch's device-to-host result copies that outlasts the last
                                    table's sorts */
  int64_t device_bytes;          /* device memory held by the plan */
  int32_t smem_bytes;            /* dynamic shared memory per CTA of the search kernel */
  int32_t kernel;                /* kernel that ran (motif_kernel) */
  int32_t grid;                  /* CTAs launched */
  int32_t block;                 /* threads per CTA */
  double search_ms_sum;          /* device time of the search kernels, summed over the */
  double sort_ms_sum;            /* searches since the previous motif_stats call, and of */
  int64_t searches;              /* sort/dedup; `searches` is how many were summed */
} motif_stats_t;

/* ---- plans ------------------------------------------------------------------------------ */

/* Fills *o with defaults: every field zero / NULL (tuned or library defaults). */
void motif_opts_default(motif_opts* o);

/* Creates a plan for an (l,d) search over n sequences of length t (Sec. I.A; the inputs of
 * Sec. IV.A: the sequences, the pattern length l and the allowed mutations d).  Validates the
 * argument rules, reserves the device buffers and fixes the kernel configuration.  opts may be
 * NULL.  *out receives the plan, released by motif_plan_destroy.
 * Errors: MOTIF_ERR_ARG, MOTIF_ERR_OOM, MOTIF_ERR_CUDA. */
int motif_plan_create(int32_t n, int32_t t, int32_t l, int32_t d, const motif_opts* opts,
                      motif_plan* out);

/* Releases the plan and its device memory (after its stream has drained).  NULL is a no-op. */
void motif_plan_destroy(motif_plan p);

/* ---- input: window extraction (Sec. IV.A: windows are extracted before the search) ------ */

/* Copies n rows of t characters (row r at seqs + r*stride, stride >= t) to the device and
 * packs every window into its 2l-bit code (a 64-bit word) and two l-bit planes (the low and
 * the high bit of every base, one 32-bit word each).  Returns once the characters are
 * validated and the caller's buffer may be reused: a load of at most 64 KB is checked and
 * staged on the host (its upload and packing may still be in flight on the plan's stream); a
 * larger one is checked on the device before the return.  A character outside ACGTacgt returns
 * MOTIF_ERR_ALPHABET (the plan then holds no sequences).
 * Errors: MOTIF_ERR_ARG, MOTIF_ERR_ALPHABET, MOTIF_ERR_OOM, MOTIF_ERR_CUDA. */
int motif_load_seqs(motif_plan p, const char* seqs, int64_t stride);

/* Same as motif_load_seqs for characters already in device memory (d_seqs, row stride
 * `stride` bytes).  Asynchronous on the plan's stream; an invalid character is recorded on
 * the device and reported as MOTIF_ERR_ALPHABET by the next motif_search (for
 * motif_search_device, through *d_out_count = -1). */
int motif_load_seqs_device(motif_plan p, const char* d_seqs, int64_t stride);

/* Loads n sequences of their own lengths (the paper uses one length, Sec. IV.B, and names real
 * and larger sequence data as future work, Sec. VI).  Row r holds lengths[r] characters,
 * 0 <= lengths[r] <= min(t, stride), at seqs + r*stride; it has lengths[r] - l + 1 windows
 * (none when shorter than l).  With mask_unknown != 0 a character outside ACGTacgt (such as N)
 * masks every window that contains it: a masked window matches no candidate.  With
 * mask_unknown == 0 such a character is MOTIF_ERR_ALPHABET.  A sequence without an unmasked
 * window leaves nothing to accept (the search returns no codes).  motif_count_compares counts
 * every window position of each row, masked or not; motif_count_work's unit tally counts the
 * packed rows, in which masked and missing windows are copies of valid windows of the same row.
 * Blocking.  Errors: MOTIF_ERR_ARG, MOTIF_ERR_ALPHABET, MOTIF_ERR_OOM, MOTIF_ERR_CUDA. */
int motif_load_seqs_var(motif_plan p, const char* seqs, int64_t stride, const int32_t* lengths,
                        int32_t mask_unknown);

/* Parses FASTA text (not in the paper; the input format of real sequence data): a record
 * starts with a line beginning with '>' (the header, not kept); the following lines up to the
 * next header hold its residues; whitespace is dropped and lines beginning with ';' are
 * comments.  The residues of all records are written back to back to seq_buf and their counts
 * to lengths[0 .. records); *n_out and *total_out receive the numbers of records and residues.
 * Host-only: no device work.  If max_seqs or buf_cap is too small the return is
 * MOTIF_ERR_CAPACITY with *n_out and *total_out set (nothing else is promised): call again
 * with larger buffers.  Residues before the first header are MOTIF_ERR_ARG. */
int motif_fasta_parse(const char* text, int64_t text_len, char* seq_buf, int64_t buf_cap,
                      int32_t* lengths, int32_t max_seqs, int32_t* n_out, int64_t* total_out);

/* ---- search (Sec. III.A skip-BF; Sec. IV.A range split) -------------------------------- */

/* Blocking search over the plan's candidate range.  Writes the accepted codes, ascending and
 * duplicate-free, to out_codes[0 .. *out_count).  If more than `capacity` codes are accepted
 * it returns MOTIF_ERR_CAPACITY with *out_count = the required capacity and promises nothing
 * about out_codes; call again with a larger buffer.  out_codes may be NULL when capacity == 0.
 * Errors: MOTIF_ERR_ARG, MOTIF_ERR_STATE (no sequences), MOTIF_ERR_ALPHABET,
 * MOTIF_ERR_CAPACITY, MOTIF_ERR_OOM, MOTIF_ERR_CUDA, MOTIF_ERR_TIMEOUT. */
int motif_search(motif_plan p, uint64_t* out_codes, int64_t capacity, int64_t* out_count);

/* Asynchronous search on the plan's stream with device-resident output: with LIST output the
 * search kernel appends accepted codes into d_out_codes (capacity entries) and the sort/dedup
 * kernels order them in place; with BITMAP output the ordered compaction writes them there.
 * *d_out_count (one int64 in device memory) receives the number of accepted codes.  If that
 * number exceeds capacity, only the count is meaningful for LIST output (retry with more
 * room); BITMAP output still holds the first `capacity` codes in ascending order.  -1 means
 * an invalid character was loaded.  No host synchronisation. */
int motif_search_device(motif_plan p, uint64_t* d_out_codes, int64_t capacity,
                        int64_t* d_out_count);

/* Runs the counting form of the search over the plan's range and returns in *out the
 * canonical algorithmic window-compare count: per candidate, sequences in input order, each
 * scanned left to right up to and including its first window within distance d, all W
 * windows of the first sequence with none, and no sequence after it.  Blocking. */
int motif_count_compares(motif_plan p, uint64_t* out);

/* Runs the counting forms of the search over the plan's range (blocking).  *compares receives
 * the canonical window-compare tally (as motif_count_compares; for seeded plans too, which skip
 * the first sequence's compares).  *unit_steps receives the same tally for the plan's kernel
 * formulation: for MOTIF_KERNEL_CAND and MOTIF_KERNEL_BITSLICE it equals *compares; for
 * MOTIF_KERNEL_GROUP it counts (group, window) prefix compares: per group of 4^k candidates
 * sharing their first l-k bases, sequences in input order, windows left to right up to and
 * including the first window after which every candidate of the group still alive has a
 * window within d, W for a sequence that leaves none alive, and nothing after it.  Either
 * pointer may be NULL. */
int motif_count_work(motif_plan p, uint64_t* compares, uint64_t* unit_steps);

/* Work units of the whole-tile prefix-tiled pass (the tiled form of the Sec. III.A compare; not
 * in the paper, whose compare is per l-mer): for a plan whose search runs that pass
 * (motif_stats' kernel is MOTIF_KERNEL_TILED and its output is not split into sequence blocks),
 * one search by a counting build of the same kernel fills units[0..7):
 *   [0] tile-sequence visits (a tile is 65,536 candidates sharing their first l - 8 bases; it
 *       visits sequences in order until none of its candidates is left: the skip),
 *   [1] windows filtered (W per visit),
 *   [2] map marks (distinct candidates marked by windows at tile-prefix distance exactly d),
 *   [3] listed windows (tile-prefix distance below d; for l <= 16 the filter takes windows in
 *       fours, and a row's padding slots up to a multiple of 4, copies of its last window, are
 *       listed with it),
 *   [4] scan rounds (per visit, warps with a live lane x ceil(listed / 32)),
 *   [5] warp hit iterations (per scan round, the largest hit count of one live lane of the warp),
 *   [6] lane hits (suffix-ball ORs of live lanes).
 * The codes of that search land in the plan's own buffers; the next motif_search repeats it.
 * Blocking.  MOTIF_ERR_STATE for other plans or before a load. */
int motif_count_tiled_work(motif_plan p, uint64_t* units);

/* For a plan with MOTIF_SEED_NEIGHBOURHOOD: *out receives how many candidates of its range lie
 * within d of some window of the first loaded sequence (the candidates its search scans from
 * the second sequence on).  Blocking.  MOTIF_ERR_STATE for other plans or before a load. */
int motif_seed_count(motif_plan p, uint64_t* out);

/* Statistics of the plan: the last search / served job, plus device times summed over every
 * search since the previous call (waits for the plan's stream). */
int motif_stats(motif_plan p, motif_stats_t* s);

/* Kernel launches the library has issued in this process, over all entry points. */
uint64_t motif_kernel_launches(void);

/* ---- batching: many uneven jobs in one persistent launch -------------------------------- */

/* Runs `njobs` loaded plans together in one persistent launch of the batched kernel, which
 * pulls candidate tiles of every job from one device tile queue; use_graph != 0 runs the step
 * loop as one CUDA graph (a conditional while node), instantiated once per batch shape and kept
 * for later batches.  Per job j the results follow motif_search's rules on out_codes[j] /
 * capacities[j] / out_counts[j]; statuses[j] receives job j's status.  Returns MOTIF_OK when
 * every job succeeded, else the first failing status.  Blocking: it waits for each plan's
 * stream, then works on the library's per-device batch streams.  Jobs run as one table per
 * kernel variant.  Where every job of a variant ends in one step (the whole tiled pass over one
 * chunk), its jobs with bitmap output (the dense ones, with large results) form a table of
 * their own that runs first, so that their result copies overlap the steps of the tables after
 * them (out_codes in pinned host memory let the copies run asynchronously at full link rate;
 * pageable buffers are correct but serialise them).  Every job of the batch reports the
 * batch's device times in motif_stats: search_ms and sort_ms summed over its tables, queue_ms
 * the copy time left after the last table's sorts. */
int motif_batch_search(int32_t njobs, const motif_plan* plans, uint64_t* const* out_codes,
                       const int64_t* capacities, int64_t* out_counts, int32_t* statuses,
                       int32_t use_graph);

/* Autotuner: times each candidate configuration (kernel, block, CTAs per SM, candidates per
 * lane, queue levels, suffix bases) on a sub-range of the plan's candidates, keeps the
 * fastest in the plan and in the process-wide cache keyed by (word width, l, d, n, W, SMs),
 * and copies it into *best when best != NULL.  budget_ms bounds the tuning time. */
int motif_autotune(motif_plan p, int32_t budget_ms, motif_opts* best);

/* Saves / loads the process-wide tuning cache as JSON.  MOTIF_ERR_ARG when path is NULL or
 * the file cannot be opened; loading skips entries it cannot parse and entries outside the
 * option rules (kernel, block, candidates per lane, suffix bases, negative counts). */
int motif_tune_cache_save(const char* path);
int motif_tune_cache_load(const char* path);

/* ---- serving: continuous batching (no counterpart in the paper; each job is the Sec. III.A
 * search) ---------------------------------------------------------------------------------- */

typedef struct {
  int32_t max_active;      /* jobs resident on the device at once; 0 = 64 */
  int32_t max_queued;      /* jobs waiting for admission before submit returns BUSY; 0 = 4096 */
  int64_t device_budget;   /* bytes of device memory the admitted jobs may hold; 0 = 8 GiB */
  int32_t step_tiles;      /* candidate tiles one device step may take over all its warps
                              (admissions happen between steps); 0 = 48 per warp, 192 while
                              jobs wait for admission */
  int32_t use_graph;       /* != 0: replay the step launch from a CUDA graph */
  int32_t timeout_ms;      /* not used: each server step is bounded by step_tiles, and callers
                              bound their waits with motif_poll's timeout_ms */
} motif_server_opts;

/* Starts the process-wide serving loop (a scheduler thread with its own stream).  opts may be
 * NULL.  MOTIF_ERR_STATE if it is already running.
 *
 * Admission (between device steps): queued jobs are taken in arrival order while table slots
 * (max_active) and the device budget allow.  The resident table runs one step-kernel variant,
 * chosen by the first job admitted into an empty table (the suffix length k = min(l, 4)); a job
 * that needs another variant waits until the table drains, and later jobs of the table's
 * variant are admitted past it until it has waited 50 ms, after which nothing more is admitted
 * until it is.  A job whose footprint exceeds the remaining budget stops admission. */
int motif_server_start(const motif_server_opts* opts);

/* Stops the serving loop.  The scheduler first runs every submitted job, queued or active, to
 * completion; then the server is released together with the jobs it still holds (results not
 * yet polled are discarded), and their IDs are unknown afterwards (motif_poll returns
 * MOTIF_ERR_NOTFOUND).  It does not wait for motif_submit or motif_poll calls of other threads:
 * call it once no other thread is inside either.  MOTIF_ERR_STATE if no server is running. */
int motif_server_stop(void);

/* Submits the loaded plan as a job (starting the loop with defaults if needed).  The plan's
 * packed windows are copied, so the plan may be reused or destroyed after this returns.
 * *job_id receives the job id.  Errors: MOTIF_ERR_ARG (NULL arguments, or a plan on another
 * device than the running server), MOTIF_ERR_STATE (no sequences), MOTIF_ERR_ALPHABET (an
 * invalid character from motif_load_seqs_device; the plan then holds no sequences),
 * MOTIF_ERR_BUSY (max_queued jobs already wait), MOTIF_ERR_OOM, MOTIF_ERR_CUDA. */
int motif_submit(motif_plan p, int64_t* job_id);

/* Submits a job straight from n host rows of t characters (row r at seqs + r * stride, stride
 * >= t, only ACGTacgt; the inputs of Sec. IV.A), searched for (l, d) by the Sec. III.A skip-BF
 * search as motif_search runs it, without a plan: the job is configured as
 * motif_plan_create would configure a plan with these options (opts may be NULL; its stream and
 * allocator are not used, the server's are), the characters are checked on the host, copied to
 * the device and packed on the server's submit stream.  seqs may be reused once this returns.
 * *job_id receives the job id; poll it with motif_poll.  Errors: MOTIF_ERR_ARG (NULL
 * arguments, stride < t, and motif_plan_create's argument errors), MOTIF_ERR_ALPHABET,
 * MOTIF_ERR_BUSY, MOTIF_ERR_OOM, MOTIF_ERR_CUDA. */
int motif_submit_seqs(const char* seqs, int64_t stride, int32_t n, int32_t t, int32_t l,
                      int32_t d, const motif_opts* opts, int64_t* job_id);

/* Waits up to timeout_ms (0 = do not wait) for the job.  Returns MOTIF_PENDING while it runs;
 * on completion writes the codes by motif_search's rules and releases the job (on
 * MOTIF_ERR_CAPACITY the job stays so that it can be polled again).  stats may be NULL.
 * Errors: MOTIF_ERR_ARG, MOTIF_ERR_NOTFOUND (an unknown or already released id, or no server
 * running), MOTIF_ERR_CAPACITY, and a failed job's own status (MOTIF_ERR_OOM when it can never
 * fit the device budget, MOTIF_ERR_CUDA), after which the job is released. */
int motif_poll(int64_t job_id, uint64_t* out_codes, int64_t capacity, int64_t* out_count,
               int32_t timeout_ms, motif_stats_t* stats);

/* ---- sharding over several workers (Sec. IV.A: per-worker first/last l-mer index) -------- */

/* Splits the candidate space [0, total) into `world` contiguous ranges with sizes in
 * proportion to weights[0..world) (NULL = equal) and returns rank's [*lo, *hi).  Concatenating
 * the per-rank ascending results in rank order gives the global ascending result.
 * Errors: MOTIF_ERR_ARG (world < 1, rank outside [0, world), NULL lo or hi, a negative or NaN
 * weight, weights summing to zero). */
int motif_shard_range(uint64_t total, int32_t rank, int32_t world, const double* weights,
                      uint64_t* lo, uint64_t* hi);

/* ---- helpers ------------------------------------------------------------------------------ */

const char* motif_strerror(int status);

/* Encodes the first l characters of s (ACGTacgt) into a 2l-bit code (layout above).
 * Errors: MOTIF_ERR_ARG (NULL pointers, l outside [1, 31]), MOTIF_ERR_ALPHABET. */
int motif_encode(const char* s, int32_t l, uint64_t* code);

/* Decodes a 2l-bit code into l characters (no terminator written).
 * Errors: MOTIF_ERR_ARG (NULL out, l outside [1, 31], a code of 4^l or more). */
int motif_decode(uint64_t code, int32_t l, char* out);

/* K4 issue-rate probes: operations per SM per clock of one instruction class, measured with
 * one 1024-thread CTA per SM on the current device. */
typedef enum {
  MOTIF_PROBE_POPC = 0,
  MOTIF_PROBE_LOP3 = 1,
  MOTIF_PROBE_IMNMX = 2,
  MOTIF_PROBE_SHF = 3,
  MOTIF_PROBE_IADD = 4,
  MOTIF_PROBE_IMAD = 5,
  MOTIF_PROBE_POPC_LOP3 = 6,   /* 1 POPC + 3 LOP3 on independent chains; rate in POPC+LOP3 ops */
  MOTIF_PROBE_CMP_SPLIT = 7,   /* split-plane window compares */
  MOTIF_PROBE_CMP_FOLD = 8,    /* folded window compares */
  MOTIF_PROBE_LDS64_DIV = 9,   /* 64-bit shared loads at distinct conflict-free addresses */
  MOTIF_PROBE_ATOMS_OR = 10,   /* 32-bit shared-memory atomic ORs (result unused), every lane of
                                  a warp on its own bank */
  MOTIF_PROBE_SHFL = 11,       /* warp butterfly shuffles (shfl.sync.bfly.b32) */
  MOTIF_PROBE_COUNT = 12
} motif_probe_kind;

/* Runs probe `kind` for `iters` loop trips: *ops_per_sm_clk receives its rate and, when
 * sm_cycles != NULL, *sm_cycles the SM cycles it took.  Errors: MOTIF_ERR_ARG, MOTIF_ERR_OOM,
 * MOTIF_ERR_CUDA. */
int motif_probe_rate(int32_t kind, int32_t iters, double* ops_per_sm_clk, double* sm_cycles);

/* ---- ordering codes without allocating ------------------------------------------------------ */

/* Sorts `count` codes at d_codes ascending and removes repeats, in place, without allocating
 * any device memory, and writes the number of distinct codes to *d_unique_count (one int64 in
 * device memory).  The paper has no counterpart: this serves callers that cannot allocate at
 * that point (a host whose framework allocator owns all free device memory, loops that must not
 * block on cudaMalloc / cudaFree).  Its
 * scratch is one fixed array inside the library (about 2.6 MB, held by every device that loads
 * the library until the process exits).  Limits and rules:
 *  - count <= 262144 (2^18); larger counts return MOTIF_ERR_CAPACITY and touch nothing;
 *  - key_bits in [1, 64]: the number of low bits that can be non-zero (2l for l-mer codes);
 *  - asynchronous on `stream` (a cudaStream_t; NULL = the legacy default stream);
 *  - the first call on a device looks up the array's device address (again after the device's
 *    context changes, e.g. after cudaDeviceReset), so make that first call before any stream
 *    capture begins;
 *  - every call uses the same array: calls that overlap on the GPU race and must be serialised
 *    by the caller.
 * Errors: MOTIF_ERR_ARG, MOTIF_ERR_CAPACITY, MOTIF_ERR_CUDA. */
int motif_sort_codes_noalloc(uint64_t* d_codes, int64_t count, int32_t key_bits,
                             int64_t* d_unique_count, void* stream);

/* Library version string. */
const char* motif_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MOTIF_H_ */

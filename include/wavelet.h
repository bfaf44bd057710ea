/*
 * wavelet.h -- C ABI of the GB300 wavelet-tree / wavelet-matrix library.
 *
 * Builds the level bitmaps of wavelet trees and wavelet matrices on one GPU
 * (Shun, "Improved Parallel Construction of Wavelet Trees and Rank/Select
 * Structures"), plus rank/select directories on every level, and answers
 * access / rank / select queries in batches.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Pointers named d_* are device pointers (CUDA global memory of the
 *    current device); h_* are host pointers.  Sizes are element counts.
 *  * `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Builds and queries enqueue their work on it and return
 *    (huff_wt_build finishes its build from a library thread, as stated
 *    there); results are final once the stream is synchronised.  Calls that
 *    hand results to the host
 *    (wt_sync, wt_export, wt_export_select, wt_dd_merge for its parts,
 *    wt_free, wm_autotune, wm_autotune_config) synchronise the handle's stream themselves.  Device-side errors found during
 *    a build (a symbol >= sigma: WT_ERR_SYMBOL_GE_SIGMA; an internal table
 *    that disagrees with the data, which leaves the affected bits unwritten,
 *    or a tile's bulk copy into shared memory that did not complete within
 *    about a second, after which the waiting block stops: WT_ERR_CUDA) are
 *    reported by wt_sync() or by the next call on the handle.
 *  * Symbol sequences are contiguous arrays of width_bytes = 1, 2 or 4
 *    (little-endian unsigned), read-only, borrowed for the duration of the
 *    call and never retained.  n must be below 2^40; longer sequences return
 *    WT_ERR_UNSUPPORTED.
 *  * A build returns WT_OK and a handle in *out, or an error status and
 *    leaves *out == NULL.  The handle owns every array it exports (except
 *    the caller's bitvector for rs_build) until wt_free().
 *  * Level l of a binary structure uses bit L-1-l of the symbol (most
 *    significant first), L = ceil(log2 sigma) and L = 1 for sigma = 1.  Level
 *    bitmaps are u64 words, bit i at word i/64, bit i%64, zero-padded to a
 *    multiple of 2048 bits, levels stored back to back.
 *  * Query semantics (Section 2 of the paper): access(i) = S[i];
 *    rank(c, i) = number of c in S[0..i] (inclusive); select(c, k) = position
 *    of the k-th occurrence of c, k >= 1.  An invalid argument (i >= n,
 *    c >= sigma, k == 0, k > count of c) yields UINT64_MAX in that slot and
 *    does not fail the batch.
 *  * Thread safety: distinct handles may be used from distinct threads;
 *    one handle must not be built/freed concurrently with its own use.
 */
#ifndef GB300_WAVELET_H
#define GB300_WAVELET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WT_OK = 0,
  WT_ERR_INVALID_ARG = 1,      /* bad size, width, sigma, NULL pointer, option */
  WT_ERR_SYMBOL_GE_SIGMA = 2,  /* the sequence holds a symbol >= sigma */
  WT_ERR_NO_MEMORY = 3,        /* device allocation failed */
  WT_ERR_CUDA = 4,             /* a CUDA runtime call failed */
  WT_ERR_TIMEOUT = 5,          /* a serving-loop request has not finished yet */
  WT_ERR_UNSUPPORTED = 6       /* valid but not supported (e.g. sigma too large) */
} wt_status;

typedef struct wt_struct* wt_handle;
typedef void* wt_stream;

/* Build options; a zero field means "choose automatically".
 *  tau           levels per partition pass (1..8); the paper's tau (Sections 3, 4.1).
 *  tile_symbols  symbols per tile; the paper's sub-sequence size n/K (Section 4.2).
 *                wm_build: 2048, 4096 or 8192; the trees, 4-ary trees and batched
 *                builds: 4096 only.  Other values return WT_ERR_UNSUPPORTED.
 *  ctas_per_sm   resident CTAs per SM for the persistent partition kernel (capped
 *                at the kernel's occupancy).
 *  k_chunks      number of tiles K; only 0 (K = ceil(n / tile_symbols)) is
 *                supported.
 *  wm_build fills tau, tile_symbols and ctas_per_sm left at 0 from the
 *  autotuner's record for the sequence's (L, ceil(log2 n)), if any (see
 *  wm_autotune_config), else tau 8, 4096 symbols and the occupancy limit.
 *  select_sample sampling period of the select directory; only 4096 is supported.
 *  flags         WT_FLAG_* below. */
typedef struct {
  uint32_t tau, tile_symbols, ctas_per_sm, k_chunks, select_sample, flags;
} wt_build_opts;

#define WT_FLAG_NO_DIRECTORY 1u  /* skip rank/select directories (timing of the bitmap build) */
#define WT_FLAG_SELECT_O1 2u     /* also build the constant-time select directory of every
                                    level: binary levels (wt/wm/Huffman/rs) and the digit
                                    levels of 4-ary trees (per digit value); not batched */

enum { WT_KIND_WT = 0, WT_KIND_WM = 1, WT_KIND_HUFF = 2, WT_KIND_MULTI = 3, WT_KIND_RS = 4 };

/* Everything a handle holds, for parity checks and export.  Device arrays:
 * bits, dir, samp.  Host arrays (owned by the handle, valid until wt_free):
 * the offset tables, zeros, code_len, code.  For kind MULTI the "levels" are
 * digit levels with bits_per_elem = 2 and dir records of 8 u64. */
typedef struct {
  uint32_t kind;
  uint32_t levels;          /* binary levels, or digit levels (MULTI) */
  uint64_t n;               /* sequence length (bits for RS) */
  uint32_t sigma;
  uint32_t bits_per_elem;   /* 1, or 2 for MULTI */
  uint32_t dir_words_per_rec; /* 2 (binary) or 8 (MULTI) */
  uint32_t max_code_len;    /* HUFF only */
  const uint64_t* bits;     /* device */
  const uint64_t* dir;      /* device */
  const uint64_t* samp;     /* device */
  const uint64_t* level_len;  /* host [levels]: elements on each level */
  const uint64_t* level_off;  /* host [levels+1]: word offset of each level in bits */
  const uint64_t* dir_off;    /* host [levels+1]: u64 offset of each level in dir */
  const uint64_t* samp_off;   /* host [V*levels+1], V = 2 (binary) or 4 (MULTI): u64
                                 offsets into samp; level l holds the positions of
                                 occurrences 0, 4096, 8192, ... of value v from
                                 samp_off[V*l+v] (ceil(count_v/4096) of them; the
                                 offsets are capacities); v = bit value, or digit
                                 value of a MULTI digit level (Section 5.2
                                 generalized select) */
  const uint64_t* zeros;      /* host [levels]: 0 bits per level (binary kinds) */
  const uint8_t* code_len;    /* host [sigma] (HUFF) */
  const uint32_t* code;       /* host [sigma] (HUFF) */
} wt_export_view;

/* Balanced binary wavelet tree, levelwise and pointer-free (paper Section 2,
 * definition of the tree; Section 4.1 integer-sort construction; Section 4.2
 * domain decomposition).  sigma in [1, 2^24]. */
wt_status wt_build(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                   const wt_build_opts* opts, wt_stream stream, wt_handle* out);

/* Wavelet matrix (Section 4.3, wavelet-matrix paragraph): level l holds bit
 * l (from the top) of T_l, T_{l+1} = zeros of T_l then ones, order kept;
 * zeros per level exported.  One pass handles tau levels by a stable
 * partition on the reversed tau-bit digit.  sigma in [1, 2^32-1]. */
wt_status wm_build(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                   const wt_build_opts* opts, wt_stream stream, wt_handle* out);

/* The same wavelet matrix from a sequence in HOST memory: the call enqueues
 * a copy of the n * width_bytes bytes at h_seq into a device buffer of its
 * own (from the library's memory pool), then on `stream` the build wm_build
 * makes of that buffer and the buffer's release, and returns.  The copies
 * of all host-memory builds on a device go, in call order, through one
 * stream of the library's, which `stream` waits for, so that calls on
 * several streams copy one after another while earlier builds run (the
 * library creates that stream on the device's first host-memory build and
 * keeps it for the life of the process: after cudaDeviceReset, host-memory
 * builds on that device are not supported).  h_seq
 * is borrowed until that copy has finished (wt_sync on the handle, or any
 * later synchronisation of `stream`, passes that point); the copy runs
 * asynchronously from page-locked memory, while the driver copies pageable
 * memory before the call returns.  Arguments, result and errors
 * are those of wm_build; in addition, WT_ERR_NO_MEMORY when the device
 * buffer cannot be had and WT_ERR_CUDA when the copy cannot be enqueued,
 * both with *out left NULL. */
wt_status wm_build_host(const void* h_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                        const wt_build_opts* opts, wt_stream stream, wt_handle* out);

/* Huffman-shaped binary wavelet tree (Section 4.3, arbitrarily-shaped
 * trees).  h_code_len: sigma code lengths (0 = absent symbol), or NULL to
 * derive Huffman lengths from the sequence's histogram, limited to 32 bits.
 * Codes are canonical.  Level l holds the elements with code length > l,
 * ordered by their l-bit code prefix; its bit is code bit l.  sigma in
 * [1, 2^24].  The code is built on the host from the sequence's histogram,
 * so this build is asynchronous in a different way from the others: the call
 * enqueues a copy of d_seq on `stream` (d_seq may be released once the
 * stream has passed that point) and returns; a library thread then builds the
 * histogram, the code and the tree on the handle's own stream, which starts
 * after the copy.  Every later call on the handle (queries, wt_sync,
 * wt_export, wt_export_select, wt_query_multi, wt_free, wt_symbol_levels)
 * first waits for that thread and orders its own stream after the build.
 * Errors of the build itself (a symbol >= sigma, caller lengths that leave a
 * present symbol without a code or whose Kraft sum exceeds 1, no memory) are
 * reported by the next call on the handle, as device-side errors are. */
wt_status huff_wt_build(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                        const uint8_t* h_code_len, const wt_build_opts* opts,
                        wt_stream stream, wt_handle* out);

/* Multiary wavelet tree of degree 4 (Section 4.3, multiary trees; Section
 * 5.2 generalized rank): digit level beta keeps binary level 2*beta and
 * stores the 2-bit digit below it (1 bit on the last level when L is odd),
 * 32 digits per u64.  Per-digit-value rank directory per 1024 digits.
 * degree must be 4 (WT_ERR_UNSUPPORTED otherwise).  sigma in [1, 2^24]. */
wt_status multiary_build(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                         uint32_t degree, const wt_build_opts* opts, wt_stream stream,
                         wt_handle* out);

/* Rank/select directory over a caller bitvector (Section 5.1): d_bits holds
 * nbits bits LSB-first in u64 words; bits at positions >= nbits inside the
 * last word must be zero.  The handle keeps a reference to d_bits, which
 * must stay alive and unchanged until wt_free().  Queries use c in {0,1}. */
wt_status rs_build(const uint64_t* d_bits, uint64_t nbits, const wt_build_opts* opts,
                   wt_stream stream, wt_handle* out);

/* Rank/select directory of a bitvector that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc when they need the directory (a component that owns
 * all device memory through its own manager, paths that must not wait on an
 * allocation, runtimes that forbid allocation after start-up).  The build's
 * scratch lives in a static device array of about 4 MiB that every GPU
 * loading this library keeps until the process exits.
 * d_bits: nbits bits LSB-first (bits >= nbits in the last word zero).
 * Outputs, allocated by the caller: d_dir, 2*(ceil(nbits/2048)+1) u64 in the
 * rs_build record layout; d_samp0 / d_samp1, nbits/4096+1 u64 each, receiving
 * the positions of the 0-based 4096k-th zero / one (as rs_build's samples).
 * nbits must be <= 2^30; larger sizes return WT_ERR_UNSUPPORTED.  Each call
 * outside stream capture looks up the array's device address on the current
 * device (so the address stays right after cudaDeviceReset); a call during
 * capture reuses the address of the last call outside capture, so issue a
 * first call on each device before any stream capture.  All calls share the
 * scratch array, so calls whose kernels overlap on the GPU race: order them
 * (e.g. one stream).  WT_ERR_CUDA reports only this call's own launch errors;
 * an error left pending by an earlier, unrelated CUDA call is neither
 * reported nor cleared.  Asynchronous on `stream` like every other call. */
wt_status rs_dir_build_static(const uint64_t* d_bits, uint64_t nbits, uint64_t* d_dir,
                              uint64_t* d_samp0, uint64_t* d_samp1, wt_stream stream);

/* One sequence of a batched build. */
typedef struct {
  const void* d_seq;     /* device, read-only, borrowed for the call */
  uint64_t n;
  uint32_t sigma;
  uint32_t width_bytes;  /* 1, 2 or 4 */
} wt_batch_item;

/* Wavelet matrices of m sequences, with directories, built by one set of
 * launches (Section 4.2's domain decomposition applied across sequences:
 * the tiles of all sequences form one work list of a persistent kernel per
 * pass; class counts are chained only between tiles of one sequence).
 * outs[i] receives the handle of items[i], exactly the structure wm_build
 * returns for it; the m handles share one device allocation, released when
 * the last of them is freed.  opts->tau == 0 takes each sequence's levels
 * per pass from the autotuner's table (8 when not tuned).  Each sequence has
 * its own error word: a symbol >= sigma (WT_ERR_SYMBOL_GE_SIGMA), or a failed
 * internal consistency check of its tiles (WT_ERR_CUDA; never for consistent
 * tables), is reported on that sequence's handle only.  A failed call
 * (invalid argument, no memory, a CUDA error) sets every outs[i] to NULL. */
wt_status wm_batch_build(const wt_batch_item* items, uint32_t m, const wt_build_opts* opts,
                         wt_stream stream, wt_handle* outs);

/* The same batched build behind one object (Section 4.2's decomposition
 * across sub-problems, as wm_batch_build): a caller that builds and releases
 * many sequences per step handles one object instead of m.  *out receives
 * the batch, or NULL on a failed call (the statuses of wm_batch_build).
 * wt_batch_handle(b, i) returns the structure of items[i] (borrowed: valid
 * until wt_batch_free, never passed to wt_free; NULL for i >= m).
 * wt_batch_sync waits for the batch's stream once and writes the status of
 * every sequence into st[0..m) (st may be NULL); it returns WT_OK when every
 * sequence built, else the first failing status.  wt_batch_free releases
 * every structure of the batch (waiting for the work queued on its stream)
 * and the object. */
typedef struct wt_batch_s* wt_batch;
wt_status wm_batch_build_one(const wt_batch_item* items, uint32_t m, const wt_build_opts* opts,
                             wt_stream stream, wt_batch* out);
wt_handle wt_batch_handle(wt_batch b, uint32_t i);
wt_status wt_batch_sync(wt_batch b, wt_status* st);
wt_status wt_batch_free(wt_batch b);

/* Autotuner for the levels per pass tau (Section 4.2: fewer, wider passes
 * against more work per pass).  Times wavelet-matrix builds of d_seq
 * (without directories; one untimed and the best of two timed builds) for
 * tau = 1 .. min(8, L), writes the fastest to *best_tau and the times to
 * ms_out[tau-1] (ms_out may be NULL; 0 where not tried), and records it (with
 * the default tile and occupancy) for every later wm_build / wm_batch_build
 * with opts->tau == 0 of a sequence with the same L and ceil(log2 n).
 * Synchronises the stream. */
wt_status wm_autotune(const void* d_seq, uint64_t n, uint32_t sigma, uint32_t width_bytes,
                      wt_stream stream, uint32_t* best_tau, float* ms_out);
/* A tuned wavelet-matrix configuration. */
typedef struct {
  uint32_t tau;           /* levels per partition pass */
  uint32_t tile_symbols;  /* symbols per tile: 2048, 4096 or 8192 */
  uint32_t ctas_per_sm;   /* resident partition CTAs per SM, 0 = as many as fit */
  uint32_t reserved;
  uint64_t k_chunks;      /* K = ceil(n / tile_symbols), the number of sub-problems */
  float ms;               /* best measured build time (no directories), ms */
} wt_tuning;

/* Autotuner of the whole configuration (Section 4.2: the number of
 * sub-problems K against the per-sub-problem work, and tau against the
 * number of passes).  Times wavelet-matrix builds of d_seq (without
 * directories; one untimed and the best of two timed builds per
 * configuration): first tau = 1 .. min(8, L) at 4096-symbol tiles and full
 * occupancy, then, for the two fastest tau, tiles of 2048 / 4096 / 8192
 * symbols at full occupancy and at 4 and 3 CTAs per SM.  Writes the fastest
 * to *out and records it for every later wm_build with zero options (and the
 * tau for wm_batch_build) of a sequence with the same L and ceil(log2 n).
 * Synchronises the stream. */
wt_status wm_autotune_config(const void* d_seq, uint64_t n, uint32_t sigma,
                             uint32_t width_bytes, wt_stream stream, wt_tuning* out);
/* The configuration a wm_build with zero options takes for a sequence of n
 * symbols over sigma (ms = 0). */
wt_status wm_tuning(uint64_t n, uint32_t sigma, wt_tuning* out);
/* Forgets every recorded configuration. */
void wm_autotune_clear(void);

/* Queries over several structures in one launch: query i applies d_op[i]
 * (0 access, 1 rank, 2 select) with d_c[i] and d_x[i] (i or k) to
 * hs[d_sid[i]].  d_sid[i] >= nh or d_op[i] > 2 yields UINT64_MAX in that
 * slot; otherwise each slot is what wt_access / wt_rank / wt_select return
 * for it.  d_* are device arrays of q entries owned by the caller. */
wt_status wt_query_multi(const wt_handle* hs, uint32_t nh, const uint32_t* d_sid,
                         const uint8_t* d_op, const uint32_t* d_c, const uint64_t* d_x,
                         uint64_t q, uint64_t* d_out, wt_stream stream);

/* Serving loop (no counterpart in the paper): builds and query batches
 * submitted from any thread are served continuously by two worker threads
 * of the library on their own streams.  The build worker admits pending
 * builds in arrival order while the device bytes they need fit in
 * budget_bytes (structures kept plus the running builds' inputs and
 * workspace), and builds every admitted sequence with one wm_batch_build.
 * The query worker gathers every pending query request whose structures are
 * built into one wt_query_multi launch.  A build's request id is also the id
 * of its structure; query requests name structures by those ids.
 * Latency of a request = from its submission to its results in host
 * memory. */
typedef struct wt_server_s* wt_server;
typedef struct {
  uint64_t budget_bytes;       /* > 0 */
  uint32_t max_batch_builds;   /* sequences per batched build (0 = 4096) */
  uint32_t max_batch_queries;  /* queries per launch, whole requests (0 = 2^22) */
} wt_server_opts;
typedef struct {
  wt_status status;
  uint32_t kind;               /* 1 build, 2 queries */
  uint64_t submit_ns, done_ns; /* steady-clock nanoseconds */
} wt_request_info;
typedef struct {
  uint64_t used_bytes, budget_bytes, build_batches, query_launches;
  uint64_t pending_builds, pending_queries, structures;
} wt_server_stats_t;

wt_status wt_server_create(const wt_server_opts* opts, wt_server* out);
/* Wavelet matrix of the host sequence h_seq (copied before returning).
 * *req = request id = structure id.  A build whose own need exceeds the
 * budget ends with WT_ERR_NO_MEMORY; others wait for memory. */
wt_status wt_server_submit_build(wt_server s, const void* h_seq, uint64_t n, uint32_t sigma,
                                 uint32_t width_bytes, uint64_t* req);
/* q queries on host arrays (copied before returning): structure id, op
 * (0 access, 1 rank, 2 select), c, i or k.  A query naming an unknown,
 * failed or released structure yields UINT64_MAX; one naming a structure
 * still being built waits for it. */
wt_status wt_server_submit_queries(wt_server s, uint64_t q, const uint64_t* h_sid,
                                   const uint8_t* h_op, const uint32_t* h_c, const uint64_t* h_x,
                                   uint64_t* req);
/* State of a request.  wait != 0 blocks until it has finished; wait == 0
 * returns WT_ERR_TIMEOUT while it runs.  For a finished query request,
 * h_out (q u64, may be NULL) receives the answers and the request is
 * forgotten.  info (may be NULL) receives status and times. */
wt_status wt_server_poll(wt_server s, uint64_t req, int wait, uint64_t* h_out,
                         wt_request_info* info);
/* The handle of a built structure (owned by the server; valid until the
 * structure is released). */
wt_status wt_server_handle(wt_server s, uint64_t sid, wt_handle* out);
/* Frees a built (or failed) structure once no query launch uses it. */
wt_status wt_server_release(wt_server s, uint64_t sid);
wt_status wt_server_stats(wt_server s, wt_server_stats_t* out);
/* Stops the workers (requests not finished end with WT_ERR_INVALID_ARG) and
 * frees every structure. */
wt_status wt_server_destroy(wt_server s);

/* Batched queries (definitions of Section 2).  q queries; d_i / d_c / d_k /
 * d_out are device arrays of q entries owned by the caller. */
wt_status wt_access(wt_handle h, const uint64_t* d_i, uint64_t q, uint64_t* d_out,
                    wt_stream stream);
wt_status wt_rank(wt_handle h, const uint32_t* d_c, const uint64_t* d_i, uint64_t q,
                  uint64_t* d_out, wt_stream stream);
wt_status wt_select(wt_handle h, const uint32_t* d_c, const uint64_t* d_k, uint64_t q,
                    uint64_t* d_out, wt_stream stream);

/* Domain-decomposition merge (Section 4.2: the K sub-problems' levels are
 * concatenated node by node, at offsets from prefix sums of the node sizes).
 * parts[0..r-1] are wavelet matrices (all of them) or balanced wavelet trees
 * (all of them) of consecutive pieces S_0, ..., S_{r-1} of one sequence,
 * built with the same sigma and with directories; *out receives the
 * structure of the concatenation S_0 S_1 ... S_{r-1}, bit for bit the one a
 * single build of it gives, with its own directories (opts->flags may ask
 * for WT_FLAG_SELECT_O1, or skip them with WT_FLAG_NO_DIRECTORY).  The parts
 * are read (each is synchronised first) and stay valid.  Limits:
 * ceil(log2 sigma) <= 20 and r * 2^ceil(log2 sigma) <= 2^26
 * (WT_ERR_UNSUPPORTED otherwise). */
wt_status wt_dd_merge(const wt_handle* parts, uint32_t r, const wt_build_opts* opts,
                      wt_stream stream, wt_handle* out);

/* Waits for the handle's build stream and returns its deferred status. */
wt_status wt_sync(wt_handle h);

/* Fills *out with views of the handle's arrays (synchronises the stream). */
wt_status wt_export(wt_handle h, wt_export_view* out);

/* The constant-time select directory of one level and value (after Clark,
 * Section 5.1 select; per digit value on the digit levels of a 4-ary tree,
 * Section 5.2 generalized select, with positions and lengths counted in
 * digits; bit = the bit value 0..1, or the digit value 0..3), built with
 * WT_FLAG_SELECT_O1.  Ranges
 * of 4096 occurrences start at the select samples; a range of at least 2^32
 * bits keeps the positions of its occurrences ("huge"); the others keep the
 * offsets of occurrences 256i (i < 16) from the range's start ("sub"), and a
 * sub-range of at least 2^16 bits keeps the offsets of its 256 occurrences
 * ("sparse").  Shorter sub-ranges are searched in the rank directory within
 * their fewer than 2^16 bits, so a select visits a bounded number of words.
 *   desc[k]: huge: 2^63 | first index of the range in huge;
 *            else: index (in sub-ranges of 256) of its first sparse sub-range
 *            | (16-bit mask of its sparse sub-ranges) << 40
 *   sub[16k+i], sparse[256s+j]: u32 offsets (0xffffffff past the last
 *   occurrence; sub is 0 in huge ranges); huge[4096h+j]: u64 positions
 *   (UINT64_MAX past the last occurrence).
 * Device pointers, owned by the handle.  Synchronises the stream. */
typedef struct {
  uint64_t nranges, nhuge, nsparse;
  const uint64_t* desc;    /* nranges */
  const uint32_t* sub;     /* 16 * nranges */
  const uint32_t* sparse;  /* 256 * nsparse */
  const uint64_t* huge;    /* 4096 * nhuge */
} wt_select_view;
wt_status wt_export_select(wt_handle h, uint32_t level, uint32_t bit, wt_select_view* out);

/* Frees the handle and every array it owns (after its stream's work). */
wt_status wt_free(wt_handle h);

/* Number of symbol levels the structure represents (sum of level lengths). */
uint64_t wt_symbol_levels(wt_handle h);

const char* wt_status_str(wt_status s);

/* Copies `bytes` from device memory d_src to host memory h_dst (synchronous;
 * a utility for reading exported arrays). */
wt_status wt_memcpy_d2h(void* h_dst, const void* d_src, uint64_t bytes);

/* Measurement hooks (process-wide; library threads record too): wt_prof_enable(1)
 * starts counting every kernel this library launches and recording CUDA
 * events around each partition-pass launch on its stream; wt_prof_read()
 * waits for those events and returns the kernel count, the number of pass
 * launches and their summed device time in milliseconds, then clears them. */
void wt_prof_enable(int on);
wt_status wt_prof_read(uint64_t* launches, uint64_t* pass_launches, double* pass_ms);

/* Host-side helpers (no GPU needed): Huffman code lengths and canonical
 * codes.  The lengths are those of Huffman's merge with ties broken by
 * (weight, id), leaf id = symbol and internal id = sigma + creation order
 * (computed by a two-queue merge over the leaves sorted by weight), or of
 * package-merge when that code is longer than cap.  wt_huffman_lengths
 * returns the longest length, or 0 with every length 0 when no code exists
 * (no symbol present, or more than 2^cap present symbols); it returns 0
 * without writing h_len when the arguments are out of range (a NULL pointer,
 * cap not in 1..64, sigma > 2^24: the alphabet limit of huff_wt_build).  Used by huff_wt_build (cap 32); exported for
 * testing.  A calling thread keeps its scratch arrays (at most about 126 MB,
 * for alphabets of up to 2^21 symbols) between calls until it exits. */
uint32_t wt_huffman_lengths(const uint64_t* h_hist, uint32_t sigma, uint32_t cap,
                            uint8_t* h_len);
void wt_canonical_codes(const uint8_t* h_len, uint32_t sigma, uint32_t* h_code);

#ifdef __cplusplus
}
#endif
#endif

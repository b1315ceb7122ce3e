/*
 * kmerco.h -- C ABI of the GB300 countBF K-mer counter (KmerCo, arXiv
 * 2305.07545).
 *
 * The library counts K-mers of DNA reads in a countBF: a flat array of
 * 64-bit cells, each holding eta = floor(64 / alpha) counters of alpha bits
 * (Section 2.1).  It has two phases (Section 3, Fig. "Working of KmerCo"):
 *
 *   insertion       every K-mer window of every read is 2-bit packed,
 *                   replaced by its canonical form and hashed by k_h seeded
 *                   hash functions; each hash saturating-increments one
 *                   counter (Algorithm 1, Algorithm 3);
 *   classification  the distinct K-mers are found exactly, each is queried
 *                   for the minimum of its k_h counters, and the distinct
 *                   list is split into trustworthy (estimate > tau) and
 *                   erroneous (estimate <= tau) K-mers (Algorithm 2,
 *                   Algorithm 5).
 *
 * Conventions shared by every call:
 *  - Status: every int-returning call returns KMERCO_OK (0) or one of the
 *    KMERCO_E* codes below; kmerco_strerror() names them.  A non-zero
 *    status leaves the handle usable unless it is KMERCO_ECUDA, after which
 *    only kmerco_destroy() is meaningful.
 *  - Pointers: "host or device" arguments may point to ordinary host memory,
 *    pinned host memory, or CUDA device memory of the handle's device; the
 *    library tells them apart with cudaPointerGetAttributes.
 *  - Ownership: the library owns the countBF, the distinct-key set and the
 *    classification results; the caller owns every buffer it passes and
 *    must keep insert inputs alive until the next synchronising call
 *    (classify, stats, any getter, reset, destroy).
 *  - Streams: all device work of a handle runs in order on its stream
 *    (kmerco_config_t.stream, else a private non-blocking stream).
 *  - Threads: one handle must not be used from two host threads at once;
 *    different handles are independent.
 *  - Keys: a packed K-mer is sum_i code(b_i) * 4^(K-1-i) with A=0, C=1,
 *    G=2, T=3, first base most significant.  For K <= 32 a key is one
 *    uint64_t; for 33 <= K <= 64 it is two uint64_t words, low word first
 *    (the little-endian layout of a 128-bit integer).  Keys are reported in
 *    ascending numeric order, which is lexicographic order of the bases.
 */
#ifndef KMERCO_H
#define KMERCO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define KMERCO_OK 0
#define KMERCO_EINVAL 1   /* an argument is out of range or inconsistent */
#define KMERCO_ENOMEM 2   /* device or pinned allocation failed, or the HBM budget is exceeded */
#define KMERCO_ECUDA 3    /* a CUDA runtime call or kernel launch failed */
#define KMERCO_ETIMEOUT 4 /* a bounded device retry loop gave up; results are incomplete */
#define KMERCO_ESTATE 5   /* call not valid in the handle's state (e.g. a getter before classify) */
#define KMERCO_ESIZE 6    /* the caller's buffer is too small; the required count is returned */

typedef struct kmerco kmerco_t;

/*
 * Device allocator of a handle (kmerco_config_t.dev_alloc / dev_free), so
 * that the library's device memory can come from the caller's own pool (a
 * framework's caching allocator) instead of cudaMalloc.  alloc returns
 * `bytes` of device memory of the handle's device, 16-byte aligned at
 * least, or NULL; stream is the handle's cudaStream_t, on which the block is
 * used.  free returns a block with the size it was allocated with; the
 * library calls it only after the handle's device work has finished (it
 * synchronises the handle's streams first).  ctx is passed through.
 */
typedef void *(*kmerco_alloc_fn)(void *ctx, size_t bytes, void *stream);
typedef void (*kmerco_free_fn)(void *ctx, void *ptr, size_t bytes, void *stream);

/* Options of kmerco_create_ex().  Zero-initialise, then set fields. */
typedef struct {
    int k;                 /* K-mer length, 1..64 (Table 1) */
    uint64_t m;            /* counters requested, >= 1; rounded up to a multiple of eta */
    int counter_bits;      /* alpha, 1..32 (Section 2.1) */
    int nhash;             /* k_h, 1..32 (Table 1) */
    uint32_t threshold;    /* tau, must be < 2^alpha - 1 (Table 1, Algorithm 2) */
    int forward_only;      /* 0: canonical K-mers (Section 2.3, default); 1: forward strand as read */
    void *stream;          /* cudaStream_t to run on; NULL: the library creates its own */
    uint64_t hbm_budget;   /* bytes of device memory the handle may hold; 0: no limit */
    int device;            /* CUDA device ordinal; -1: the current device */
    int update_mode;       /* how counter increments reach the countBF (same result either way):
                              0 automatic; 1 atomic compare-and-swap on each 64-bit cell;
                              2 partitioned: increments grouped by countBF slice and applied in
                              shared memory (needs nhash <= 4 and at most 2^30 cells;
                              otherwise create returns EINVAL) */
    uint64_t dim_x;        /* two-dimensional countBF (Section 2.1, Algorithm 3): dim_x x dim_y
                              cells of eta counters; m is then ignored and m_actual is
                              dim_x * dim_y * eta.  Hash value h selects cell
                              (h mod dim_x, h mod dim_y), stored row-major at
                              (h mod dim_x) * dim_y + (h mod dim_y), and counter h mod eta.
                              Both 0: flat countBF of m counters.  Otherwise both 1..2^24;
                              the paper takes primes from Eq. 1 (kmerco_paper_dims). */
    uint64_t dim_y;
    int canonical_hash;    /* 1: the canonical K-mer is the strand with the smaller H_0 hash
                              (Section 2.3's equation with h = H_0; equal hashes take the
                              reverse complement); 0: the smaller packed value, i.e. the
                              lexicographically smaller strand (default).  Needs
                              forward_only == 0. */
    int whole_file;        /* 1: the reads of one kmerco_insert call are taken as one sequence
                              and windows run across read boundaries (a window spanning the
                              end of one read and the start of the next is counted); 0:
                              windows stay inside reads (default). */
    uint64_t pass_codes;   /* partitioned design: counter increments staged per pass, 1..2^31;
                              0: 2^31.  A batch with more increments is inserted in several
                              passes over consecutive parts of its reads; smaller values bound
                              the scratch memory (about 7 bytes per staged increment with the
                              counting apply: a 4-byte region code and a 2-byte slice code,
                              with headroom; about 10 with the compare-and-swap apply). */
    uint32_t retry_limit;  /* bound of the device retry loops: compare-and-swap retries of one
                              counter update (Algorithm 3's read-modify-write) and probes of one
                              distinct-set insert.  0: 2^22 and 2^20.  A loop that reaches it
                              stops, so the counts are incomplete, and the next classify or
                              stats returns KMERCO_ETIMEOUT; reset clears the state.  Small
                              values exist to exercise that path on contended input. */
    uint64_t max_distinct; /* most distinct keys the handle's distinct list may hold; 0: no
                              limit (it grows with the input).  Keys beyond it are left out of
                              the list and the next classify or stats returns KMERCO_ENOMEM;
                              reset clears the state. */
    kmerco_alloc_fn dev_alloc;  /* device allocator of every buffer of the handle; both NULL:
                                   cudaMalloc / cudaFree.  Only one of the two set: EINVAL. */
    kmerco_free_fn dev_free;
    void *alloc_ctx;       /* passed to dev_alloc and dev_free */
} kmerco_config_t;

/* Running totals and results of one handle (kmerco_stats). */
typedef struct {
    uint64_t windows;            /* sum over reads of max(0, len - K + 1) (Section 1.1) */
    uint64_t n_skipped;          /* windows holding a byte other than ACGTacgt */
    uint64_t inserted;           /* windows inserted into the countBF = windows - n_skipped */
    uint64_t distinct;           /* distinct canonical K-mers inserted so far */
    uint64_t trustworthy;        /* distinct K-mers with estimate > tau (after classify) */
    uint64_t erroneous;          /* distinct K-mers with estimate <= tau (after classify) */
    uint64_t saturated_counters; /* counters equal to 2^alpha - 1 */
    uint64_t m_actual;           /* counters in the countBF (m rounded up to a multiple of eta) */
    uint64_t words;              /* 64-bit cells: m_actual / eta */
    uint64_t device_bytes;       /* device memory held by the handle */
    uint64_t launches;           /* CUDA kernels this handle has launched since creation */
    uint64_t dim_x, dim_y;       /* two-dimensional geometry, or 0, 0 for a flat countBF */
    int k, counter_bits, eta, nhash;
    uint32_t threshold;
    int classified;              /* 1 when trustworthy/erroneous reflect every insert so far */
    float insert_ms;             /* device time of the last kmerco_insert */
    float classify_ms;           /* device time of the last kmerco_classify */
} kmerco_stats_t;

/*
 * Create a countBF handle (Section 2.1 countBF; Algorithm 1 inputs K, k_h;
 * Algorithm 2 input tau).  Equivalent to kmerco_create_ex() with
 * canonical K-mers, a private stream, no HBM budget and the current device.
 * The countBF (m_actual / eta cells) is allocated and zeroed.
 * Errors: EINVAL when k, counter_bits, nhash or m is out of range or
 * threshold >= 2^counter_bits - 1 (a counter at its maximum could no longer
 * separate the classes; Section 3 after Algorithm 3); ENOMEM; ECUDA.
 * On success *out receives the handle; on error *out is set to NULL.
 */
int kmerco_create(int k, uint64_t m, int counter_bits, int nhash, uint32_t threshold,
                  kmerco_t **out);

/*
 * countBF dimensions by Eq. 1 (Section 2.1): m = -n ln(FPP) / (ln 2)^2
 * (the standard Bloom filter size for n items), v = sqrt(m / 128),
 * dim_x = the smallest prime above v, dim_y = the third prime after dim_x;
 * the countBF then holds dim_x * dim_y cells of 64 bits.  n is the number of
 * items the filter is sized for, fpp the false positive probability.
 * Errors: EINVAL for NULL outputs, n == 0, fpp outside (0, 1), or v >= 2^24.
 */
int kmerco_paper_dims(uint64_t n, double fpp, uint64_t *dim_x, uint64_t *dim_y);

/*
 * Device bytes a handle with options *cfg holds at most after one
 * kmerco_insert of nreads reads (nbytes bases, `windows` windows: the sum of
 * max(0, len - K + 1), or the whole-file count) and one kmerco_classify:
 * the countBF, a distinct set and list sized for every window being a new
 * key, the increment-code buffers of the update design the call would take,
 * the classification buffers for that many distinct keys, and with
 * host_inputs != 0 the staging copy of the reads.  This is the figure a
 * scheduler can admit a job by, and give the handle as its hbm_budget.
 * No device work; cfg->dev_alloc must be NULL.  Errors: EINVAL.
 */
int kmerco_estimate_bytes(const kmerco_config_t *cfg, uint64_t nreads, uint64_t nbytes,
                          uint64_t windows, int host_inputs, uint64_t *bytes);

/* As kmerco_create() with every option of kmerco_config_t. */
int kmerco_create_ex(const kmerco_config_t *cfg, kmerco_t **out);

/* Release the handle and all device memory it holds.  NULL is ignored. */
void kmerco_destroy(kmerco_t *h);

/*
 * Insertion phase (Algorithm 1 with Algorithm 3) over one batch of reads.
 * bases:   host or device, ASCII nucleotides of all reads back to back.
 * offsets: host or device, nreads + 1 non-decreasing uint64 indexes into
 *          bases; read r is bases[offsets[r] .. offsets[r+1]).
 * Every window of K bases inside one read is taken; a window holding any
 * byte other than A, C, G, T (either case) is skipped.  Each window's
 * canonical key (the smaller of the forward and reverse-complement packed
 * values, Section 2.2-2.3) is hashed by H_a = MurmurHash3_x64_128 with seed
 * a, a = 0..k_h-1, first output word; counter g = H_a mod m_actual, cell
 * g / eta, counter g mod eta (a two-dimensional countBF: the cell and
 * counter of kmerco_config_t.dim_x) is incremented unless it already holds
 * 2^alpha - 1.  The key also joins the handle's distinct-key set.
 * Calls accumulate; order of reads and calls does not change any result.
 * Asynchronous on the handle's stream.  The buffers are sized from the
 * call's window count: host offsets of up to 2^16 reads are checked and
 * summed on the host, so the call does not wait for the device; device
 * offsets, and host offsets of more reads, are summed by a kernel whose
 * result the call waits for (copied ahead of the reads, so the wait is for
 * the offsets and the kernel only).  A call that has to grow the distinct set
 * also waits for the keys already held.
 * Errors: EINVAL (NULL pointer with nreads > 0, nreads >= 2^32 - 1,
 * decreasing offsets); ENOMEM; ECUDA.
 */
int kmerco_insert(kmerco_t *h, const char *bases, const uint64_t *offsets, uint64_t nreads);

/*
 * Classification phase (Algorithm 2 with QcountBF-II, Algorithm 5): sort the
 * distinct-key set ascending, estimate each key as 0 if any of its k_h
 * counters is 0 and otherwise their minimum, and split the keys into
 * trustworthy (estimate > tau) and erroneous (estimate <= tau), both kept in
 * ascending order.  The split needs only whether the estimate exceeds tau,
 * so a key's counters are read until one is at or below tau; the full
 * estimates of erroneous keys are computed when kmerco_get_distinct() asks
 * for them.  Synchronises.  Idempotent until the next insert.
 * Errors: ETIMEOUT if an earlier insert's bounded retry loop gave up;
 * EINVAL if an earlier insert found decreasing offsets; ENOMEM; ECUDA.
 */
int kmerco_classify(kmerco_t *h);

/* Fill *s (host pointer) with the handle's totals.  Synchronises; counts
 * saturated counters on the device.  Errors: EINVAL (NULL), ECUDA. */
int kmerco_stats(kmerco_t *h, kmerco_stats_t *s);

/*
 * A 128-bit digest of the countBF cells, computed on the device, so that two
 * countBFs can be compared without copying them out (the serving loop checks
 * that a job's countBF is the same alone and among other jobs).  With
 * f(x) = the MurmurHash3 64-bit finalizer and C = 0x9E3779B97F4A7C15:
 *   out[0] = sum over cells i of f(cell[i] ^ (i * C))            mod 2^64
 *   out[1] = sum over cells i of f(cell[i] + f(i + 1))           mod 2^64
 * Not cryptographic: equal countBFs give equal digests; different ones
 * collide only by chance.  out: host pointer to two uint64_t.
 * Synchronises.  Errors: EINVAL (NULL), ECUDA.
 */
int kmerco_digest(kmerco_t *h, uint64_t *out);

/*
 * Copy the countBF cells (Section 2.1 layout: counter l of a cell in bits
 * [alpha*l, alpha*l + alpha), wasted high bits zero) to dst (host or
 * device).  nwords must be >= stats.words; fewer gives ESIZE.
 */
int kmerco_get_counters(kmerco_t *h, uint64_t *dst, uint64_t nwords);

/*
 * Copy the distinct keys (ascending) and their estimates after
 * kmerco_classify().  keys: host or device, room for cap keys (cap * words
 * per key uint64_t); est: host or device, cap uint32_t, or NULL (the first
 * call with est computes every key's estimate, one query pass).  *n
 * receives the number of distinct keys; keys == NULL only queries it.
 * ESTATE before classify (or after a later insert), ESIZE when cap < *n.
 */
int kmerco_get_distinct(kmerco_t *h, uint64_t *keys, uint32_t *est, uint64_t cap, uint64_t *n);

/* Trustworthy keys (estimate > tau), ascending; same contract as
 * kmerco_get_distinct() without estimates (Algorithm 2, trustworthy file). */
int kmerco_get_trusted(kmerco_t *h, uint64_t *keys, uint64_t cap, uint64_t *n);

/* Erroneous keys (estimate <= tau), ascending (Algorithm 2, erroneous file). */
int kmerco_get_erroneous(kmerco_t *h, uint64_t *keys, uint64_t cap, uint64_t *n);

/*
 * Both classified lists of Algorithm 2 at once, without waiting: the copies
 * of the trustworthy keys to `trusted` (n_trusted * key_words words) and of
 * the erroneous keys to `erroneous` are queued on a result stream of the
 * handle, after the classification, and the call returns.  Either pointer
 * may be NULL (that list is not copied); each is host (pinned, for the copy
 * to run asynchronously) or device memory owned by the caller, with room for
 * tcap / ecap keys.  *nt and *ne receive the list lengths at once.
 *
 * The caller's buffers hold the lists after kmerco_sync(h); until then the
 * caller must neither read nor free them.  Further insert and reset calls
 * run beside the copies (they touch neither list); the next kmerco_classify
 * of this handle waits on the device for them before it rewrites the lists,
 * and on the host only when it must grow the lists' buffer.  Errors: ESTATE
 * (not classified), ESIZE (a cap below its list; nothing queued), ECUDA.
 */
int kmerco_get_lists_async(kmerco_t *h, uint64_t *trusted, uint64_t tcap, uint64_t *erroneous,
                           uint64_t ecap, uint64_t *nt, uint64_t *ne);

/* Waits for all work of the handle: its stream, its host-input copies and
 * its result copies.  Reports a device error flag if one was set. */
int kmerco_sync(kmerco_t *h);

/*
 * QcountBF-II (Algorithm 5) for n arbitrary packed keys: est[i] = 0 when any
 * of key i's k_h counters is zero, else their minimum.  keys and est are
 * host or device (layout as above).  Synchronises.
 */
int kmerco_query(kmerco_t *h, const uint64_t *keys, uint64_t n, uint32_t *est);

/*
 * Merge the countBF and distinct-key set of src into dst, as if dst had also
 * inserted src's reads: every counter becomes min(a + b, 2^alpha - 1), which
 * equals the countBF of the union of both inputs because saturating
 * increments commute (Algorithm 3 read per counter).  Both handles must have
 * the same K, m, counter_bits, nhash and strand mode and the same device;
 * src is left unchanged.  Errors: EINVAL (mismatch), ENOMEM, ECUDA.
 */
int kmerco_merge(kmerco_t *dst, kmerco_t *src);

/*
 * Sharded counting (one sample's reads spread over several handles, on one
 * or several GPUs; the paper counts on one thread, so this is an exchange
 * step of the GPU schedule, exact by Algorithm 3's per-counter saturation):
 *
 * kmerco_merge_cells: counters of cells [first_word, first_word + nwords)
 *   become min(a + b, 2^alpha - 1) with b the counters of src (host or
 *   device, nwords cells in the kmerco_get_counters layout, e.g. another
 *   shard's cells of that range).  Merging every shard's countBF this way
 *   gives the countBF of all shards' reads.  Synchronises.
 *   Errors: EINVAL (NULL), ESIZE (range outside the countBF), ECUDA.
 * kmerco_rank_of: after kmerco_classify, ranks[i] = the number of the
 *   handle's distinct keys below probes[i] (the lower bound of the probe in
 *   the ascending distinct list), for n probe keys (host or device, key
 *   layout as above); ranks is host or device, n uint64.  Cuts the sorted
 *   distinct keys at key-range splitters when routing them to the shard
 *   that owns each range.  Synchronises.  Errors: EINVAL, ESTATE (not
 *   classified), ENOMEM, ECUDA.
 */
int kmerco_merge_cells(kmerco_t *h, const uint64_t *src, uint64_t first_word, uint64_t nwords);
int kmerco_rank_of(kmerco_t *h, const uint64_t *probes, uint64_t n, uint64_t *ranks);

/*
 * Allocation-free classification.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory themselves
 * -- a process whose GPU memory is all reserved up front by its own pool
 * allocator (a serving stack, a framework that owns the device), a plug-in
 * running inside such a host, or a latency-bound path that cannot afford
 * cudaMalloc/cudaFree, which may synchronise the whole device.
 *
 * It computes over caller-owned device buffers what kmerco_classify()
 * computes for a handle:
 *   est[i] = QcountBF-II of keys[i] against the countBF `cells` (m counters
 *            of counter_bits bits, laid out as kmerco_get_counters() returns
 *            them), k_h = nhash hash functions, K = k;
 *   out    = the keys with est > threshold, in input order, followed by the
 *            keys with est <= threshold, in input order (sorted input gives
 *            two sorted lists);
 *   *n_trusted (host memory) = the number of keys with est > threshold.
 * cells, keys (n keys of 1 word for k <= 32, 2 words low-first otherwise),
 * est (n uint32) and out (n keys) are device memory on the current device.
 * m must be a multiple of floor(64 / counter_bits), e.g. stats.m_actual.
 * The countBF is the flat one (addressing g = h mod m); a two-dimensional
 * countBF (kmerco_config_t.dim_x) is classified through its handle instead.
 *
 * Nothing is allocated.  The only scratch is one fixed device array of
 * KMERCO_NOALLOC_MAX_KEYS / 4096 + 1 uint64 (512 KiB + 8 bytes) that every
 * GPU loading this library holds until the process exits.  Hence:
 *  - n above KMERCO_NOALLOC_MAX_KEYS returns KMERCO_EINVAL before any GPU
 *    work;
 *  - every call shares that array, so calls that overlap on the GPU (other
 *    streams, other host threads) race and must be serialised by the caller;
 *  - the first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress, and so does the first call in a new CUDA context
 *    of the device (after cudaDeviceReset); make that first call before
 *    any stream capture.
 * Runs on `stream` (a cudaStream_t; NULL is the legacy default stream) and
 * synchronises it before returning.  Errors: EINVAL (argument out of range,
 * NULL pointer, n too large), ECUDA.
 */
#define KMERCO_NOALLOC_MAX_KEYS 268435456ull
int kmerco_classify_noalloc(const uint64_t *cells, uint64_t m, int k, int counter_bits,
                            int nhash, uint32_t threshold, const uint64_t *keys, uint64_t n,
                            uint32_t *est, uint64_t *out, uint64_t *n_trusted, void *stream);

/*
 * Persistence: a countBF and its distinct keys can be saved with
 * kmerco_get_counters / kmerco_get_distinct and restored into a handle of
 * the same parameters with these two calls (the paper keeps the countBF for
 * later membership and frequency queries, Section 1).
 * kmerco_set_counters: replace the countBF's cells with src (host or device,
 *   nwords == stats.words, the layout of kmerco_get_counters).  ESIZE when
 *   nwords differs.
 * kmerco_add_distinct: add n keys (host or device, the layout of
 *   kmerco_get_distinct: one uint64 each for K <= 32, [lo, hi] pairs
 *   otherwise) to the distinct set; keys already present are ignored.
 *   The window totals of kmerco_stats are not restored.
 * Both leave the handle unclassified.  Errors: EINVAL, ESIZE, ENOMEM, ECUDA.
 */
int kmerco_set_counters(kmerco_t *h, const uint64_t *src, uint64_t nwords);
int kmerco_add_distinct(kmerco_t *h, const uint64_t *keys, uint64_t n);

/* Zero the countBF, empty the distinct set and all totals; keeps memory. */
int kmerco_reset(kmerco_t *h);

/*
 * Batches: many samples, each with its own handle and countBF, inserted
 * together under one CUDA graph.  Two schedules, chosen by a timed
 * autotuner on the first input:
 *   persistent   one kernel launch over the chunks of all samples (atomic
 *                update design), chunk size and resident blocks tuned;
 *   per-sample   each sample's own insert kernels (the partitioned design
 *                where kmerco_insert would use it), samples spread over 1,
 *                2, 4 or 8 concurrent streams, largest first.
 * The per-window work is that of kmerco_insert either way, and so are the
 * results.  The handles must share device, stream, K and the key width;
 * their m, counter_bits and nhash may differ.  The paper counts one sample
 * at a time; batching is a GPU schedule, not a change of method.
 */
typedef struct kmerco_batch kmerco_batch_t;

typedef struct {
    int samples;
    int chunk;            /* window starts per work unit chosen by the autotuner */
    int blocks_per_sm;    /* resident blocks per SM chosen by the autotuner */
    int tuned;            /* 1 after the first reset-insert tuned the schedule */
    float tuned_ms;       /* device time of the best schedule when it was tuned */
    int graph;            /* 1 when a CUDA graph of reset + insert is captured */
    uint64_t launches;    /* kernels launched by the batch */
    uint64_t total_chunks;
    int schedule;         /* 0 persistent launch, 1 per-sample kernels on concurrent streams */
    int streams;          /* streams of the per-sample schedule (0 for the persistent one) */
} kmerco_batch_info_t;

/* Group n handles (not owned; they must outlive the batch).  EINVAL when
 * they differ in device, stream, K or key width, or repeat. */
int kmerco_batch_create(kmerco_t *const *handles, int n, kmerco_batch_t **out);

/* Release the batch (not its handles).  NULL is ignored. */
void kmerco_batch_destroy(kmerco_batch_t *b);

/*
 * Insert sample i's reads (device pointers bases[i], offsets[i], nreads[i],
 * the CSR layout of kmerco_insert) into handle i, all in one launch.  With
 * reset != 0 every handle is first reset (kmerco_reset).  The first reset
 * call times every candidate schedule (persistent: chunk 1024/2048 x
 * resident blocks; per-sample: 1, 2, 4, 8 streams) on this input, keeps the
 * fastest, and captures reset + insert in a CUDA graph; a later call with
 * the same pointers and read counts replays it.  The per-sample schedule
 * holds increment-code scratch per stream for the largest sample.
 * Asynchronous except for the planning of a new input (one readback).
 * Errors: EINVAL (host pointers, decreasing offsets, mixed K); ENOMEM; ECUDA.
 */
int kmerco_batch_insert(kmerco_batch_t *b, const char *const *bases,
                        const uint64_t *const *offsets, const uint64_t *nreads, int reset);

/* Pin the schedule instead of tuning it: schedule 0 persistent launch (chunk
 * 2048, 4 resident blocks per SM or fewer), 1 per-sample kernels on
 * `streams` streams (1, 2, 4 or 8); -1 tunes again on the next reset call.
 * The per-sample schedule falls back to the persistent one when its scratch
 * cannot be allocated.  Errors: EINVAL. */
int kmerco_batch_schedule(kmerco_batch_t *b, int schedule, int streams);

/* Classification of every handle of the batch (the results of
 * kmerco_classify on each): every sample's sort, query and split launched
 * on the batch's concurrent streams with one readback before and one after
 * (and a radix sort afterwards of any run of more than 2^22 keys sharing
 * their top 24 bits); handle by handle when the batch has not set up its
 * streams yet. */
int kmerco_batch_classify(kmerco_batch_t *b);

/* Schedule and counters of the batch. */
int kmerco_batch_info(kmerco_batch_t *b, kmerco_batch_info_t *info);

/* Static description of a status code; never NULL. */
const char *kmerco_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* KMERCO_H */

// Internal declarations of the countBF library: device helpers shared by the
// kernels and the launchers the host API calls.  Nothing here is part of the
// public ABI (include/kmerco.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace countbf {

// ---------------------------------------------------------------- constants
constexpr uint64_t kEmptyKey = ~0ull;      // empty slot of the distinct-key set;
                                           // no canonical key is all ones
constexpr int kChunk = 2048;               // window starts per insert work unit
constexpr int kSmallChunk = 512;           // the same for inputs too small to fill the GPU
constexpr int kPartChunk = 1024;           // the same in the partitioned update design
constexpr int kPartMaxHash = 4;            // hashes the partitioned design stages per window
constexpr int kCoarseBins = 64;            // coarse countBF regions of the partitioned design
constexpr int kSliceShift = 13;            // 2^13 cells (64 KiB) per shared-memory slice
constexpr int kMaxCoarseShift = 24;        // cell-in-region bits of an increment code
constexpr int kMaxFine = 1 << (kMaxCoarseShift - kSliceShift);   // slices per coarse region
constexpr uint64_t kMaxBatchCodes = 1ull << 31;   // increments staged per partitioned pass
constexpr int kRepartTile = 8192;          // codes per repartition block
constexpr int kRepartThreads = 512;
constexpr int kApplyThreads = 1024;        // counting apply
constexpr int kCasApplyThreads = 512;      // compare-and-swap apply: three blocks per SM
constexpr int kHistBits = 16;              // classify: top key bits histogrammed for buckets
constexpr int kHistTile = 65535;           // keys per histogram block (16-bit counters)
constexpr int kHistBins = 1 << kHistBits;
constexpr int kBucketCap = 8192;           // keys one block sorts in shared memory
constexpr int kSubBins = 4096;             // counting-sort bins inside one super-bucket
constexpr int kSubMax = 32;                // largest sub-bin insertion-sorted
constexpr int kBucketThreads = 1024;
constexpr int kScatterTile = 16384;        // keys per bucket-scatter block
constexpr int kMaxSuper = 24576;           // super-buckets the scatter kernel can count
constexpr int kInsertThreads = 256;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;   // keys per radix tile
constexpr int kRadixBits = 8;
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kSplitTile = 4096;
constexpr uint32_t kCasLimit = 1u << 22;   // retries of one counter update
constexpr uint32_t kProbeLimit = 1u << 20; // probes of one distinct-set insert

// Device error bits (DevCounters::error).
constexpr unsigned kErrCasLimit = 1u;
constexpr unsigned kErrProbeLimit = 2u;
constexpr unsigned kErrOffsets = 4u;
constexpr unsigned kErrListFull = 8u;

// Running totals of a handle, resident on the device.
struct DevCounters {
    unsigned long long windows;
    unsigned long long skipped;
    unsigned long long inserted;
    unsigned long long distinct;    // keys appended to the distinct list
    unsigned long long trusted;     // written by classify
    unsigned long long bound;       // window upper bound of the last batch
    unsigned long long first;       // offsets[0] of the last batch
    unsigned long long last;        // offsets[nreads] of the last batch
    unsigned long long saturated;   // written by the saturated-counter count
    unsigned int error;         // sticky kErr* bits
    unsigned int bad_offsets;   // set by the window-bound kernel
};

// countBF geometry (Section 2.1): m counters of alpha bits, eta per cell.
struct Geometry {
    uint64_t *cells;
    uint64_t m;          // counters (a multiple of eta)
    uint64_t words;      // m / eta
    uint64_t m_mask;     // m - 1 when m is a power of two, else 0
    uint64_t maxc;       // 2^alpha - 1
    uint64_t dim_x;      // two-dimensional countBF of dim_x x dim_y cells; 0: flat
    uint64_t dim_y;
    uint64_t mag_m, mag_x, mag_y, mag_eta;   // floor((2^64 - 1) / d) of m, dim_x, dim_y, eta
    int alpha;
    int eta;
    int eta_log2;        // log2(eta) when eta is a power of two, else -1
    int nhash;
    uint32_t cas_limit;    // retries of one counter update before it gives up
    uint32_t probe_limit;  // probes of one distinct-set insert before it gives up
};

// Geometry of a countBF of `words` cells (flat: dim_x == 0) or of
// dim_x * dim_y cells (two-dimensional).  Host side; cells left NULL.
inline Geometry make_geometry(uint64_t words, uint64_t dim_x, uint64_t dim_y, int alpha,
                              int nhash) {
    Geometry G;
    G.cells = nullptr;
    G.alpha = alpha;
    G.eta = 64 / alpha;
    G.nhash = nhash;
    G.dim_x = dim_x;
    G.dim_y = dim_x ? dim_y : 0;
    G.words = dim_x ? dim_x * dim_y : words;
    G.m = G.words * (uint64_t)G.eta;
    G.m_mask = (G.m & (G.m - 1)) == 0 ? G.m - 1 : 0;
    G.maxc = (1ull << alpha) - 1;
    G.eta_log2 = -1;
    for (int b = 0; b < 7; ++b)
        if ((1 << b) == G.eta) G.eta_log2 = b;
    G.mag_m = ~0ull / G.m;
    G.mag_x = dim_x ? ~0ull / dim_x : 0;
    G.mag_y = dim_x ? ~0ull / dim_y : 0;
    G.mag_eta = ~0ull / (uint64_t)G.eta;
    G.cas_limit = kCasLimit;
    G.probe_limit = kProbeLimit;
    return G;
}

// ------------------------------------------------------------ hash family
// H_a(x) = MurmurHash3_x64_128(bytes(x), seed = a).h1 (Appleby's published
// algorithm).  A K <= 32 key is 8 bytes: no 16-byte block, one tail lane.
// A 33..64-mer key is 16 bytes: one block, no tail.

__device__ __forceinline__ uint64_t rotl64(uint64_t x, int r) {
    return (x << r) | (x >> (64 - r));
}

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

constexpr uint64_t kMurC1 = 0x87c37b91114253d5ull;
constexpr uint64_t kMurC2 = 0x4cf5ad432745937full;

// Lane-1 mix of an 8-byte tail; independent of the seed, so it is computed
// once per key and reused for all k_h hashes.
__device__ __forceinline__ uint64_t premix8(uint64_t key) {
    return rotl64(key * kMurC1, 31) * kMurC2;
}

// Both output words of MurmurHash3_x64_128 for an 8-byte key whose lane-1
// mix is k1m.
__device__ __forceinline__ void murmur8(uint64_t k1m, uint32_t seed, uint64_t &o1,
                                        uint64_t &o2) {
    uint64_t h1 = (uint64_t)seed ^ k1m ^ 8ull;
    uint64_t h2 = (uint64_t)seed ^ 8ull;
    h1 += h2;
    h2 += h1;
    h1 = fmix64(h1);
    h2 = fmix64(h2);
    h1 += h2;
    h2 += h1;
    o1 = h1;
    o2 = h2;
}

// Both output words for a 16-byte key (lo bytes first, then hi).
__device__ __forceinline__ void murmur16(uint64_t lo, uint64_t hi, uint32_t seed, uint64_t &o1,
                                         uint64_t &o2) {
    uint64_t h1 = seed, h2 = seed;
    uint64_t k1 = rotl64(lo * kMurC1, 31) * kMurC2;
    h1 ^= k1;
    h1 = rotl64(h1, 27) + h2;
    h1 = h1 * 5 + 0x52dce729ull;
    uint64_t k2 = rotl64(hi * kMurC2, 33) * kMurC1;
    h2 ^= k2;
    h2 = rotl64(h2, 31) + h1;
    h2 = h2 * 5 + 0x38495ab5ull;
    h1 ^= 16ull;
    h2 ^= 16ull;
    h1 += h2;
    h2 += h1;
    h1 = fmix64(h1);
    h2 = fmix64(h2);
    h1 += h2;
    h2 += h1;
    o1 = h1;
    o2 = h2;
}

// h mod d by Barrett reduction with magic = floor((2^64 - 1) / d): the
// quotient estimate floor(h * magic / 2^64) is the true quotient or one less
// (h * magic / 2^64 lies in (h/d - 1, h/d]), so one conditional subtraction
// leaves the exact remainder.  Valid for every d >= 1 and every 64-bit h.
__device__ __forceinline__ uint64_t mod_by(uint64_t h, uint64_t d, uint64_t magic) {
    const uint64_t r = h - __umul64hi(h, magic) * d;
    return r >= d ? r - d : r;
}

// Cell and counter of hash value h (Algorithm 3's addressing).
//   flat:              g = h mod m, cell g / eta, counter g mod eta;
//   two-dimensional:   i = h mod x, j = h mod y, l = h mod eta, cell (i, j)
//                      stored row-major at i * y + j, counter l.
__device__ __forceinline__ void address(const Geometry &G, uint64_t h, uint64_t &cell,
                                        unsigned &slot) {
    if (G.dim_x) {
        cell = mod_by(h, G.dim_x, G.mag_x) * G.dim_y + mod_by(h, G.dim_y, G.mag_y);
        slot = G.eta_log2 >= 0 ? (unsigned)(h & (uint64_t)(G.eta - 1))
                               : (unsigned)mod_by(h, (uint64_t)G.eta, G.mag_eta);
        return;
    }
    const uint64_t g = G.m_mask ? (h & G.m_mask) : mod_by(h, G.m, G.mag_m);
    if (G.eta_log2 >= 0) {
        cell = g >> G.eta_log2;
        slot = (unsigned)(g & (uint64_t)(G.eta - 1));
    } else {
        uint64_t q = __umul64hi(g, G.mag_eta);
        uint64_t r = g - q * (uint64_t)G.eta;
        if (r >= (uint64_t)G.eta) {
            r -= (uint64_t)G.eta;
            ++q;
        }
        cell = q;
        slot = (unsigned)r;
    }
}

// ------------------------------------------------------------ block scan
// Exclusive prefix sum of one value per thread across a block of NT threads
// (a multiple of 32, at most 1024): warp shuffles, then a scan of the warp
// totals by the first warp.  `total` receives the block's sum.  Every thread
// of the block must call it; it synchronises the block.
template <typename T, int NT>
__device__ __forceinline__ T block_exclusive_scan(T v, T &total) {
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps, one block");
    __shared__ T wsum[NT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NT / 32 ? wsum[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) wsum[lane] = w;
    }
    __syncthreads();
    const T before = warp ? wsum[warp - 1] : T(0);
    total = wsum[NT / 32 - 1];
    __syncthreads();
    return before + x - v;
}

// ---------------------------------------------------------------- K-mers
// Reverse complement of a packed K-mer (K <= 32; the key fills the low 2K
// bits, first base most significant): complement every 2-bit code (3 - c == ~c), reverse the order of the
// 2-bit groups, drop the 64 - 2K bits that came from outside the key.
__device__ __forceinline__ uint64_t revcomp64(uint64_t fwd, int K) {
    uint64_t r = __brevll(~fwd);   // reverses bits, so each 2-bit group is also flipped
    r = ((r >> 1) & 0x5555555555555555ull) | ((r & 0x5555555555555555ull) << 1);
    return r >> (64 - 2 * K);
}

// Reverse complement of a 33..64-mer held as the 128-bit value hi:lo (low
// 2K bits used, first base most significant).
__device__ __forceinline__ void revcomp128(uint64_t hi, uint64_t lo, int K, uint64_t &rhi,
                                           uint64_t &rlo) {
    // full 128-bit reverse of ~(hi:lo): new_hi = rev(~lo), new_lo = rev(~hi)
    uint64_t a = __brevll(~lo), b = __brevll(~hi);
    a = ((a >> 1) & 0x5555555555555555ull) | ((a & 0x5555555555555555ull) << 1);
    b = ((b >> 1) & 0x5555555555555555ull) | ((b & 0x5555555555555555ull) << 1);
    // value occupies the top 2K bits of a:b; shift right by 128 - 2K
    int s = 128 - 2 * K;           // 0..62 for K in 33..64
    if (s == 0) {
        rhi = a;
        rlo = b;
    } else {
        rlo = (b >> s) | (a << (64 - s));
        rhi = a >> s;
    }
}

// Generation tag of a distinct set: `tag` in the `mask` bits of a slot's
// top word (the bits above the key); mask 0 when the key leaves fewer than
// two spare bits (a free slot is then all ones).
struct SetTag {
    uint64_t tag;
    uint64_t mask;
};

// ------------------------------------------------------------- launchers
struct InsertArgs {
    const uint8_t *bases;        // points at absolute position `first`
    const uint64_t *offsets;     // nreads + 1 entries
    uint64_t nreads;
    uint64_t first, last;        // offsets[0], offsets[nreads]
    const uint32_t *first_read;  // per chunk: first read starting at or after the chunk
    uint64_t chunk_begin;        // insert_kernel takes chunks [chunk_begin, nchunks)
    uint64_t nchunks;
    int K;
    int canonical;               // 0 forward strand, 1 lexicographic minimum, 2 smaller H_0
    int whole_file;              // windows run across read boundaries
    Geometry G;
    uint64_t *table;             // distinct-key set, cap slots of kw words
    uint64_t cap;
    SetTag set_tag;              // current generation of the set
    uint64_t *dlist;             // distinct keys in arrival order
    uint64_t dlist_cap;
    DevCounters *ctr;
    // partitioned update design (part != 0)
    int part;
    int coarse_shift;                      // coarse region = cell >> coarse_shift
    uint32_t *coarse;                      // kCoarseBins regions of coarse_cap codes
    uint64_t coarse_cap;
    unsigned long long *coarse_cursor;     // codes reserved per region
    unsigned long long *coarse_written;    // codes written per region (a prefix)
};

struct PartArgs {
    Geometry G;
    int coarse_shift;
    int slice_shift;                       // fine slice = cell >> slice_shift
    const uint32_t *coarse;
    uint64_t coarse_cap;
    const unsigned long long *coarse_written;
    void *fine;                            // one region of fine_cap codes per slice:
                                           // uint16 lane codes when lane_codes, else uint32
    uint64_t fine_cap;
    int lane_codes;                        // slice codes are counting-apply lanes
    unsigned long long *fine_cursor;
    unsigned long long *fine_written;
    DevCounters *ctr;
};

struct ApplyArgs {
    Geometry G;
    int slice_shift;                       // cells per slice = 2^slice_shift
    const void *codes;                     // one region of cap codes per slice:
                                           // uint16 lane codes when lane_codes, else uint32
    uint64_t cap;
    int lane_codes;
    const unsigned long long *written;     // codes per slice
    DevCounters *ctr;
};

cudaError_t launch_window_bound(const uint64_t *offsets, uint64_t nreads, int K,
                                DevCounters *ctr, cudaStream_t s);
cudaError_t launch_first_read(const uint64_t *offsets, uint64_t nreads, uint64_t first,
                              uint64_t nchunks, uint64_t chunk, uint32_t *first_read,
                              cudaStream_t s);
// chunk: the window starts per work unit the call was planned with (kChunk
// or kSmallChunk in the atomic design, kPartChunk in the partitioned one).
cudaError_t launch_insert(const InsertArgs &a, int grid, int chunk, cudaStream_t s);
// Resident insert blocks per SM; part: 0 atomic design, 1 partitioned with
// region bits inside the codes (coarse_shift <= 20), 2 partitioned (wide).
int insert_blocks_per_sm(int kw, int part);
cudaError_t launch_repartition(const PartArgs &p, cudaStream_t s);

// Batched insertion (atomic design): many samples, each with its own
// InsertArgs (device array), chunks of all samples in one index space with
// chunk_end[s] = chunks of samples 0..s.  Launches the batched first_read
// kernel and the persistent insert kernel.
constexpr int kBoundOutWords = 4;   // per-sample output of launch_window_bound_batch
int insert_batch_blocks_per_sm(int kw, int chunk);
cudaError_t launch_window_bound_batch(const uint64_t *const *offsets, const uint64_t *nreads,
                                      int n, int K, void *out, uint64_t max_reads, cudaStream_t s);
cudaError_t launch_insert_batch(const InsertArgs *args, const unsigned long long *chunk_end,
                                int nsamples, unsigned long long total_chunks, int kw, int chunk,
                                int grid, cudaStream_t s);
cudaError_t launch_apply(const ApplyArgs &p, uint64_t nslices, cudaStream_t s);
// Counting apply (alpha <= 15): the slice's increments are first counted in
// 32-bit shared-memory lanes (2^slice_shift * eta of them, at most
// kCountLanes), then added to the counters with saturation.
constexpr int kCountLanes = 16384;
cudaError_t launch_apply_count(const ApplyArgs &p, uint64_t nslices, cudaStream_t s);
// Insert n keys into a distinct set; when dlist is not null, keys new to the
// set are appended to it (ctr->distinct counts them).
cudaError_t launch_reinsert(const uint64_t *keys, uint64_t n, int kw, uint64_t *table,
                            uint64_t cap, SetTag tag, uint64_t *dlist, uint64_t dlist_cap,
                            DevCounters *ctr, uint32_t probe_limit, cudaStream_t s);

// Radix sort of n keys of kw words (1 or 2) on their low `bits` bits.  The
// sorted keys end in *result, which is one of in, alt0 or alt1; in is left
// unchanged when passes > 0.  counts needs sort_scratch_words(n, kw) uint32.
uint64_t sort_scratch_words(uint64_t n, int kw);
cudaError_t radix_sort(const uint64_t *in, uint64_t *alt0, uint64_t *alt1, uint64_t n, int kw,
                       int bits, uint32_t *counts, const uint64_t **result, cudaStream_t s);
// One stable pass of radix_sort on the 8-bit digit at bit `shift`.
cudaError_t radix_pass(const uint64_t *src, uint64_t *dst, uint64_t n, int kw, int shift,
                       uint32_t *counts, cudaStream_t s);

// Large key sets: after three radix_pass calls on the top kTopSortBits of
// the 2K key bits, top_segment_sort finishes the sort in place: the keys are
// cut into segments where their top bits change (b: seg_bounds_entries(n, kw)
// words) and each segment is sorted in shared memory.  Segments too large
// for it are written to big as (begin, count) pairs, their number to *nbig
// (at most seg_bounds_entries words of pairs); the caller radix-sorts them.
// Needs 2K >= kTopSortBits + 12.
constexpr int kTopSortBits = 24;
uint64_t seg_bounds_entries(uint64_t n, int kw);
// The big segments of top_segment_sort up to big_segment_max() keys, one
// block each, sorted in place (alt: scratch of the same layout as data).
cudaError_t big_segment_sort(uint64_t *data, uint64_t *alt, uint64_t n, int kw, int bits,
                             const unsigned long long *big, const unsigned long long *nbig,
                             cudaStream_t s);
uint64_t big_segment_max();
cudaError_t top_segment_sort(uint64_t *data, uint64_t n, int kw, int bits, unsigned long long *b,
                             unsigned long long *big, unsigned long long *nbig, cudaStream_t s);


// Bucket sort of one-word keys (classify): bucket_histogram counts
// key >> shift over kHistBins bins; the host merges adjacent bins into
// super-buckets of at most kBucketCap keys (map: bin -> super-bucket,
// start: first position of each super-bucket, nsuper + 1 entries);
// bucket_place_and_sort scatters in -> out by super-bucket and sorts every
// super-bucket of at most kBucketCap keys in shared memory.  Larger ones (a
// single bin) are left to the caller.  cursor needs nsuper words.
uint64_t bucket_hist_blocks(uint64_t n);   // partial histograms: this many x kHistBins u16
cudaError_t bucket_histogram(const uint64_t *keys, uint64_t n, int shift, unsigned short *partial,
                             unsigned *hist, cudaStream_t s);
// lo[b] / rsh[b]: lowest key value of super-bucket b and the shift that
// maps its key range onto kSubBins sub-bins.
cudaError_t bucket_place_and_sort(const uint64_t *in, uint64_t *out, uint64_t n, int shift,
                                  const unsigned *map, unsigned nsuper,
                                  const unsigned long long *start, const unsigned long long *lo,
                                  const int *rsh, unsigned long long *cursor, cudaStream_t s);

cudaError_t launch_query(const uint64_t *keys, uint64_t n, int kw, int K, Geometry G,
                         uint32_t *est, cudaStream_t s);
// Algorithm 5 only as far as the split on tau needs it (classify_query_kernel):
// est exact for keys above tau, at most tau otherwise.
cudaError_t launch_classify_query(const uint64_t *keys, uint64_t n, int kw, Geometry G,
                                  uint32_t tau, uint32_t *est, cudaStream_t s);
// est > tau split, stable: trusted keys to out[0, T), erroneous to out[T, n);
// T written to ctr->trusted.  scratch needs split_scratch_words(n) uint64.
uint64_t split_scratch_words(uint64_t n);
cudaError_t launch_split(const uint64_t *keys, const uint32_t *est, uint64_t n, int kw,
                         uint32_t tau, uint64_t *out, uint64_t *scratch, DevCounters *ctr,
                         cudaStream_t s);
cudaError_t launch_merge(uint64_t *dst, const uint64_t *src, Geometry G, cudaStream_t s);
// pos[i] = lower bound of probe i (kw words) in n sorted keys.
cudaError_t launch_lower_bound(const uint64_t *keys, uint64_t n, int kw, const uint64_t *probes,
                               uint64_t np, uint64_t *pos, cudaStream_t s);

cudaError_t launch_count_saturated(Geometry G, DevCounters *ctr, cudaStream_t s);

}  // namespace countbf

// Host side of the countBF C ABI (include/kmerco.h): argument validation,
// device memory, pointer-kind detection, capacity management of the
// distinct-key set, and the order of kernel launches for each phase.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/kmerco.h"
#include "kmerco_internal.cuh"

using namespace countbf;

constexpr int kCopyPieces = 8;   // pieces of a host input copied while earlier ones are inserted
// Host offsets of up to this many reads are checked and summed on the host
// (a few milliseconds at most), so the insert does not wait for the device;
// larger ones are copied and summed by a kernel, which the call waits for.
constexpr uint64_t kHostBoundReads = 1ull << 16;

// Distinct one-word keys above which classification takes the bucket sort
// (its histogram readback and host-side merge cost more than a full radix
// sort of a smaller set).
constexpr uint64_t kBucketSortMin = 1ull << 20;

// The handle's device counters and their pinned mirror hold a DevCounters
// followed by kmerco_digest's two sums.
constexpr size_t kCtrBytes = sizeof(DevCounters) + 2 * sizeof(unsigned long long);

struct kmerco {
    int K, kw, alpha, eta, nhash, canonical;   // canonical: 0 forward, 1 lexicographic, 2 hash
    int whole_file;
    uint32_t tau;
    int device;
    cudaStream_t stream;
    bool own_stream;
    int update_mode;         // 0 automatic, 1 atomic, 2 partitioned
    uint64_t pass_codes;     // increments staged per partitioned pass
    int grid_atomic, grid_part, grid_wide;   // insert grids: atomic, partitioned, wide partitioned
    uint64_t budget, used;
    uint64_t max_distinct;   // cap of the distinct list; 0: none
    kmerco_alloc_fn alloc_fn;   // caller's device allocator, or NULL for cudaMalloc
    kmerco_free_fn free_fn;
    void *alloc_ctx;
    Geometry G;
    DevCounters *ctr;        // device
    DevCounters *ctr_host;   // pinned, mapped mirror
    DevCounters *ctr_mirror; // the mirror's device address
    uint64_t *table;         // distinct-key set: cap slots of kw words
    uint64_t cap;
    uint32_t gen;            // generation tag of the set's current keys
    uint64_t *dlist;         // distinct keys in arrival order
    uint64_t dlist_cap;
    uint64_t d_ub;           // upper bound of the distinct keys held
    uint8_t *in_bases;       // staging of host inputs
    uint64_t in_bases_cap;
    uint64_t *in_offsets;
    uint64_t in_offsets_cap;
    uint32_t *first_read;
    uint64_t first_read_cap;
    uint64_t *alt0, *alt1;   // radix-sort buffers
    uint64_t alt0_cap, alt1_cap;
    uint32_t *est;
    uint64_t est_cap;
    uint64_t *split;         // trusted keys then erroneous keys
    uint64_t split_cap;
    uint32_t *sort_scratch;
    uint64_t sort_scratch_cap;
    uint64_t *split_scratch;
    uint64_t split_scratch_cap;
    uint64_t *q_keys;        // staging of kmerco_query
    uint32_t *q_est;
    uint64_t q_cap;
    const uint64_t *sorted;  // sorted distinct keys (one of dlist, alt0, alt1)
    uint64_t n_distinct, n_trusted;
    bool classified;
    bool est_exact;          // est holds Algorithm 5's value for every key, not only
                             // for the trustworthy ones
    cudaEvent_t ev[4];
    cudaStream_t copy_stream;                      // host input copies (created on first use)
    cudaEvent_t copy_ev[kCopyPieces + 1], copy_fork;
    bool insert_timed, classify_timed;
    uint64_t launches;       // kernels launched by this handle
    uint32_t *coarse;        // partitioned design: increment codes per coarse region
    uint64_t coarse_alloc;
    uint32_t *fine;          // ... and per slice
    uint64_t fine_alloc;
    unsigned long long *part_ctr;   // region cursors and written counts
    uint64_t part_ctr_alloc;
    unsigned long long *bucket_scratch;   // classify: bucket histogram, starts, cursors
    uint64_t bucket_scratch_cap;
    unsigned long long *bucket_host;      // pinned copy of the bucket starts
    unsigned short *hist_partial;         // per-block partial histograms
    uint64_t hist_partial_cap;
    unsigned long long *seg_scratch;      // classify of large key sets: segment bounds, big segments
    uint64_t seg_scratch_cap;
    cudaStream_t out_stream;              // result copies of kmerco_get_lists_async
    cudaEvent_t out_ready, out_done;      // lists written / copies finished
    bool out_pending;                     // copies queued since the last classify
};

namespace {

// NVTX range around one API call, so profilers show the phases by name.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

struct DeviceGuard {
    int prev = -1, want;
    explicit DeviceGuard(int d) : want(d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != want) cudaSetDevice(want);
    }
    ~DeviceGuard() {
        if (prev >= 0 && prev != want) cudaSetDevice(prev);
    }
};

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return KMERCO_OK;
    return e == cudaErrorMemoryAllocation ? KMERCO_ENOMEM : KMERCO_ECUDA;
}

#define KM_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)
#define KM_TRY(call)                     \
    do {                                 \
        int r_ = (call);                 \
        if (r_ != KMERCO_OK) return r_;  \
    } while (0)

// Device memory from the handle's allocator: the caller's callbacks when
// it gave them, else cudaMalloc / cudaFree.
int raw_alloc(const kmerco_t *h, void **p, uint64_t bytes) {
    *p = nullptr;
    if (h->alloc_fn) {
        void *q = h->alloc_fn(h->alloc_ctx, (size_t)bytes, (void *)h->stream);
        if (!q) return KMERCO_ENOMEM;
        if ((uintptr_t)q & 15) {   // vector loads need 16-byte alignment
            h->free_fn(h->alloc_ctx, q, (size_t)bytes, (void *)h->stream);
            return KMERCO_EINVAL;
        }
        *p = q;
        return KMERCO_OK;
    }
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return KMERCO_ENOMEM;
    }
    return KMERCO_OK;
}

void raw_free(const kmerco_t *h, void *p, uint64_t bytes) {
    if (!p) return;
    if (h->free_fn) {
        // the block goes back to the caller's pool, which may hand it out
        // at once: the work that used it must have finished
        cudaStreamSynchronize(h->stream);
        if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
        if (h->out_stream) cudaStreamSynchronize(h->out_stream);
        h->free_fn(h->alloc_ctx, p, (size_t)bytes, (void *)h->stream);
        return;
    }
    cudaFree(p);
}

int dev_alloc(kmerco_t *h, void **p, uint64_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (h->budget && h->used + bytes > h->budget) return KMERCO_ENOMEM;
    KM_TRY(raw_alloc(h, p, bytes));
    h->used += bytes;
    return KMERCO_OK;
}

void dev_free(kmerco_t *h, void *p, uint64_t bytes) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    raw_free(h, p, bytes);
    h->used -= bytes;
}

// Make *p hold at least `need` elements of `elem` bytes (contents dropped).
template <typename T>
int ensure(kmerco_t *h, T **p, uint64_t *cap, uint64_t need, uint64_t elem = sizeof(T)) {
    if (*p && *cap >= need) return KMERCO_OK;
    uint64_t want = need + need / 4 + 64;
    dev_free(h, *p, *cap * elem);
    *p = nullptr;
    *cap = 0;
    void *q;
    KM_TRY(dev_alloc(h, &q, want * elem));
    *p = (T *)q;
    *cap = want;
    return KMERCO_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The counters are written into the mapped pinned mirror by a kernel, not
// copied by a copy engine: a device-to-host copy would queue behind any
// large copy in flight in that direction (the lists of the previous sample
// that kmerco_get_lists_async is still moving), and every readback of the
// next insert would wait for it.
__global__ void mirror_counters_kernel(const unsigned long long *src, unsigned long long *dst) {
    const unsigned i = threadIdx.x;
    if (i < kCtrBytes / 8) dst[i] = src[i];
}
static_assert(sizeof(DevCounters) % 8 == 0, "the mirror is copied in 8-byte words");

// kmerco_digest's two sums, after the DevCounters.
unsigned long long *digest_sums(const kmerco_t *h) {
    return (unsigned long long *)((char *)h->ctr + sizeof(DevCounters));
}

// kmerco_digest: the two sums of mixed (index, cell) values, summed per warp
// and added to the handle's counters (wrapping, so the order does not matter).
__global__ void digest_kernel(const uint64_t *cells, uint64_t words, unsigned long long *acc) {
    uint64_t s0 = 0, s1 = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t c = cells[i];
        s0 += fmix64(c ^ (i * 0x9E3779B97F4A7C15ull));
        s1 += fmix64(c + fmix64(i + 1));
    }
    for (int o = 16; o; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, (unsigned long long)s0);
        atomicAdd(acc + 1, (unsigned long long)s1);
    }
}

int read_counters(kmerco_t *h) {
    mirror_counters_kernel<<<1, 32, 0, h->stream>>>((const unsigned long long *)h->ctr,
                                                    (unsigned long long *)h->ctr_mirror);
    KM_CUDA(cudaGetLastError());
    h->launches += 1;
    KM_CUDA(cudaStreamSynchronize(h->stream));
    return KMERCO_OK;
}

// Generation tag of the handle's distinct set: the spare bits above the key
// in a slot's top word (2K key bits; two-word keys keep 2K - 64 of them in
// the top word).  Fewer than two spare bits: no tag, free slots are all ones.
SetTag set_tag(const kmerco_t *h) {
    const int used = h->kw == 1 ? 2 * h->K : 2 * h->K - 64;
    const int spare = 64 - used;
    if (spare < 2) return SetTag{0, 0};
    return SetTag{(uint64_t)h->gen << used, (~0ull >> used) << used};
}

// Generations the tag can tell apart (the all-ones tag is left to cleared
// slots), or 0 without a tag.
uint32_t tag_count(const kmerco_t *h) {
    const int spare = 64 - (h->kw == 1 ? 2 * h->K : 2 * h->K - 64);
    if (spare < 2) return 0;
    return spare >= 32 ? 0xFFFFFFFFu : (1u << spare) - 1;
}

int device_error_status(unsigned err) {
    if (err & kErrListFull) return KMERCO_ENOMEM;
    if (err & (kErrCasLimit | kErrProbeLimit)) return KMERCO_ETIMEOUT;
    return KMERCO_OK;
}

// The distinct-key set must keep its load factor at or below 1/2 for every
// key the next launch could add: cap >= 2 * (distinct so far + new windows).
int ensure_set_capacity(kmerco_t *h, uint64_t add) {
    uint64_t need = h->d_ub + add;
    if (need <= h->dlist_cap && 2 * need <= h->cap) {
        h->d_ub = need;
        return KMERCO_OK;
    }
    uint64_t D = 0;   // nothing inserted since create or reset: no keys to read back
    if (h->d_ub) {
        KM_TRY(read_counters(h));
        D = h->ctr_host->distinct;
    }
    need = D + add;
    // with a cap on the distinct list, keys beyond it are dropped on the
    // device (the list-full error) instead of growing the list
    const uint64_t list_need = h->max_distinct && need > h->max_distinct ? h->max_distinct : need;
    if (list_need > h->dlist_cap) {
        uint64_t want = list_need > h->dlist_cap + h->dlist_cap / 2 ? list_need
                                                                    : h->dlist_cap + h->dlist_cap / 2;
        if (h->max_distinct && want > h->max_distinct) want = h->max_distinct;
        void *q;
        KM_TRY(dev_alloc(h, &q, want * h->kw * 8));
        if (D) KM_CUDA(cudaMemcpyAsync(q, h->dlist, (D < h->dlist_cap ? D : h->dlist_cap) * h->kw * 8,
                                       cudaMemcpyDeviceToDevice, h->stream));
        KM_CUDA(cudaStreamSynchronize(h->stream));
        dev_free(h, h->dlist, h->dlist_cap * h->kw * 8);
        h->dlist = (uint64_t *)q;
        h->dlist_cap = want;
    }
    if (2 * need > h->cap) {
        uint64_t want = 2 * need;
        if (want < h->cap + h->cap / 2) want = h->cap + h->cap / 2;
        if (want < 1024) want = 1024;
        void *q;
        KM_TRY(dev_alloc(h, &q, want * h->kw * 8));
        KM_CUDA(cudaMemsetAsync(q, 0xFF, want * h->kw * 8, h->stream));
        KM_CUDA(launch_reinsert(h->dlist, D < h->dlist_cap ? D : h->dlist_cap, h->kw,
                                (uint64_t *)q, want, set_tag(h), nullptr, 0, h->ctr,
                                h->G.probe_limit, h->stream));
        h->launches += D ? 1 : 0;
        KM_CUDA(cudaStreamSynchronize(h->stream));
        dev_free(h, h->table, h->cap * h->kw * 8);
        h->table = (uint64_t *)q;
        h->cap = want;
    }
    h->d_ub = need;
    return KMERCO_OK;
}

int validate(const kmerco_config_t *c) {
    if (!c) return KMERCO_EINVAL;
    if (c->k < 1 || c->k > 64) return KMERCO_EINVAL;
    if (c->counter_bits < 1 || c->counter_bits > 32) return KMERCO_EINVAL;
    if (c->nhash < 1 || c->nhash > 32) return KMERCO_EINVAL;
    if (c->dim_x || c->dim_y) {
        // two-dimensional countBF: m is implied by the dimensions
        if (c->dim_x < 1 || c->dim_y < 1 || c->dim_x > (1ull << 24) || c->dim_y > (1ull << 24))
            return KMERCO_EINVAL;
    } else if (c->m < 1 || c->m > (1ull << 48)) {
        return KMERCO_EINVAL;
    }
    const uint64_t maxc = (1ull << c->counter_bits) - 1;
    if ((uint64_t)c->threshold >= maxc) return KMERCO_EINVAL;
    if (c->forward_only != 0 && c->forward_only != 1) return KMERCO_EINVAL;
    if (c->canonical_hash != 0 && (c->canonical_hash != 1 || c->forward_only)) return KMERCO_EINVAL;
    if (c->whole_file != 0 && c->whole_file != 1) return KMERCO_EINVAL;
    if (c->update_mode < 0 || c->update_mode > 2) return KMERCO_EINVAL;
    if (c->pass_codes > kMaxBatchCodes) return KMERCO_EINVAL;
    if ((c->dev_alloc == nullptr) != (c->dev_free == nullptr)) return KMERCO_EINVAL;
    if (c->update_mode == 2) {
        const uint64_t eta = 64 / (uint64_t)c->counter_bits;
        const uint64_t words = c->dim_x ? c->dim_x * c->dim_y : (c->m + eta - 1) / eta;
        if (c->nhash > kPartMaxHash || words > (1ull << (kMaxCoarseShift + 6)))
            return KMERCO_EINVAL;
    }
    return KMERCO_OK;
}

// Whether this handle applies counter increments with the partitioned design.
bool use_partitioned(const kmerco_t *h) {
    if (h->update_mode == 1) return false;
    const bool able = h->nhash <= kPartMaxHash && h->G.words <= (1ull << (kMaxCoarseShift + 6));
    if (h->update_mode == 2) return able;
    return able && h->G.words >= (1ull << 17);   // smaller countBFs stay L2-resident
}

// Trial division; n is at most about 2^24 here.
bool is_prime(uint64_t n) {
    if (n < 2) return false;
    for (uint64_t d = 2; d * d <= n; ++d)
        if (n % d == 0) return false;
    return true;
}

// Pinned host mirror of the classification scratch, sized for the largest
// user (the bucket sort's histogram, map, starts, bounds and shifts).
constexpr uint64_t kBucketHostWords = 4 * (uint64_t)kHistBins + 1 + kHistBins / 2;

int ensure_bucket_host(kmerco_t *h) {
    if (h->bucket_host) return KMERCO_OK;
    if (cudaMallocHost((void **)&h->bucket_host, kBucketHostWords * 8) != cudaSuccess) {
        h->bucket_host = nullptr;
        return KMERCO_ENOMEM;
    }
    return KMERCO_OK;
}

// Smallest l with 2^l >= x (64 for x above 2^63).
int ceil_log2(uint64_t x) {
    int l = 0;
    while (l < 64 && (1ull << l) < x) ++l;
    return l;
}

// Classification sorts a distinct-key set this large by its top bits and
// then by segments in shared memory (top_segment_sort) rather than by a full
// radix sort or the bucket sort.
bool use_top_sort(uint64_t D, int kw, int bits) {
    if (bits < kTopSortBits + 12) return false;
    if (kw == 2) return D > (1ull << 21);
    return D > (uint64_t)kHistBins * (kBucketCap / 4);
}

// ------------------------------------------------------------ insert plan

// How one insert call applies its counter increments (partitioned design),
// decided on the host from the call's window bound and input size.
struct PartPlan {
    bool part = false, repart = false, count = false;
    int coarse_shift = 0, slice_shift = 0;
    uint64_t coarse_cap = 0, fine_cap = 0, nslices = 0, passes = 1;
    uint64_t coarse_words() const { return kCoarseBins * coarse_cap; }   // uint32 codes
    // slice codes: uint16 counting lanes (two per 32-bit word) or uint32 codes
    bool lane_codes() const { return repart && count; }
    uint64_t fine_words() const {
        return !repart ? 0 : lane_codes() ? (nslices * fine_cap + 1) / 2 : nslices * fine_cap;
    }
    uint64_t ctr_words() const { return 2 * kCoarseBins + 2 * nslices; }
};

struct PartBufs {
    uint32_t *coarse, *fine;
    unsigned long long *ctr;
};

// Increment-code buffers sized for one pass of at most pass_codes
// increments; larger inputs run in several passes over consecutive chunk
// ranges.  Counting apply for alpha <= 15 (slices of kCountLanes / eta cells,
// rounded down to a power of two), compare-and-swap apply otherwise or when
// the slices would be too many for one coarse region.
PartPlan plan_partition(const kmerco_t *h, uint64_t bound, uint64_t nbytes) {
    PartPlan pp;
    if (!use_partitioned(h) || bound == 0) return pp;
    pp.part = true;
    const uint64_t W = h->G.words, U = bound * (uint64_t)h->nhash;
    const uint64_t part_chunks = (nbytes + kPartChunk - 1) / kPartChunk;
    pp.passes = (U + h->pass_codes - 1) / h->pass_codes;
    if (pp.passes > part_chunks) pp.passes = part_chunks;   // a pass takes one chunk at least
    if (pp.passes < 1) pp.passes = 1;
    const uint64_t Up = (U + pp.passes - 1) / pp.passes;   // increments per pass, on average
    pp.coarse_shift = ceil_log2(W) - 6;
    if (pp.coarse_shift < 0) pp.coarse_shift = 0;
    int count_shift = 0;
    while ((2ull << count_shift) * (uint64_t)h->eta <= (uint64_t)kCountLanes) ++count_shift;
    pp.count = h->alpha <= 15 && pp.coarse_shift - count_shift <= kMaxCoarseShift - kSliceShift;
    pp.slice_shift = pp.count ? count_shift : kSliceShift;
    pp.repart = pp.coarse_shift > pp.slice_shift;
    if (!pp.repart) pp.slice_shift = pp.coarse_shift;
    pp.nslices = (W + (1ull << pp.slice_shift) - 1) >> pp.slice_shift;
    pp.coarse_cap = Up / kCoarseBins;
    pp.coarse_cap = (pp.coarse_cap + pp.coarse_cap / 6 + 4096 + 3) & ~3ull;   // multiple of 4
    pp.fine_cap = pp.repart ? Up / pp.nslices : 0;
    pp.fine_cap = (pp.fine_cap + pp.fine_cap / 5 + 1024 + 7) & ~7ull;   // multiple of 8
    return pp;
}

// Insert arguments of one call that do not depend on the plan.
InsertArgs sample_args(const kmerco_t *h, const uint8_t *d_bases, const uint64_t *d_off,
                       uint64_t nreads, uint64_t first, uint64_t last) {
    InsertArgs a;
    memset(&a, 0, sizeof(a));
    a.bases = d_bases;
    a.offsets = d_off;
    a.nreads = nreads;
    a.first = first;
    a.last = last;
    a.first_read = h->first_read;
    a.K = h->K;
    a.canonical = h->canonical;
    a.whole_file = h->whole_file;
    a.G = h->G;
    a.table = h->table;
    a.cap = h->cap;
    a.set_tag = set_tag(h);
    a.dlist = h->dlist;
    a.dlist_cap = h->dlist_cap;
    a.ctr = h->ctr;
    return a;
}

// A host input copied to the device on its own stream in npieces equal byte
// pieces, each with an event; an insert launch waits only for the pieces
// holding its bytes (its chunks and the K - 1 bytes after them).
struct HostCopy {
    uint64_t nbytes;
    int npieces;
    cudaEvent_t *ev;             // one per piece
    uint64_t piece_lo(int i) const { return nbytes * (uint64_t)i / (uint64_t)npieces; }
};

// Issue the copy of nbytes host bytes src -> dst in pieces on the handle's
// copy stream, after the work already queued on the handle's stream (the
// previous call may still read dst).
int issue_host_copy(kmerco_t *h, const uint8_t *src, uint8_t *dst, uint64_t nbytes,
                    HostCopy &hc) {
    if (!h->copy_stream) {
        bool ok = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&h->copy_fork, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; ok && i <= kCopyPieces; ++i)
            ok = cudaEventCreateWithFlags(&h->copy_ev[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) return KMERCO_ECUDA;
    }
    hc.nbytes = nbytes;
    hc.npieces = nbytes >= (8ull << 20) ? kCopyPieces : 1;
    hc.ev = h->copy_ev;
    KM_CUDA(cudaEventRecord(h->copy_fork, h->stream));
    KM_CUDA(cudaStreamWaitEvent(h->copy_stream, h->copy_fork, 0));
    for (int i = 0; i < hc.npieces; ++i) {
        const uint64_t lo = hc.piece_lo(i), hi = hc.piece_lo(i + 1);
        if (hi > lo)
            KM_CUDA(cudaMemcpyAsync(dst + lo, src + lo, hi - lo, cudaMemcpyHostToDevice,
                                    h->copy_stream));
        KM_CUDA(cudaEventRecord(h->copy_ev[i], h->copy_stream));
    }
    return KMERCO_OK;
}

// Window starts per work unit of an insert call: the partitioned design's
// chunk, else kChunk, or kSmallChunk when the call's chunks of kChunk would
// not give every resident block of the GPU one (small inputs).
uint64_t insert_chunk(const kmerco_t *h, const PartPlan &pp, uint64_t nbytes) {
    if (pp.part) return kPartChunk;
    return (nbytes + kChunk - 1) / kChunk < (uint64_t)h->grid_atomic ? kSmallChunk : kChunk;
}

// All device work of one insert call on stream s, without host
// synchronisation (so it can be captured): first reads of the chunks, then
// per pass the insert kernel and, in the partitioned design, repartition and
// apply.  h->first_read must hold the call's chunks; pb holds pp's buffers.
// With hc (a host input being copied), each pass is split into up to
// kCopyPieces launches, each waiting only for the pieces it reads.
int launch_sample_insert(const kmerco_t *h, InsertArgs a, const PartPlan &pp,
                         const PartBufs &pb, cudaStream_t s, uint64_t &launches,
                         const HostCopy *hc = nullptr) {
    const uint64_t nbytes = a.last - a.first;
    const uint64_t chunk = insert_chunk(h, pp, nbytes);
    const uint64_t nchunks = (nbytes + chunk - 1) / chunk;
    // chunk ranges of the insert launches: per pass, pieces when copying
    const uint64_t q = hc && pp.passes <= (uint64_t)kCopyPieces
                           ? std::max<uint64_t>(1, kCopyPieces / pp.passes) : 1;
    std::vector<uint64_t> cut;   // launch r takes chunks [cut[r], cut[r + 1])
    for (uint64_t pass = 0; pass < pp.passes; ++pass) {
        const uint64_t cb = nchunks * pass / pp.passes, ce = nchunks * (pass + 1) / pp.passes;
        const uint64_t qq = std::min<uint64_t>(q, std::max<uint64_t>(1, ce - cb));
        for (uint64_t j = 0; j < qq; ++j) cut.push_back(cb + (ce - cb) * j / qq);
    }
    cut.push_back(nchunks);
    const uint64_t nr = cut.size() - 1;
    KM_CUDA(launch_first_read(a.offsets, a.nreads, a.first, nchunks, chunk, h->first_read, s));
    launches += nchunks ? 1 : 0;
    a.part = pp.part ? 1 : 0;
    a.coarse_shift = pp.coarse_shift;
    a.coarse = pb.coarse;
    a.coarse_cap = pp.coarse_cap;
    a.coarse_cursor = pb.ctr;
    a.coarse_written = pb.ctr ? pb.ctr + kCoarseBins : nullptr;
    const int grid = !pp.part ? h->grid_atomic : pp.coarse_shift <= 20 ? h->grid_part
                                                                       : h->grid_wide;
    uint64_t r = 0;   // next launch range
    for (uint64_t pass = 0; pass < pp.passes; ++pass) {
        const uint64_t pass_end = nchunks * (pass + 1) / pp.passes;
        if (pp.part) KM_CUDA(cudaMemsetAsync(pb.ctr, 0, pp.ctr_words() * 8, s));
        for (; r < nr && cut[r + 1] <= pass_end && cut[r] < pass_end; ++r) {
            if (hc) {   // the pieces holding this range's bytes and the K - 1 after it
                const uint64_t lo = cut[r] * chunk;
                const uint64_t hi = std::min(cut[r + 1] * chunk + (uint64_t)a.K - 1, nbytes);
                for (int i = 0; i < hc->npieces; ++i)
                    if (hc->piece_lo(i) < hi && hc->piece_lo(i + 1) > lo)
                        KM_CUDA(cudaStreamWaitEvent(s, hc->ev[i], 0));
            }
            a.chunk_begin = cut[r];
            a.nchunks = cut[r + 1];
            KM_CUDA(launch_insert(a, grid, (int)chunk, s));
            launches += a.nchunks > a.chunk_begin ? 1 : 0;
        }
        if (!pp.part) continue;
        unsigned long long *fine_cursor = pb.ctr + 2 * kCoarseBins;
        unsigned long long *fine_written = fine_cursor + pp.nslices;
        if (pp.repart) {
            PartArgs p;
            p.G = h->G;
            p.coarse_shift = pp.coarse_shift;
            p.slice_shift = pp.slice_shift;
            p.coarse = pb.coarse;
            p.coarse_cap = pp.coarse_cap;
            p.coarse_written = a.coarse_written;
            p.fine = pb.fine;
            p.fine_cap = pp.fine_cap;
            p.lane_codes = pp.lane_codes() ? 1 : 0;
            p.fine_cursor = fine_cursor;
            p.fine_written = fine_written;
            p.ctr = h->ctr;
            KM_CUDA(launch_repartition(p, s));
            launches += 1;
        }
        ApplyArgs ap;
        ap.G = h->G;
        ap.slice_shift = pp.slice_shift;
        ap.codes = pp.repart ? pb.fine : pb.coarse;
        ap.cap = pp.repart ? pp.fine_cap : pp.coarse_cap;
        ap.lane_codes = pp.lane_codes() ? 1 : 0;
        ap.written = pp.repart ? fine_written : a.coarse_written;
        ap.ctr = h->ctr;
        KM_CUDA(pp.count ? launch_apply_count(ap, pp.nslices, s) : launch_apply(ap, pp.nslices, s));
        launches += 1;
    }
    return KMERCO_OK;
}

}  // namespace

extern "C" {

const char *kmerco_strerror(int status) {
    switch (status) {
    case KMERCO_OK: return "ok";
    case KMERCO_EINVAL: return "invalid argument";
    case KMERCO_ENOMEM: return "out of device memory or over the HBM budget";
    case KMERCO_ECUDA: return "CUDA error";
    case KMERCO_ETIMEOUT: return "a bounded device retry loop gave up";
    case KMERCO_ESTATE: return "call not valid in the current state";
    case KMERCO_ESIZE: return "buffer too small";
    default: return "unknown status";
    }
}

int kmerco_paper_dims(uint64_t n, double fpp, uint64_t *dim_x, uint64_t *dim_y) {
    if (!dim_x || !dim_y || n < 1 || !(fpp > 0.0 && fpp < 1.0)) return KMERCO_EINVAL;
    const double ln2 = log(2.0);
    const double m = -(double)n * log(fpp) / (ln2 * ln2);   // standard Bloom filter size
    const double v = sqrt(m / 128.0);
    if (!(v < (double)(1ull << 24))) return KMERCO_EINVAL;
    uint64_t x = (uint64_t)floor(v) + 1;                     // first integer above v
    while (!is_prime(x)) ++x;
    uint64_t y = x;
    for (int found = 0; found < 3;)                          // third prime after x
        if (is_prime(++y)) ++found;
    *dim_x = x;
    *dim_y = y;
    return KMERCO_OK;
}

int kmerco_estimate_bytes(const kmerco_config_t *cfg, uint64_t nreads, uint64_t nbytes,
                          uint64_t windows, int host_inputs, uint64_t *bytes) {
    if (!bytes) return KMERCO_EINVAL;
    KM_TRY(validate(cfg));
    if (cfg->dev_alloc) return KMERCO_EINVAL;   // plain sizes only; no handle is made
    // a handle's sizing state without any device object
    kmerco_t t;
    memset(&t, 0, sizeof(t));
    t.K = cfg->k;
    t.kw = cfg->k <= 32 ? 1 : 2;
    t.alpha = cfg->counter_bits;
    t.eta = 64 / cfg->counter_bits;
    t.nhash = cfg->nhash;
    t.update_mode = cfg->update_mode;
    t.pass_codes = cfg->pass_codes ? cfg->pass_codes : kMaxBatchCodes;
    t.G = make_geometry((cfg->m + (uint64_t)t.eta - 1) / (uint64_t)t.eta, cfg->dim_x, cfg->dim_y,
                        t.alpha, t.nhash);
    const uint64_t kw = (uint64_t)t.kw;
    // ensure(): need + need / 4 + 64 elements
    auto grown = [](uint64_t need, uint64_t elem) { return (need + need / 4 + 64) * elem; };
    uint64_t b = t.G.words * 8 + kCtrBytes;
    if (host_inputs) b += grown(nbytes, 1) + grown(nreads + 1, 8);
    if (windows) {
        // distinct list and set for every window being a new key
        uint64_t list = windows;
        if (cfg->max_distinct && list > cfg->max_distinct) list = cfg->max_distinct;
        b += list * kw * 8 + std::max<uint64_t>(2 * windows, 1024) * kw * 8;
        const PartPlan pp = plan_partition(&t, windows, nbytes);
        if (pp.part) {
            b += grown(pp.coarse_words(), 4) + grown(pp.ctr_words(), 8);
            if (pp.repart) b += grown(pp.fine_words(), 4);
        }
        const uint64_t chunk = pp.part ? kPartChunk : kSmallChunk;   // the most chunks
        b += grown((nbytes + chunk - 1) / chunk, 4);
        // classification of at most `windows` distinct keys
        const uint64_t D = windows;
        b += 2 * grown(D * kw, 8) + grown(D, 4) + grown(D * kw, 8) +
             grown(sort_scratch_words(D, kw), 4) + grown(split_scratch_words(D), 8);
        if (use_top_sort(D, t.kw, 2 * t.K)) b += grown(3 * seg_bounds_entries(D, t.kw) + 1, 8);
        if (kw == 1 && 2 * t.K >= kHistBits + 8 && D > kBucketSortMin)   // the bucket sort may run
            b += grown(kBucketHostWords + kHistBins, 8) +
                 grown(bucket_hist_blocks(D) * kHistBins, 2);
    }
    *bytes = b;
    return KMERCO_OK;
}

int kmerco_create(int k, uint64_t m, int counter_bits, int nhash, uint32_t threshold,
                  kmerco_t **out) {
    kmerco_config_t c;
    memset(&c, 0, sizeof(c));
    c.k = k;
    c.m = m;
    c.counter_bits = counter_bits;
    c.nhash = nhash;
    c.threshold = threshold;
    c.device = -1;
    return kmerco_create_ex(&c, out);
}

int kmerco_create_ex(const kmerco_config_t *cfg, kmerco_t **out) {
    if (!out) return KMERCO_EINVAL;
    *out = nullptr;
    KM_TRY(validate(cfg));
    kmerco_t *h = new (std::nothrow) kmerco_t;
    if (!h) return KMERCO_ENOMEM;
    memset(h, 0, sizeof(*h));
    h->K = cfg->k;
    h->kw = cfg->k <= 32 ? 1 : 2;
    h->alpha = cfg->counter_bits;
    h->eta = 64 / cfg->counter_bits;
    h->nhash = cfg->nhash;
    h->tau = cfg->threshold;
    h->canonical = cfg->forward_only ? 0 : cfg->canonical_hash ? 2 : 1;
    h->whole_file = cfg->whole_file;
    h->budget = cfg->hbm_budget;
    h->max_distinct = cfg->max_distinct;
    h->alloc_fn = cfg->dev_alloc;
    h->free_fn = cfg->dev_free;
    h->alloc_ctx = cfg->alloc_ctx;
    if (cfg->device >= 0) {
        h->device = cfg->device;
    } else if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return KMERCO_ECUDA;
    }
    DeviceGuard guard(h->device);
    int status = KMERCO_OK;
    do {
        if (cfg->stream) {
            h->stream = (cudaStream_t)cfg->stream;
        } else {
            if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
                status = KMERCO_ECUDA;
                break;
            }
            h->own_stream = true;
        }
        for (int i = 0; i < 4; ++i)
            if (cudaEventCreate(&h->ev[i]) != cudaSuccess) status = KMERCO_ECUDA;
        if (status) break;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        if (sms <= 0) sms = 1;
        h->update_mode = cfg->update_mode;
        h->pass_codes = cfg->pass_codes ? cfg->pass_codes : kMaxBatchCodes;
        h->grid_atomic = sms * insert_blocks_per_sm(h->kw, 0);
        h->grid_part = sms * insert_blocks_per_sm(h->kw, 1);
        h->grid_wide = sms * insert_blocks_per_sm(h->kw, 2);

        const uint64_t eta = (uint64_t)h->eta;
        h->G = make_geometry((cfg->m + eta - 1) / eta, cfg->dim_x, cfg->dim_y, h->alpha,
                             h->nhash);
        if (cfg->retry_limit) h->G.cas_limit = h->G.probe_limit = cfg->retry_limit;
        Geometry &G = h->G;
        void *p;
        if ((status = dev_alloc(h, &p, G.words * 8))) break;
        G.cells = (uint64_t *)p;
        if ((status = dev_alloc(h, &p, kCtrBytes))) break;
        h->ctr = (DevCounters *)p;
        if (cudaHostAlloc((void **)&h->ctr_host, kCtrBytes, cudaHostAllocMapped) !=
            cudaSuccess) {
            cudaGetLastError();
            h->ctr_host = nullptr;
            status = KMERCO_ENOMEM;
            break;
        }
        if (cudaHostGetDevicePointer((void **)&h->ctr_mirror, h->ctr_host, 0) != cudaSuccess) {
            cudaGetLastError();
            status = KMERCO_ECUDA;
            break;
        }
        memset(h->ctr_host, 0, kCtrBytes);
        if (cudaMemsetAsync(G.cells, 0, G.words * 8, h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->ctr, 0, sizeof(DevCounters), h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess) {
            status = KMERCO_ECUDA;
            break;
        }
    } while (0);
    if (status) {
        cudaGetLastError();
        kmerco_destroy(h);
        return status;
    }
    *out = h;
    return KMERCO_OK;
}

void kmerco_destroy(kmerco_t *h) {
    if (!h) return;
    {
        DeviceGuard guard(h->device);
        if (h->stream) cudaStreamSynchronize(h->stream);
        if (h->out_stream) cudaStreamSynchronize(h->out_stream);
        dev_free(h, h->G.cells, h->G.words * 8);
        dev_free(h, h->ctr, kCtrBytes);
        dev_free(h, h->table, h->cap * h->kw * 8);
        dev_free(h, h->dlist, h->dlist_cap * h->kw * 8);
        dev_free(h, h->in_bases, h->in_bases_cap);
        dev_free(h, h->in_offsets, h->in_offsets_cap * 8);
        dev_free(h, h->first_read, h->first_read_cap * 4);
        dev_free(h, h->alt0, h->alt0_cap * 8);
        dev_free(h, h->alt1, h->alt1_cap * 8);
        dev_free(h, h->est, h->est_cap * 4);
        dev_free(h, h->split, h->split_cap * 8);
        dev_free(h, h->sort_scratch, h->sort_scratch_cap * 4);
        dev_free(h, h->split_scratch, h->split_scratch_cap * 8);
        dev_free(h, h->q_keys, h->q_cap * 16);
        dev_free(h, h->q_est, h->q_cap * 4);
        dev_free(h, h->coarse, h->coarse_alloc * 4);
        dev_free(h, h->fine, h->fine_alloc * 4);
        dev_free(h, h->part_ctr, h->part_ctr_alloc * 8);
        dev_free(h, h->bucket_scratch, h->bucket_scratch_cap * 8);
        dev_free(h, h->hist_partial, h->hist_partial_cap * 2);
        dev_free(h, h->seg_scratch, h->seg_scratch_cap * 8);
        if (h->bucket_host) cudaFreeHost(h->bucket_host);
        if (h->ctr_host) cudaFreeHost(h->ctr_host);
        for (int i = 0; i < 4; ++i)
            if (h->ev[i]) cudaEventDestroy(h->ev[i]);
        for (int i = 0; i <= kCopyPieces; ++i)
            if (h->copy_ev[i]) cudaEventDestroy(h->copy_ev[i]);
        if (h->copy_fork) cudaEventDestroy(h->copy_fork);
        if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
        if (h->out_ready) cudaEventDestroy(h->out_ready);
        if (h->out_done) cudaEventDestroy(h->out_done);
        if (h->out_stream) cudaStreamDestroy(h->out_stream);
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        cudaGetLastError();
    }
    delete h;
}

int kmerco_reset(kmerco_t *h) {
    if (!h) return KMERCO_EINVAL;
    DeviceGuard guard(h->device);
    KM_CUDA(cudaMemsetAsync(h->G.cells, 0, h->G.words * 8, h->stream));
    if (h->table && h->d_ub) {
        // the next generation tag makes every held key read as a free slot;
        // once the tags run out the table is cleared and they start again
        if (h->gen + 1 < tag_count(h)) {
            ++h->gen;
        } else {
            KM_CUDA(cudaMemsetAsync(h->table, 0xFF, h->cap * h->kw * 8, h->stream));
            h->gen = 0;
        }
    }
    KM_CUDA(cudaMemsetAsync(h->ctr, 0, sizeof(DevCounters), h->stream));
    h->d_ub = 0;
    h->classified = false;
    h->n_distinct = h->n_trusted = 0;
    h->insert_timed = h->classify_timed = false;
    return KMERCO_OK;
}

int kmerco_insert(kmerco_t *h, const char *bases, const uint64_t *offsets, uint64_t nreads) {
    Range range("kmerco_insert");
    if (!h) return KMERCO_EINVAL;
    if (nreads == 0) return KMERCO_OK;
    if (!offsets || nreads >= 0xFFFFFFFFull) return KMERCO_EINVAL;
    DeviceGuard guard(h->device);
    const int K = h->K;
    uint64_t first, last, bound = 0;
    const uint64_t *d_off = offsets;
    const bool host_offsets = !is_device_ptr(offsets);
    const bool host_bases = bases && !is_device_ptr(bases);
    HostCopy hc;
    bool copying = false;
    if (host_offsets) {   // checked and summed on the device too
        // the offsets go first: a check that waits for them then does not wait
        // for the reads' bytes queued behind them on the copy engine
        KM_TRY(ensure(h, &h->in_offsets, &h->in_offsets_cap, nreads + 1));
        KM_CUDA(cudaMemcpyAsync(h->in_offsets, offsets, (nreads + 1) * 8, cudaMemcpyHostToDevice,
                                h->stream));
        d_off = h->in_offsets;
        if (host_bases && offsets[nreads] > offsets[0]) {
            // the reads' bytes start moving now, while the offsets are checked;
            // the insert launches wait only for the pieces they read
            const uint64_t nb = offsets[nreads] - offsets[0];
            KM_TRY(ensure(h, &h->in_bases, &h->in_bases_cap, nb));
            KM_TRY(issue_host_copy(h, (const uint8_t *)bases + offsets[0], h->in_bases, nb, hc));
            copying = true;
        }
    }
    if (host_offsets && nreads <= kHostBoundReads) {
        // summed on the host: the call does not wait for the device
        first = offsets[0];
        last = offsets[nreads];
        for (uint64_t r = 0; r < nreads; ++r) {
            const uint64_t s = offsets[r], e = offsets[r + 1];
            if (e < s) return KMERCO_EINVAL;
            if (e - s >= (uint64_t)K) bound += e - s - K + 1;
        }
    } else {
        KM_CUDA(cudaMemsetAsync(&h->ctr->bound, 0, sizeof(h->ctr->bound), h->stream));
        KM_CUDA(cudaMemsetAsync(&h->ctr->bad_offsets, 0, sizeof(h->ctr->bad_offsets), h->stream));
        KM_CUDA(launch_window_bound(d_off, nreads, K, h->ctr, h->stream));
        h->launches += 1;
        KM_TRY(read_counters(h));
        if (h->ctr_host->bad_offsets) return KMERCO_EINVAL;
        first = h->ctr_host->first;
        last = h->ctr_host->last;
        bound = h->ctr_host->bound;
    }
    if (h->whole_file)   // the reads are one sequence of last - first bases
        bound = last - first >= (uint64_t)K ? last - first - K + 1 : 0;
    const uint64_t nbytes = last - first;
    if (nbytes && !bases) return KMERCO_EINVAL;
    const uint8_t *d_bases = nullptr;
    if (nbytes) {
        if (!host_bases) {
            d_bases = (const uint8_t *)bases + first;
        } else {   // copied piece by piece on the copy stream (issued above when it could be)
            if (!copying) {
                KM_TRY(ensure(h, &h->in_bases, &h->in_bases_cap, nbytes));
                KM_TRY(issue_host_copy(h, (const uint8_t *)bases + first, h->in_bases, nbytes, hc));
                copying = true;
            }
            d_bases = h->in_bases;
        }
    }
    if (bound == 0) return KMERCO_OK;   // no window fits in any read
    KM_TRY(ensure_set_capacity(h, bound));

    PartPlan pp = plan_partition(h, bound, nbytes);
    if (pp.part &&
        (ensure(h, &h->coarse, &h->coarse_alloc, pp.coarse_words()) != KMERCO_OK ||
         (pp.repart && ensure(h, &h->fine, &h->fine_alloc, pp.fine_words()) != KMERCO_OK) ||
         ensure(h, &h->part_ctr, &h->part_ctr_alloc, pp.ctr_words()) != KMERCO_OK))
        pp = PartPlan();   // the atomic design when the buffers cannot be had
    const uint64_t chunk = insert_chunk(h, pp, nbytes);
    KM_TRY(ensure(h, &h->first_read, &h->first_read_cap, (nbytes + chunk - 1) / chunk));
    const InsertArgs a = sample_args(h, d_bases, d_off, nreads, first, last);
    KM_CUDA(cudaEventRecord(h->ev[0], h->stream));
    KM_TRY(launch_sample_insert(h, a, pp, PartBufs{h->coarse, h->fine, h->part_ctr}, h->stream,
                                h->launches, copying ? &hc : nullptr));
    KM_CUDA(cudaEventRecord(h->ev[1], h->stream));
    h->insert_timed = true;
    h->classified = false;
    return KMERCO_OK;
}

namespace {

// After the top-bits sort of D keys in alt0 (the big-segment count at
// nbig_host, read back by the caller): radix-sorts the runs of equal top
// bits too long for one block, on stream s.  *any: whether there was one.
int sort_long_runs(kmerco_t *h, uint64_t D, int bits, uint64_t nb, bool *any, cudaStream_t s) {
    *any = false;
    if (!nb) return KMERCO_OK;
    const int kw = h->kw, passes = (bits + kRadixBits - 1) / kRadixBits;
    const uint64_t nbe = seg_bounds_entries(D, kw);
    const unsigned long long *big = h->seg_scratch + nbe;
    std::vector<unsigned long long> list(2 * nb);
    KM_CUDA(cudaMemcpyAsync(list.data(), big, 2 * nb * 8, cudaMemcpyDeviceToHost, s));
    KM_CUDA(cudaStreamSynchronize(s));
    for (uint64_t q = 0; q < nb; ++q) {
        if (list[2 * q + 1] <= big_segment_max()) continue;
        uint64_t *range = h->alt0 + list[2 * q] * kw;
        const uint64_t n_b = list[2 * q + 1];
        const uint64_t *res = range;
        KM_CUDA(radix_sort(range, h->alt1 + list[2 * q] * kw, range, n_b, kw, bits,
                           h->sort_scratch, &res, s));
        h->launches += 3 * (uint64_t)passes;
        if (res != range)
            KM_CUDA(cudaMemcpyAsync(range, res, n_b * kw * 8, cudaMemcpyDeviceToDevice, s));
        *any = true;
    }
    return KMERCO_OK;
}

// Orders a classification that rewrites the lists (into `words` words) after
// the result copies still queued: on the device when the lists' buffer is
// kept, on the host when it must be reallocated under them.
int wait_result_copies(kmerco_t *h, uint64_t words) {
    if (!h->out_pending) return KMERCO_OK;
    if (words > h->split_cap) {
        KM_CUDA(cudaStreamSynchronize(h->out_stream));
    } else {
        KM_CUDA(cudaStreamWaitEvent(h->stream, h->out_done, 0));
    }
    h->out_pending = false;
    return KMERCO_OK;
}

}  // namespace

int kmerco_classify(kmerco_t *h) {
    Range range("kmerco_classify");
    if (!h) return KMERCO_EINVAL;
    if (h->classified) return KMERCO_OK;
    DeviceGuard guard(h->device);
    KM_TRY(read_counters(h));
    KM_TRY(device_error_status(h->ctr_host->error));
    const uint64_t D = h->ctr_host->distinct;
    if (D >= 0xFFFFFFFFull) return KMERCO_ENOMEM;   // sort tiles index keys with 32 bits
    const int kw = h->kw;
    KM_TRY(ensure(h, &h->alt0, &h->alt0_cap, D * kw));
    KM_TRY(ensure(h, &h->alt1, &h->alt1_cap, D * kw));
    KM_TRY(ensure(h, &h->est, &h->est_cap, D));
    KM_TRY(wait_result_copies(h, D * kw));
    KM_TRY(ensure(h, &h->split, &h->split_cap, D * kw));
    KM_TRY(ensure(h, &h->sort_scratch, &h->sort_scratch_cap, sort_scratch_words(D, kw)));
    KM_TRY(ensure(h, &h->split_scratch, &h->split_scratch_cap, split_scratch_words(D)));
    KM_CUDA(cudaEventRecord(h->ev[2], h->stream));
    const uint64_t *const distinct_in = h->dlist;   // arrival order; left unchanged
    const uint64_t *sorted = distinct_in;
    const int bits = 2 * h->K;
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    // (small sets: the radix sort, without the bucket sort's fixed scratch)
    if (use_top_sort(D, kw, bits)) {
        // three stable passes on the top bits (dlist -> alt0 -> alt1 -> alt0),
        // then the segments in shared memory
        const int s0 = bits - kTopSortBits;
        KM_CUDA(radix_pass(distinct_in, h->alt0, D, kw, s0, h->sort_scratch, h->stream));
        KM_CUDA(radix_pass(h->alt0, h->alt1, D, kw, s0 + 8, h->sort_scratch, h->stream));
        KM_CUDA(radix_pass(h->alt1, h->alt0, D, kw, s0 + 16, h->sort_scratch, h->stream));
        h->launches += 9;
        const uint64_t nbe = seg_bounds_entries(D, kw);
        KM_TRY(ensure(h, &h->seg_scratch, &h->seg_scratch_cap, 3 * nbe + 1));
        unsigned long long *bnd = h->seg_scratch, *big = bnd + nbe, *nbig = big + 2 * nbe;
        KM_CUDA(top_segment_sort(h->alt0, D, kw, bits, bnd, big, nbig, h->stream));
        // runs of equal top bits longer than a segment: one block each ...
        KM_CUDA(big_segment_sort(h->alt0, h->alt1, D, kw, bits, big, nbig, h->stream));
        h->launches += 3;
        KM_TRY(ensure_bucket_host(h));
        KM_CUDA(cudaMemcpyAsync(h->bucket_host, nbig, 8, cudaMemcpyDeviceToHost, h->stream));
        KM_CUDA(cudaStreamSynchronize(h->stream));
        // ... and the few too long for one block: radix sorts of their own
        bool any;
        KM_TRY(sort_long_runs(h, D, bits, h->bucket_host[0], &any, h->stream));
        sorted = h->alt0;
    } else if (kw == 1 && bits >= kHistBits + 8 && D > kBucketSortMin &&
               D <= (uint64_t)kHistBins * (kBucketCap / 4)) {
        // Bucket sort: histogram of the top kHistBits key bits, adjacent bins
        // merged into super-buckets of at most kBucketCap keys, each sorted in
        // shared memory.  A single bin above kBucketCap is radix sorted.
        const int shift = bits - kHistBits;
        // device and pinned layout: hist u32[B] | map u32[B] | start u64[B+1] |
        // lo u64[B] | rsh i32[B] (| cursor u64[B] on the device only)
        const uint64_t words = kBucketHostWords;
        KM_TRY(ensure(h, &h->bucket_scratch, &h->bucket_scratch_cap, words + kHistBins));
        unsigned *d_hist = (unsigned *)h->bucket_scratch;
        unsigned *d_map = d_hist + kHistBins;
        unsigned long long *d_start = h->bucket_scratch + kHistBins;
        unsigned long long *d_lo = d_start + kHistBins + 1;
        int *d_rsh = (int *)(d_lo + kHistBins);
        unsigned long long *d_cursor = (unsigned long long *)(d_rsh + kHistBins);
        KM_TRY(ensure_bucket_host(h));
        unsigned *hist = (unsigned *)h->bucket_host, *map = hist + kHistBins;
        unsigned long long *start = h->bucket_host + kHistBins;
        unsigned long long *lo = start + kHistBins + 1;
        int *rsh = (int *)(lo + kHistBins);
        const uint64_t hb = bucket_hist_blocks(D);
        KM_TRY(ensure(h, &h->hist_partial, &h->hist_partial_cap, hb * kHistBins));
        KM_CUDA(bucket_histogram(distinct_in, D, shift, h->hist_partial, d_hist, h->stream));
        KM_CUDA(cudaMemcpyAsync(hist, d_hist, kHistBins * sizeof(unsigned), cudaMemcpyDeviceToHost,
                                h->stream));
        KM_CUDA(cudaStreamSynchronize(h->stream));
        // greedy merge of adjacent bins into super-buckets of <= kBucketCap keys;
        // super-bucket b covers bins [first, last]: key range lo .. (last+1) << shift
        unsigned nsuper = 0;
        unsigned long long cur = 0;
        int first = 0;
        start[0] = 0;
        auto close = [&](int last) {
            lo[nsuper] = (unsigned long long)first << shift;
            // key range of the super-bucket is (last - first + 1) << shift, which
            // needs up to 64 + log2(bins) bits; map it onto 2^12 sub-bins
            int r = ceil_log2((uint64_t)(last - first + 1)) + shift - 12;
            if (r > 63) r = 63;
            rsh[nsuper] = r < 0 ? 0 : r;
            start[nsuper + 1] = start[nsuper] + cur;
            ++nsuper;
        };
        for (int i = 0; i < kHistBins; ++i) {
            if (cur > 0 && cur + hist[i] > (unsigned long long)kBucketCap) {
                close(i - 1);
                cur = 0;
                first = i;
            }
            map[i] = nsuper;
            cur += hist[i];
        }
        close(kHistBins - 1);
        if (nsuper > (unsigned)kMaxSuper) {
            // too many super-buckets for the scatter's shared counters
            KM_CUDA(radix_sort(distinct_in, h->alt0, h->alt1, D, kw, bits, h->sort_scratch,
                               &sorted, h->stream));
            h->launches += 3 * (uint64_t)passes;
            goto sorted_done;
        }
        KM_CUDA(cudaMemcpyAsync(d_map, map, kHistBins * sizeof(unsigned), cudaMemcpyHostToDevice,
                                h->stream));
        KM_CUDA(cudaMemcpyAsync(d_start, start, (nsuper + 1) * sizeof(unsigned long long),
                                cudaMemcpyHostToDevice, h->stream));
        KM_CUDA(cudaMemcpyAsync(d_lo, lo, nsuper * sizeof(unsigned long long),
                                cudaMemcpyHostToDevice, h->stream));
        KM_CUDA(cudaMemcpyAsync(d_rsh, rsh, nsuper * sizeof(int), cudaMemcpyHostToDevice, h->stream));
        KM_CUDA(bucket_place_and_sort(distinct_in, h->alt0, D, shift, d_map, nsuper, d_start, d_lo,
                                      d_rsh, d_cursor, h->stream));
        h->launches += 4;
        sorted = h->alt0;
        for (unsigned b = 0; b < nsuper; ++b) {
            const uint64_t n_b = start[b + 1] - start[b];
            if (n_b <= (uint64_t)kBucketCap) continue;
            uint64_t *range = h->alt0 + start[b];
            const uint64_t *res = range;
            KM_CUDA(radix_sort(range, h->alt1, range, n_b, 1, bits, h->sort_scratch, &res,
                               h->stream));
            h->launches += 3 * (uint64_t)passes;
            if (res != range)
                KM_CUDA(cudaMemcpyAsync(range, res, n_b * 8, cudaMemcpyDeviceToDevice, h->stream));
        }
    } else {
        KM_CUDA(radix_sort(distinct_in, h->alt0, h->alt1, D, kw, bits, h->sort_scratch,
                           &sorted, h->stream));
        if (D > 1) h->launches += 3 * (uint64_t)passes;
    }
sorted_done:
    KM_CUDA(launch_classify_query(sorted, D, kw, h->G, h->tau, h->est, h->stream));
    h->est_exact = false;
    KM_CUDA(launch_split(sorted, h->est, D, kw, h->tau, h->split, h->split_scratch, h->ctr,
                         h->stream));
    if (D > 0) h->launches += 4;   // query + three split kernels
    KM_CUDA(cudaEventRecord(h->ev[3], h->stream));
    KM_TRY(read_counters(h));
    h->sorted = sorted;
    h->n_distinct = D;
    h->n_trusted = h->ctr_host->trusted;
    h->classified = true;
    h->classify_timed = true;
    return KMERCO_OK;
}

int kmerco_stats(kmerco_t *h, kmerco_stats_t *s) {
    if (!h || !s) return KMERCO_EINVAL;
    DeviceGuard guard(h->device);
    KM_CUDA(launch_count_saturated(h->G, h->ctr, h->stream));
    h->launches += 1;
    KM_TRY(read_counters(h));
    memset(s, 0, sizeof(*s));
    const DevCounters &c = *h->ctr_host;
    s->windows = c.windows;
    s->n_skipped = c.skipped;
    s->inserted = c.inserted;
    s->distinct = c.distinct;
    if (h->classified) {
        s->trustworthy = h->n_trusted;
        s->erroneous = h->n_distinct - h->n_trusted;
    }
    s->saturated_counters = c.saturated;
    s->m_actual = h->G.m;
    s->words = h->G.words;
    s->dim_x = h->G.dim_x;
    s->dim_y = h->G.dim_y;
    s->device_bytes = h->used;
    s->launches = h->launches;
    s->k = h->K;
    s->counter_bits = h->alpha;
    s->eta = h->eta;
    s->nhash = h->nhash;
    s->threshold = h->tau;
    s->classified = h->classified ? 1 : 0;
    if (h->insert_timed) cudaEventElapsedTime(&s->insert_ms, h->ev[0], h->ev[1]);
    if (h->classify_timed) cudaEventElapsedTime(&s->classify_ms, h->ev[2], h->ev[3]);
    cudaGetLastError();
    return device_error_status(c.error);
}

static int copy_out(kmerco_t *h, void *dst, const void *src, uint64_t bytes) {
    if (bytes == 0) return KMERCO_OK;
    KM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->stream));
    KM_CUDA(cudaStreamSynchronize(h->stream));
    return KMERCO_OK;
}

int kmerco_digest(kmerco_t *h, uint64_t *out) {
    if (!h || !out) return KMERCO_EINVAL;
    DeviceGuard guard(h->device);
    unsigned long long *acc = digest_sums(h);
    KM_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), h->stream));
    const uint64_t words = h->G.words;
    const unsigned grid = (unsigned)std::min<uint64_t>((words + 255) / 256, 152ull * 8);
    digest_kernel<<<grid, 256, 0, h->stream>>>(h->G.cells, words, acc);
    KM_CUDA(cudaGetLastError());
    h->launches += 1;
    KM_TRY(read_counters(h));
    const unsigned long long *got =
        (const unsigned long long *)((const char *)h->ctr_host + sizeof(DevCounters));
    out[0] = got[0];
    out[1] = got[1];
    return KMERCO_OK;
}

int kmerco_get_counters(kmerco_t *h, uint64_t *dst, uint64_t nwords) {
    if (!h || !dst) return KMERCO_EINVAL;
    if (nwords < h->G.words) return KMERCO_ESIZE;
    DeviceGuard guard(h->device);
    return copy_out(h, dst, h->G.cells, h->G.words * 8);
}

int kmerco_set_counters(kmerco_t *h, const uint64_t *src, uint64_t nwords) {
    if (!h || (!src && nwords)) return KMERCO_EINVAL;
    if (nwords != h->G.words) return KMERCO_ESIZE;
    DeviceGuard guard(h->device);
    KM_CUDA(cudaMemcpyAsync(h->G.cells, src, nwords * 8, cudaMemcpyDefault, h->stream));
    KM_CUDA(cudaStreamSynchronize(h->stream));
    h->classified = false;
    return KMERCO_OK;
}

int kmerco_add_distinct(kmerco_t *h, const uint64_t *keys, uint64_t n) {
    if (!h || (!keys && n)) return KMERCO_EINVAL;
    if (n == 0) return KMERCO_OK;
    DeviceGuard guard(h->device);
    const uint64_t words = n * h->kw;
    const uint64_t *d_keys = keys;
    if (!is_device_ptr(keys)) {   // stage host keys in the classification buffer
        KM_TRY(ensure(h, &h->alt0, &h->alt0_cap, words));
        KM_CUDA(cudaMemcpyAsync(h->alt0, keys, words * 8, cudaMemcpyHostToDevice, h->stream));
        d_keys = h->alt0;
    }
    KM_TRY(ensure_set_capacity(h, n));
    KM_CUDA(launch_reinsert(d_keys, n, h->kw, h->table, h->cap, set_tag(h), h->dlist,
                            h->dlist_cap, h->ctr, h->G.probe_limit, h->stream));
    h->launches += 1;
    KM_TRY(read_counters(h));
    KM_TRY(device_error_status(h->ctr_host->error));
    h->classified = false;
    return KMERCO_OK;
}

int kmerco_get_distinct(kmerco_t *h, uint64_t *keys, uint32_t *est, uint64_t cap, uint64_t *n) {
    if (!h || !n) return KMERCO_EINVAL;
    if (!h->classified) return KMERCO_ESTATE;
    *n = h->n_distinct;
    if (!keys) return KMERCO_OK;
    if (cap < h->n_distinct) return KMERCO_ESIZE;
    DeviceGuard guard(h->device);
    KM_TRY(copy_out(h, keys, h->sorted, h->n_distinct * h->kw * 8));
    if (est) {
        if (!h->est_exact) {   // the estimates of erroneous keys in full (Algorithm 5)
            KM_CUDA(launch_query(h->sorted, h->n_distinct, h->kw, h->K, h->G, h->est, h->stream));
            h->launches += h->n_distinct ? 1 : 0;
            h->est_exact = true;
        }
        KM_TRY(copy_out(h, est, h->est, h->n_distinct * 4));
    }
    return KMERCO_OK;
}

int kmerco_get_trusted(kmerco_t *h, uint64_t *keys, uint64_t cap, uint64_t *n) {
    if (!h || !n) return KMERCO_EINVAL;
    if (!h->classified) return KMERCO_ESTATE;
    *n = h->n_trusted;
    if (!keys) return KMERCO_OK;
    if (cap < h->n_trusted) return KMERCO_ESIZE;
    DeviceGuard guard(h->device);
    return copy_out(h, keys, h->split, h->n_trusted * h->kw * 8);
}

int kmerco_get_erroneous(kmerco_t *h, uint64_t *keys, uint64_t cap, uint64_t *n) {
    if (!h || !n) return KMERCO_EINVAL;
    if (!h->classified) return KMERCO_ESTATE;
    const uint64_t E = h->n_distinct - h->n_trusted;
    *n = E;
    if (!keys) return KMERCO_OK;
    if (cap < E) return KMERCO_ESIZE;
    DeviceGuard guard(h->device);
    return copy_out(h, keys, h->split + h->n_trusted * h->kw, E * h->kw * 8);
}

int kmerco_get_lists_async(kmerco_t *h, uint64_t *trusted, uint64_t tcap, uint64_t *erroneous,
                           uint64_t ecap, uint64_t *nt, uint64_t *ne) {
    if (!h || !nt || !ne) return KMERCO_EINVAL;
    if (!h->classified) return KMERCO_ESTATE;
    const uint64_t T = h->n_trusted, E = h->n_distinct - h->n_trusted;
    *nt = T;
    *ne = E;
    if ((trusted && tcap < T) || (erroneous && ecap < E)) return KMERCO_ESIZE;
    if ((!trusted || T == 0) && (!erroneous || E == 0)) return KMERCO_OK;
    DeviceGuard guard(h->device);
    if (!h->out_stream) {
        if (cudaStreamCreateWithFlags(&h->out_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->out_ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->out_done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return KMERCO_ECUDA;
        }
    }
    KM_CUDA(cudaEventRecord(h->out_ready, h->stream));
    KM_CUDA(cudaStreamWaitEvent(h->out_stream, h->out_ready, 0));
    const uint64_t w = (uint64_t)h->kw * 8;
    if (trusted && T)
        KM_CUDA(cudaMemcpyAsync(trusted, h->split, T * w, cudaMemcpyDefault, h->out_stream));
    if (erroneous && E)
        KM_CUDA(cudaMemcpyAsync(erroneous, h->split + T * h->kw, E * w, cudaMemcpyDefault,
                                h->out_stream));
    KM_CUDA(cudaEventRecord(h->out_done, h->out_stream));
    h->out_pending = true;
    return KMERCO_OK;
}

int kmerco_sync(kmerco_t *h) {
    if (!h) return KMERCO_EINVAL;
    DeviceGuard guard(h->device);
    KM_CUDA(cudaStreamSynchronize(h->stream));
    if (h->copy_stream) KM_CUDA(cudaStreamSynchronize(h->copy_stream));
    if (h->out_stream) KM_CUDA(cudaStreamSynchronize(h->out_stream));
    KM_TRY(read_counters(h));
    return device_error_status(h->ctr_host->error);
}

int kmerco_query(kmerco_t *h, const uint64_t *keys, uint64_t n, uint32_t *est) {
    if (!h) return KMERCO_EINVAL;
    if (n == 0) return KMERCO_OK;
    if (!keys || !est) return KMERCO_EINVAL;
    DeviceGuard guard(h->device);
    const int kw = h->kw;
    const uint64_t *dk = keys;
    uint32_t *de = est;
    const bool keys_dev = is_device_ptr(keys), est_dev = is_device_ptr(est);
    if (!keys_dev || !est_dev) {
        if (!h->q_keys || h->q_cap < n) {
            dev_free(h, h->q_keys, h->q_cap * 16);
            dev_free(h, h->q_est, h->q_cap * 4);
            h->q_keys = nullptr;
            h->q_est = nullptr;
            h->q_cap = 0;
            void *p;
            KM_TRY(dev_alloc(h, &p, n * 16));
            h->q_keys = (uint64_t *)p;
            if (dev_alloc(h, &p, n * 4) != KMERCO_OK) {
                dev_free(h, h->q_keys, n * 16);
                h->q_keys = nullptr;
                return KMERCO_ENOMEM;
            }
            h->q_est = (uint32_t *)p;
            h->q_cap = n;
        }
    }
    if (!keys_dev) {
        KM_CUDA(cudaMemcpyAsync(h->q_keys, keys, n * kw * 8, cudaMemcpyHostToDevice, h->stream));
        dk = h->q_keys;
    }
    if (!est_dev) de = h->q_est;
    KM_CUDA(launch_query(dk, n, kw, h->K, h->G, de, h->stream));
    h->launches += 1;
    if (!est_dev) KM_CUDA(cudaMemcpyAsync(est, de, n * 4, cudaMemcpyDeviceToHost, h->stream));
    KM_CUDA(cudaStreamSynchronize(h->stream));
    return KMERCO_OK;
}

int kmerco_merge_cells(kmerco_t *h, const uint64_t *src, uint64_t first_word, uint64_t nwords) {
    Range range("kmerco_merge_cells");
    if (!h || (!src && nwords)) return KMERCO_EINVAL;
    if (first_word > h->G.words || nwords > h->G.words - first_word) return KMERCO_ESIZE;
    if (nwords == 0) return KMERCO_OK;
    DeviceGuard guard(h->device);
    const uint64_t *d_src = src;
    if (!is_device_ptr(src)) {   // host words: staged in the classification buffer
        KM_TRY(ensure(h, &h->alt0, &h->alt0_cap, nwords));
        KM_CUDA(cudaMemcpyAsync(h->alt0, src, nwords * 8, cudaMemcpyHostToDevice, h->stream));
        d_src = h->alt0;
    }
    Geometry part = h->G;   // the same counters, over words [first_word, first_word + nwords)
    part.cells = h->G.cells + first_word;
    part.words = nwords;
    KM_CUDA(launch_merge(part.cells, d_src, part, h->stream));
    h->launches += 1;
    KM_CUDA(cudaStreamSynchronize(h->stream));
    h->classified = false;
    return KMERCO_OK;
}

int kmerco_rank_of(kmerco_t *h, const uint64_t *probes, uint64_t n, uint64_t *ranks) {
    if (!h || (n && (!probes || !ranks))) return KMERCO_EINVAL;
    if (!h->classified) return KMERCO_ESTATE;
    if (n == 0) return KMERCO_OK;
    DeviceGuard guard(h->device);
    const int kw = h->kw;
    // probes and ranks through the query staging buffer (kw words in, one
    // word out per probe; the buffer holds two words per slot)
    const uint64_t slots = (n * (uint64_t)(kw + 1) + 1) / 2;
    if (!h->q_keys || h->q_cap < slots) {
        dev_free(h, h->q_keys, h->q_cap * 16);
        dev_free(h, h->q_est, h->q_cap * 4);
        h->q_keys = nullptr;
        h->q_est = nullptr;
        h->q_cap = 0;
        void *p;
        KM_TRY(dev_alloc(h, &p, slots * 16));
        h->q_keys = (uint64_t *)p;
        if (dev_alloc(h, &p, slots * 4) != KMERCO_OK) {
            dev_free(h, h->q_keys, slots * 16);
            h->q_keys = nullptr;
            return KMERCO_ENOMEM;
        }
        h->q_est = (uint32_t *)p;
        h->q_cap = slots;
    }
    KM_CUDA(cudaMemcpyAsync(h->q_keys, probes, n * kw * 8, cudaMemcpyDefault, h->stream));
    uint64_t *d_ranks = h->q_keys + n * kw;
    KM_CUDA(launch_lower_bound(h->sorted, h->n_distinct, kw, h->q_keys, n, d_ranks, h->stream));
    h->launches += 1;
    KM_CUDA(cudaMemcpyAsync(ranks, d_ranks, n * 8, cudaMemcpyDefault, h->stream));
    KM_CUDA(cudaStreamSynchronize(h->stream));
    return KMERCO_OK;
}

int kmerco_merge(kmerco_t *dst, kmerco_t *src) {
    Range range("kmerco_merge");
    if (!dst || !src || dst == src) return KMERCO_EINVAL;
    if (dst->K != src->K || dst->G.m != src->G.m || dst->G.dim_x != src->G.dim_x ||
        dst->G.dim_y != src->G.dim_y || dst->alpha != src->alpha ||
        dst->nhash != src->nhash || dst->canonical != src->canonical || dst->device != src->device)
        return KMERCO_EINVAL;
    DeviceGuard guard(dst->device);
    KM_TRY(read_counters(src));
    KM_TRY(device_error_status(src->ctr_host->error));
    const DevCounters sc = *src->ctr_host;
    KM_TRY(ensure_set_capacity(dst, sc.distinct));
    KM_CUDA(launch_merge(dst->G.cells, src->G.cells, dst->G, dst->stream));
    KM_CUDA(launch_reinsert(src->dlist, sc.distinct, dst->kw, dst->table, dst->cap,
                            set_tag(dst), dst->dlist, dst->dlist_cap, dst->ctr,
                            dst->G.probe_limit, dst->stream));
    dst->launches += sc.distinct ? 2 : 1;
    KM_TRY(read_counters(dst));
    DevCounters dc = *dst->ctr_host;
    dc.windows += sc.windows;
    dc.skipped += sc.skipped;
    dc.inserted += sc.inserted;
    // only the three totals change; the device may not touch them meanwhile
    KM_CUDA(cudaMemcpyAsync(&dst->ctr->windows, &dc.windows, 3 * sizeof(unsigned long long),
                            cudaMemcpyHostToDevice, dst->stream));
    KM_CUDA(cudaStreamSynchronize(dst->stream));
    dst->classified = false;
    return KMERCO_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
constexpr int kBatchStreams = 8;
// Distinct keys above which a batch sample's classification sorts by the top
// key bits and segments rather than by a full radix sort.
constexpr uint64_t kBatchTopSortMin = 1ull << 16;

struct kmerco_batch {
    std::vector<kmerco_t *> h;
    int n, kw, device;
    cudaStream_t stream;
    int sms;
    InsertArgs *d_args;                      // per sample
    unsigned long long *d_chunk_end;         // inclusive prefix of chunks
    unsigned long long *d_bound;             // kBoundOutWords per sample
    const uint64_t **d_offs;                 // device copies of the pointer arrays
    uint64_t *d_nreads;
    std::vector<InsertArgs> args;
    std::vector<unsigned long long> chunk_end, bound_host;
    std::vector<const char *> p_bases;       // inputs of the planned launch
    std::vector<const uint64_t *> p_offs;
    std::vector<uint32_t> graph_gen;         // distinct-set generation of each handle at capture
    std::vector<uint64_t> p_nreads;
    bool planned, tuned, have_graph;
    int chunk, bpm;
    float tuned_ms;
    unsigned long long total_chunks;
    uint64_t launches;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaEvent_t ev[2];
    // per-sample schedule: each sample's own insert kernels (partitioned
    // design where it applies) on one of `streams` concurrent streams
    int sched;                               // 0 persistent launch, 1 per-sample kernels
    int streams;
    cudaStream_t aux[kBatchStreams];
    cudaEvent_t fork, join[kBatchStreams];
    PartBufs bufs[kBatchStreams];            // increment-code scratch of each stream
    uint64_t buf_words[kBatchStreams][3];    // their sizes (coarse, fine, counters)
    std::vector<PartPlan> plans;             // per sample
    std::vector<uint64_t> load;              // per sample: windows, for stream assignment
    // classification graph, replayed while the distinct counts and buffers match
    bool have_cls;
    cudaGraph_t cls_graph;
    cudaGraphExec_t cls_exec;
    std::vector<uint64_t> cls_key;           // D and buffer addresses of every sample
    std::vector<const uint64_t *> cls_sorted;
    uint64_t cls_launches;
};

namespace {

// Build the per-sample arguments for chunk size `chunk` and upload them.
int batch_build_args(kmerco_batch *b, int chunk) {
    b->args.resize(b->n);
    b->chunk_end.resize(b->n);
    unsigned long long acc = 0;
    for (int i = 0; i < b->n; ++i) {
        kmerco_t *h = b->h[i];
        const unsigned long long *bo = &b->bound_host[(size_t)i * kBoundOutWords];
        const uint64_t first = bo[1], last = bo[2];
        const bool any = h->whole_file ? last - first >= (uint64_t)h->K : bo[0] != 0;
        const uint64_t nchunks = any ? (last - first + chunk - 1) / chunk : 0;
        InsertArgs &a = b->args[i];
        memset(&a, 0, sizeof(a));
        a.bases = (const uint8_t *)b->p_bases[i] + first;
        a.offsets = b->p_offs[i];
        a.nreads = b->p_nreads[i];
        a.first = first;
        a.last = last;
        a.first_read = h->first_read;
        a.chunk_begin = 0;
        a.nchunks = nchunks;
        a.K = h->K;
        a.canonical = h->canonical;
        a.whole_file = h->whole_file;
        a.G = h->G;
        a.table = h->table;
        a.cap = h->cap;
        a.set_tag = set_tag(h);
        a.dlist = h->dlist;
        a.dlist_cap = h->dlist_cap;
        a.ctr = h->ctr;
        acc += nchunks;
        b->chunk_end[i] = acc;
    }
    b->total_chunks = acc;
    KM_CUDA(cudaMemcpyAsync(b->d_args, b->args.data(), b->n * sizeof(InsertArgs),
                            cudaMemcpyHostToDevice, b->stream));
    KM_CUDA(cudaMemcpyAsync(b->d_chunk_end, b->chunk_end.data(), b->n * sizeof(unsigned long long),
                            cudaMemcpyHostToDevice, b->stream));
    KM_CUDA(cudaStreamSynchronize(b->stream));
    return KMERCO_OK;
}

// Reset every sample on the stream (capturable: memsets only).
int batch_reset_device(kmerco_batch *b) {
    for (kmerco_t *h : b->h) {
        KM_CUDA(cudaMemsetAsync(h->G.cells, 0, h->G.words * 8, b->stream));
        if (h->table) KM_CUDA(cudaMemsetAsync(h->table, 0xFF, h->cap * h->kw * 8, b->stream));
        KM_CUDA(cudaMemsetAsync(h->ctr, 0, sizeof(DevCounters), b->stream));
    }
    return KMERCO_OK;
}

int batch_launch(kmerco_batch *b, int chunk, int bpm) {
    KM_CUDA(launch_insert_batch(b->d_args, b->d_chunk_end, b->n, b->total_chunks, b->kw, chunk,
                                b->sms * bpm, b->stream));
    b->launches += b->total_chunks ? 2 : 0;
    return KMERCO_OK;
}

// Streams of the per-sample schedule: each sample to the least loaded of
// `S` streams, largest samples first.
std::vector<int> batch_assign(const kmerco_batch *b, int S) {
    std::vector<int> order(b->n), out(b->n, 0);
    for (int i = 0; i < b->n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return b->load[x] > b->load[y]; });
    std::vector<uint64_t> acc(S, 0);
    for (int i : order) {
        int k = 0;
        for (int j = 1; j < S; ++j)
            if (acc[j] < acc[k]) k = j;
        out[i] = k;
        acc[k] += b->load[i];
    }
    return out;
}

// Scratch of every stream, sized for the largest plan of any sample (so any
// assignment fits).  Returns false when it cannot be had.
bool batch_alloc_scratch(kmerco_batch *b) {
    uint64_t need[3] = {0, 0, 0};
    for (const PartPlan &pp : b->plans) {
        if (!pp.part) continue;
        need[0] = std::max(need[0], pp.coarse_words());
        need[1] = std::max(need[1], pp.fine_words());
        need[2] = std::max(need[2], pp.ctr_words());
    }
    for (int k = 0; k < kBatchStreams; ++k) {
        if (!b->aux[k] && cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking) != cudaSuccess)
            return false;
        if (!b->join[k] && cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) != cudaSuccess)
            return false;
        void **ptrs[3] = {(void **)&b->bufs[k].coarse, (void **)&b->bufs[k].fine,
                          (void **)&b->bufs[k].ctr};
        const uint64_t elem[3] = {4, 4, 8};
        for (int q = 0; q < 3; ++q) {
            if (b->buf_words[k][q] >= need[q]) continue;
            if (*ptrs[q]) {
                cudaStreamSynchronize(b->aux[k]);
                raw_free(b->h[0], *ptrs[q], b->buf_words[k][q] * elem[q]);
            }
            *ptrs[q] = nullptr;
            b->buf_words[k][q] = 0;
            if (raw_alloc(b->h[0], ptrs[q], need[q] * elem[q]) != KMERCO_OK) return false;
            b->buf_words[k][q] = need[q];
        }
    }
    return b->fork || cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
}

// Per-sample schedule on S streams forked from and joined back into the
// batch stream (capturable: no host synchronisation).
int batch_launch_sliced(kmerco_batch *b, int S, bool reset) {
    const std::vector<int> where = batch_assign(b, S);
    KM_CUDA(cudaEventRecord(b->fork, b->stream));
    for (int k = 0; k < S; ++k) KM_CUDA(cudaStreamWaitEvent(b->aux[k], b->fork, 0));
    for (int i = 0; i < b->n; ++i) {
        kmerco_t *h = b->h[i];
        cudaStream_t st = b->aux[where[i]];
        if (reset) {
            KM_CUDA(cudaMemsetAsync(h->G.cells, 0, h->G.words * 8, st));
            if (h->table) KM_CUDA(cudaMemsetAsync(h->table, 0xFF, h->cap * h->kw * 8, st));
            KM_CUDA(cudaMemsetAsync(h->ctr, 0, sizeof(DevCounters), st));
        }
        const unsigned long long *bo = &b->bound_host[(size_t)i * kBoundOutWords];
        const bool any = h->whole_file ? bo[2] - bo[1] >= (uint64_t)h->K : bo[0] != 0;
        if (!any) continue;
        const InsertArgs a = sample_args(h, (const uint8_t *)b->p_bases[i] + bo[1], b->p_offs[i],
                                         b->p_nreads[i], bo[1], bo[2]);
        KM_TRY(launch_sample_insert(h, a, b->plans[i], b->bufs[where[i]], st, b->launches));
    }
    for (int k = 0; k < S; ++k) {
        KM_CUDA(cudaEventRecord(b->join[k], b->aux[k]));
        KM_CUDA(cudaStreamWaitEvent(b->stream, b->join[k], 0));
    }
    return KMERCO_OK;
}

// The chosen schedule: the persistent launch, or the per-sample kernels.
int batch_run(kmerco_batch *b, bool reset) {
    if (b->sched == 1) return batch_launch_sliced(b, b->streams, reset);
    if (reset) KM_TRY(batch_reset_device(b));
    return batch_launch(b, b->chunk, b->bpm);
}

void batch_mark_inserted(kmerco_batch *b) {
    for (kmerco_t *h : b->h) {
        h->classified = false;
        h->n_distinct = h->n_trusted = 0;
        h->insert_timed = h->classify_timed = false;
    }
}

}  // namespace

extern "C" {

int kmerco_batch_create(kmerco_t *const *handles, int n, kmerco_batch_t **out) {
    if (!out) return KMERCO_EINVAL;
    *out = nullptr;
    if (!handles || n < 1 || n > 65535) return KMERCO_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!handles[i]) return KMERCO_EINVAL;
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return KMERCO_EINVAL;
        if (handles[i]->device != handles[0]->device || handles[i]->stream != handles[0]->stream ||
            handles[i]->K != handles[0]->K)
            return KMERCO_EINVAL;
    }
    kmerco_batch *b = new (std::nothrow) kmerco_batch();
    if (!b) return KMERCO_ENOMEM;
    b->h.assign(handles, handles + n);
    b->n = n;
    b->kw = handles[0]->kw;
    b->device = handles[0]->device;
    b->stream = handles[0]->stream;
    b->chunk = kChunk;
    b->bpm = 4;
    DeviceGuard guard(b->device);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (b->sms <= 0) b->sms = 1;
    const int mx = insert_batch_blocks_per_sm(b->kw, kChunk);
    if (b->bpm > mx) b->bpm = mx;
    const kmerco_t *h0 = handles[0];   // the batch's small arrays come from its allocator
    bool ok = raw_alloc(h0, (void **)&b->d_args, n * sizeof(InsertArgs)) == KMERCO_OK &&
              raw_alloc(h0, (void **)&b->d_chunk_end, n * sizeof(unsigned long long)) == KMERCO_OK &&
              raw_alloc(h0, (void **)&b->d_bound, (size_t)n * kBoundOutWords * 8) == KMERCO_OK &&
              raw_alloc(h0, (void **)&b->d_offs, n * sizeof(uint64_t *)) == KMERCO_OK &&
              raw_alloc(h0, (void **)&b->d_nreads, n * sizeof(uint64_t)) == KMERCO_OK &&
              cudaEventCreate(&b->ev[0]) == cudaSuccess && cudaEventCreate(&b->ev[1]) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        kmerco_batch_destroy(b);
        return KMERCO_ENOMEM;
    }
    *out = b;
    return KMERCO_OK;
}

void kmerco_batch_destroy(kmerco_batch_t *b) {
    if (!b) return;
    {
        DeviceGuard guard(b->device);
        if (b->stream) cudaStreamSynchronize(b->stream);
        if (b->have_graph) {
            cudaGraphExecDestroy(b->exec);
            cudaGraphDestroy(b->graph);
        }
        if (b->have_cls) {
            cudaGraphExecDestroy(b->cls_exec);
            cudaGraphDestroy(b->cls_graph);
        }
        const kmerco_t *h0 = b->h[0];
        const size_t n = (size_t)b->n;
        raw_free(h0, b->d_args, n * sizeof(InsertArgs));
        raw_free(h0, b->d_chunk_end, n * sizeof(unsigned long long));
        raw_free(h0, b->d_bound, n * kBoundOutWords * 8);
        raw_free(h0, b->d_offs, n * sizeof(uint64_t *));
        raw_free(h0, b->d_nreads, n * sizeof(uint64_t));
        for (int i = 0; i < 2; ++i)
            if (b->ev[i]) cudaEventDestroy(b->ev[i]);
        for (int k = 0; k < kBatchStreams; ++k) {
            if (b->aux[k]) cudaStreamSynchronize(b->aux[k]);
            raw_free(h0, b->bufs[k].coarse, b->buf_words[k][0] * 4);
            raw_free(h0, b->bufs[k].fine, b->buf_words[k][1] * 4);
            raw_free(h0, b->bufs[k].ctr, b->buf_words[k][2] * 8);
            if (b->aux[k]) cudaStreamDestroy(b->aux[k]);
            if (b->join[k]) cudaEventDestroy(b->join[k]);
        }
        if (b->fork) cudaEventDestroy(b->fork);
        cudaGetLastError();
    }
    delete b;
}

int kmerco_batch_insert(kmerco_batch_t *b, const char *const *bases,
                        const uint64_t *const *offsets, const uint64_t *nreads, int reset) {
    Range range("kmerco_batch_insert");
    if (!b || !bases || !offsets || !nreads) return KMERCO_EINVAL;
    DeviceGuard guard(b->device);
    // the same inputs as the captured launch: replay the graph
    bool same = b->planned && reset && b->have_graph;
    for (int i = 0; same && i < b->n; ++i)
        same = b->p_bases[i] == bases[i] && b->p_offs[i] == offsets[i] &&
               b->p_nreads[i] == nreads[i] && b->h[i]->gen == b->graph_gen[i];
    if (same) {
        KM_CUDA(cudaGraphLaunch(b->exec, b->stream));
        b->launches += b->total_chunks ? 2 : 0;
        batch_mark_inserted(b);
        return KMERCO_OK;
    }
    uint64_t max_reads = 0;
    for (int i = 0; i < b->n; ++i) {
        if (nreads[i] >= 0xFFFFFFFFull) return KMERCO_EINVAL;
        if (nreads[i] && (!offsets[i] || !is_device_ptr(offsets[i]))) return KMERCO_EINVAL;
        if (bases[i] && !is_device_ptr(bases[i])) return KMERCO_EINVAL;
        if (nreads[i] > max_reads) max_reads = nreads[i];
    }
    b->p_bases.assign(bases, bases + b->n);
    b->p_offs.assign(offsets, offsets + b->n);
    b->p_nreads.assign(nreads, nreads + b->n);
    if (b->have_graph) {
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->have_graph = false;
    }
    // plan: window bounds and offsets of every sample in one launch
    KM_CUDA(cudaMemcpyAsync(b->d_offs, b->p_offs.data(), b->n * sizeof(uint64_t *),
                            cudaMemcpyHostToDevice, b->stream));
    KM_CUDA(cudaMemcpyAsync(b->d_nreads, nreads, b->n * sizeof(uint64_t), cudaMemcpyHostToDevice,
                            b->stream));
    KM_CUDA(launch_window_bound_batch(b->d_offs, b->d_nreads, b->n, b->h[0]->K, b->d_bound,
                                      max_reads, b->stream));
    b->launches += 1;
    b->bound_host.resize((size_t)b->n * kBoundOutWords);
    KM_CUDA(cudaMemcpyAsync(b->bound_host.data(), b->d_bound, (size_t)b->n * kBoundOutWords * 8,
                            cudaMemcpyDeviceToHost, b->stream));
    KM_CUDA(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i) {
        if (b->bound_host[(size_t)i * kBoundOutWords + 3]) return KMERCO_EINVAL;
        if (b->bound_host[(size_t)i * kBoundOutWords + 2] > b->bound_host[(size_t)i * kBoundOutWords + 1] &&
            !bases[i])
            return KMERCO_EINVAL;
    }
    // capacities (host work; never inside a capture)
    b->plans.assign(b->n, PartPlan());
    b->load.assign(b->n, 0);
    for (int i = 0; i < b->n; ++i) {
        kmerco_t *h = b->h[i];
        if (reset) KM_TRY(kmerco_reset(h));
        const unsigned long long *bo = &b->bound_host[(size_t)i * kBoundOutWords];
        uint64_t bound = bo[0];
        if (h->whole_file)   // the sample's reads are one sequence
            bound = bo[2] - bo[1] >= (uint64_t)h->K ? bo[2] - bo[1] - h->K + 1 : 0;
        KM_TRY(ensure_set_capacity(h, bound));
        const uint64_t most = (bo[2] - bo[1] + kSmallChunk - 1) / kSmallChunk;   // chunks at the smallest chunk size
        KM_TRY(ensure(h, &h->first_read, &h->first_read_cap, most ? most : 1));
        b->plans[i] = plan_partition(h, bound, bo[2] - bo[1]);
        b->load[i] = bound;
    }
    KM_CUDA(cudaStreamSynchronize(b->stream));
    const bool sliced_ok = batch_alloc_scratch(b);
    if (!sliced_ok) b->sched = 0;   // the persistent schedule needs no scratch
    b->planned = true;
    // autotune once per batch: chunk size x resident blocks, timed on this input
    if (reset && !b->tuned) {
        const int chunks[2] = {1024, 2048};
        float best = 1e30f;
        for (int c : chunks) {
            KM_TRY(batch_build_args(b, c));
            const int mx = insert_batch_blocks_per_sm(b->kw, c);
            for (int bpm = 2; bpm <= mx && bpm <= 8; ++bpm) {
                KM_TRY(batch_reset_device(b));
                KM_CUDA(cudaEventRecord(b->ev[0], b->stream));
                KM_TRY(batch_launch(b, c, bpm));
                KM_CUDA(cudaEventRecord(b->ev[1], b->stream));
                KM_CUDA(cudaEventSynchronize(b->ev[1]));
                float ms = 0;
                cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
                if (ms < best) {
                    best = ms;
                    b->chunk = c;
                    b->bpm = bpm;
                }
            }
        }
        b->sched = 0;
        // the per-sample schedule on 1, 2, 4 or 8 streams
        for (int S = 1; sliced_ok && S <= kBatchStreams; S *= 2) {
            KM_TRY(batch_reset_device(b));
            KM_CUDA(cudaEventRecord(b->ev[0], b->stream));
            KM_TRY(batch_launch_sliced(b, S, false));
            KM_CUDA(cudaEventRecord(b->ev[1], b->stream));
            KM_CUDA(cudaEventSynchronize(b->ev[1]));
            float ms = 0;
            cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
            if (ms < best) {
                best = ms;
                b->sched = 1;
                b->streams = S;
            }
        }
        b->tuned = true;
        b->tuned_ms = best;
    }
    KM_TRY(batch_build_args(b, b->chunk));
    if (reset) {
        // reset + insert of every sample as one CUDA graph (plain launches on
        // a stream that cannot be captured, such as the legacy default stream)
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            KM_TRY(batch_run(b, true));
        } else {
            int st = batch_run(b, true);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
            if (st != KMERCO_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            KM_CUDA(ec);
            if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
                cudaGraphDestroy(g);
                return KMERCO_ECUDA;
            }
            b->graph = g;
            b->have_graph = true;
            b->graph_gen.resize(b->n);   // the tags the graph's launches carry
            for (int i = 0; i < b->n; ++i) b->graph_gen[i] = b->h[i]->gen;
            KM_CUDA(cudaGraphLaunch(b->exec, b->stream));
        }
    } else {
        KM_TRY(batch_run(b, false));
    }
    batch_mark_inserted(b);
    return KMERCO_OK;
}

int kmerco_batch_schedule(kmerco_batch_t *b, int schedule, int streams) {
    if (!b || schedule < -1 || schedule > 1) return KMERCO_EINVAL;
    if (schedule == 1 && (streams < 1 || streams > kBatchStreams || (streams & (streams - 1))))
        return KMERCO_EINVAL;
    if (b->have_graph) {   // the captured graph follows the old schedule
        DeviceGuard guard(b->device);
        cudaStreamSynchronize(b->stream);
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->have_graph = false;
    }
    if (schedule < 0) {
        b->tuned = false;
        return KMERCO_OK;
    }
    b->tuned = true;
    b->tuned_ms = 0;
    b->sched = schedule;
    b->streams = schedule == 1 ? streams : 0;
    return KMERCO_OK;
}

int kmerco_batch_classify(kmerco_batch_t *b) {
    Range range("kmerco_batch_classify");
    if (!b) return KMERCO_EINVAL;
    DeviceGuard guard(b->device);
    // one readback of every sample's totals
    for (kmerco_t *h : b->h)
        KM_CUDA(cudaMemcpyAsync(h->ctr_host, h->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                                b->stream));
    KM_CUDA(cudaStreamSynchronize(b->stream));
    std::vector<uint64_t> D(b->n, 0);
    std::vector<char> top(b->n, 0);   // the sample takes the top-bits sort
    for (int i = 0; i < b->n; ++i) {
        kmerco_t *h = b->h[i];
        if (h->classified) continue;
        KM_TRY(device_error_status(h->ctr_host->error));
        D[i] = h->ctr_host->distinct;
        if (D[i] >= 0xFFFFFFFFull) return KMERCO_ENOMEM;   // sort tiles index keys with 32 bits
        const int kw = h->kw;
        // three radix passes and the segments instead of a full radix sort;
        // the bucket sort is not used here (it reads its histogram back)
        top[i] = 2 * h->K >= kTopSortBits + 12 && D[i] > kBatchTopSortMin;
        if (top[i]) {
            KM_TRY(ensure(h, &h->seg_scratch, &h->seg_scratch_cap,
                          3 * seg_bounds_entries(D[i], kw) + 1));
            KM_TRY(ensure_bucket_host(h));
        }
        KM_TRY(ensure(h, &h->alt0, &h->alt0_cap, D[i] * kw));
        KM_TRY(ensure(h, &h->alt1, &h->alt1_cap, D[i] * kw));
        KM_TRY(ensure(h, &h->est, &h->est_cap, D[i]));
        if (h->out_pending) {   // the batch writes the lists on its own streams
            KM_CUDA(cudaStreamSynchronize(h->out_stream));
            h->out_pending = false;
        }
        KM_TRY(ensure(h, &h->split, &h->split_cap, D[i] * kw));
        KM_TRY(ensure(h, &h->sort_scratch, &h->sort_scratch_cap, sort_scratch_words(D[i], kw)));
        KM_TRY(ensure(h, &h->split_scratch, &h->split_scratch_cap, split_scratch_words(D[i])));
    }
    bool streams_ok = b->fork != nullptr;
    for (int k = 0; streams_ok && k < kBatchStreams; ++k) streams_ok = b->aux[k] && b->join[k];
    if (!streams_ok) {   // no per-sample streams were set up: one handle at a time
        for (kmerco_t *h : b->h) KM_TRY(kmerco_classify(h));
        return KMERCO_OK;
    }
    // every sample's radix sort, query and split, the samples spread over the
    // streams by distinct count (no host synchronisation in between), as one
    // CUDA graph: replayed while every sample's distinct count and buffers
    // are those it was captured with
    std::vector<uint64_t> key;
    key.reserve((size_t)b->n * 11);
    for (int i = 0; i < b->n; ++i) {
        const kmerco_t *h = b->h[i];
        const uint64_t fields[11] = {h->classified ? ~0ull : D[i], (uint64_t)h->dlist,
                                     (uint64_t)h->alt0, (uint64_t)h->alt1, (uint64_t)h->est,
                                     (uint64_t)h->split, (uint64_t)h->sort_scratch,
                                     (uint64_t)h->split_scratch, (uint64_t)h->ctr,
                                     (uint64_t)h->G.cells, (uint64_t)h->seg_scratch};
        key.insert(key.end(), fields, fields + 11);
    }
    if (b->have_cls && key == b->cls_key) {
        KM_CUDA(cudaGraphLaunch(b->cls_exec, b->stream));
        b->launches += b->cls_launches;
        for (int i = 0; i < b->n; ++i) {
            kmerco_t *h = b->h[i];
            if (h->classified) continue;
            h->sorted = b->cls_sorted[i];
            h->n_distinct = D[i];
        }
    } else {
        if (b->have_cls) {
            cudaGraphExecDestroy(b->cls_exec);
            cudaGraphDestroy(b->cls_graph);
            b->have_cls = false;
        }
        const bool capture =
            cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (!capture) cudaGetLastError();   // plain launches on a stream that cannot capture
        const uint64_t l0 = b->launches;
        std::vector<int> order(b->n);
        for (int i = 0; i < b->n; ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](int x, int y) { return D[x] > D[y]; });
        std::vector<uint64_t> acc(kBatchStreams, 0);
        b->cls_sorted.assign(b->n, nullptr);
        int st_launch = KMERCO_OK;
        auto go = [&]() -> int {
            KM_CUDA(cudaEventRecord(b->fork, b->stream));
            for (int k = 0; k < kBatchStreams; ++k)
                KM_CUDA(cudaStreamWaitEvent(b->aux[k], b->fork, 0));
            for (int i : order) {
                kmerco_t *h = b->h[i];
                if (h->classified) continue;
                int k = 0;
                for (int j = 1; j < kBatchStreams; ++j)
                    if (acc[j] < acc[k]) k = j;
                acc[k] += D[i] + 4096;
                cudaStream_t st = b->aux[k];
                const int bits = 2 * h->K, passes = (bits + kRadixBits - 1) / kRadixBits;
                const uint64_t *sorted = h->dlist;
                uint64_t n_launch = D[i] ? 4 : 0;   // query + three split kernels
                if (top[i]) {   // as in kmerco_classify; long runs are checked below
                    const int s0 = bits - kTopSortBits;
                    const uint64_t nbe = seg_bounds_entries(D[i], h->kw);
                    unsigned long long *bnd = h->seg_scratch, *big = bnd + nbe,
                                       *nbig = big + 2 * nbe;
                    KM_CUDA(radix_pass(h->dlist, h->alt0, D[i], h->kw, s0, h->sort_scratch, st));
                    KM_CUDA(radix_pass(h->alt0, h->alt1, D[i], h->kw, s0 + 8, h->sort_scratch, st));
                    KM_CUDA(radix_pass(h->alt1, h->alt0, D[i], h->kw, s0 + 16, h->sort_scratch,
                                       st));
                    KM_CUDA(top_segment_sort(h->alt0, D[i], h->kw, bits, bnd, big, nbig, st));
                    KM_CUDA(big_segment_sort(h->alt0, h->alt1, D[i], h->kw, bits, big, nbig, st));
                    sorted = h->alt0;
                    n_launch += 12;
                } else {
                    KM_CUDA(radix_sort(h->dlist, h->alt0, h->alt1, D[i], h->kw, bits,
                                       h->sort_scratch, &sorted, st));
                    n_launch += D[i] > 1 ? 3 * (uint64_t)passes : 0;
                }
                KM_CUDA(launch_classify_query(sorted, D[i], h->kw, h->G, h->tau, h->est, st));
                KM_CUDA(launch_split(sorted, h->est, D[i], h->kw, h->tau, h->split,
                                     h->split_scratch, h->ctr, st));
                h->launches += n_launch;
                b->launches += n_launch;
                h->sorted = sorted;
                h->n_distinct = D[i];
                b->cls_sorted[i] = sorted;
            }
            for (int k = 0; k < kBatchStreams; ++k) {
                KM_CUDA(cudaEventRecord(b->join[k], b->aux[k]));
                KM_CUDA(cudaStreamWaitEvent(b->stream, b->join[k], 0));
            }
            return KMERCO_OK;
        };
        st_launch = go();
        if (capture) {
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
            if (st_launch != KMERCO_OK) {
                if (g) cudaGraphDestroy(g);
                return st_launch;
            }
            KM_CUDA(ec);
            if (cudaGraphInstantiate(&b->cls_exec, g, 0) != cudaSuccess) {
                cudaGraphDestroy(g);
                return KMERCO_ECUDA;
            }
            b->cls_graph = g;
            b->have_cls = true;
            b->cls_key = key;
            b->cls_launches = b->launches - l0;
            KM_CUDA(cudaGraphLaunch(b->cls_exec, b->stream));
        } else if (st_launch != KMERCO_OK) {
            return st_launch;
        }
    }
    // one readback of every sample's trustworthy count and, for the samples
    // sorted by their top bits, of the count of runs too long for one block
    for (int i = 0; i < b->n; ++i) {
        kmerco_t *h = b->h[i];
        KM_CUDA(cudaMemcpyAsync(h->ctr_host, h->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                                b->stream));
        if (top[i]) {
            const uint64_t nbe = seg_bounds_entries(D[i], h->kw);
            KM_CUDA(cudaMemcpyAsync(h->bucket_host, h->seg_scratch + 3 * nbe, 8,
                                    cudaMemcpyDeviceToHost, b->stream));
        }
    }
    KM_CUDA(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i) {
        kmerco_t *h = b->h[i];
        if (!top[i] || !h->bucket_host[0]) continue;
        // a run of equal top bits beyond one block (at most D / 2^22 of them):
        // sort it, then split the sample again
        bool any;
        KM_TRY(sort_long_runs(h, D[i], 2 * h->K, h->bucket_host[0], &any, b->stream));
        if (!any) continue;
        KM_CUDA(launch_classify_query(h->alt0, D[i], h->kw, h->G, h->tau, h->est, b->stream));
        KM_CUDA(launch_split(h->alt0, h->est, D[i], h->kw, h->tau, h->split, h->split_scratch,
                             h->ctr, b->stream));
        h->launches += 4;
        b->launches += 4;
        KM_CUDA(cudaMemcpyAsync(h->ctr_host, h->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost,
                                b->stream));
        KM_CUDA(cudaStreamSynchronize(b->stream));
    }
    for (kmerco_t *h : b->h) {
        if (h->classified) continue;
        h->n_trusted = h->ctr_host->trusted;
        h->classified = true;
        h->est_exact = false;
        h->classify_timed = false;
    }
    return KMERCO_OK;
}

int kmerco_batch_info(kmerco_batch_t *b, kmerco_batch_info_t *info) {
    if (!b || !info) return KMERCO_EINVAL;
    memset(info, 0, sizeof(*info));
    info->samples = b->n;
    info->chunk = b->chunk;
    info->blocks_per_sm = b->bpm;
    info->tuned = b->tuned ? 1 : 0;
    info->tuned_ms = b->tuned_ms;
    info->graph = b->have_graph ? 1 : 0;
    info->launches = b->launches;
    info->total_chunks = b->total_chunks;
    info->schedule = b->sched;
    info->streams = b->sched == 1 ? b->streams : 0;
    return KMERCO_OK;
}

}  // extern "C"

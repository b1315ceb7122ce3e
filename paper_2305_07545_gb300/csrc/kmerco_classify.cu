// Classification phase of KmerCo (Algorithm 2 with QcountBF-II, Algorithm 5)
// and the countBF merge, on sm_103a.
//
//  - radix_sort: least-significant-digit radix sort of the distinct keys
//    (8-bit digits, only the 2K bits a key can use).  Per pass: per-tile
//    digit counts, one scan per digit across tiles, then a stable scatter
//    in which each warp ranks equal digits with one ballot per digit bit and the
//    tile is reordered in shared memory before coalesced stores.
//  - bucket_sort (one-word keys, up to ~1.3e8): a histogram of the top 16
//    key bits, adjacent bins merged on the host into super-buckets of at
//    most kBucketCap keys, one scatter pass, then each super-bucket sorted
//    in shared memory by one block (counting sort on 12 more bits, then
//    insertion or bitonic sort).  A single bin too large for shared memory
//    is left to radix_sort.
//  - query: per key, k_h hashes and the minimum counter, 0 if any is 0.
//  - split: stable partition on est > tau (trustworthy first).
//  - merge: counter-wise min(a + b, 2^alpha - 1) of two countBFs.
#include "kmerco_internal.cuh"

namespace countbf {
namespace {

constexpr int kWarps = kSortThreads / 32;

// The 8-bit digit at bit `shift` of a key (a digit may straddle the two
// words of a two-word key).
template <int KW>
__device__ __forceinline__ unsigned digit_of(const uint64_t *k, int shift) {
    if (KW == 1 || shift + kRadixBits <= 64) return (unsigned)(k[0] >> shift) & (kRadixBins - 1);
    if (shift >= 64) return (unsigned)(k[1] >> (shift - 64)) & (kRadixBins - 1);
    return (unsigned)((k[0] >> shift) | (k[1] << (64 - shift))) & (kRadixBins - 1);
}

// Bits [s, s + 64) of a key of KW words, as one word (0 <= s < 64 * KW).
template <int KW>
__device__ __forceinline__ uint64_t bits_from(const uint64_t *k, int s) {
    if (KW == 1 || s == 0) return k[0] >> s;
    if (s >= 64) return k[1] >> (s - 64);
    return (k[0] >> s) | (k[1] << (64 - s));
}

// a < b for keys of KW words (two-word keys compare high word first).
template <int KW>
__device__ __forceinline__ bool key_less(const uint64_t *a, const uint64_t *b) {
    if (KW == 1) return a[0] < b[0];
    return a[1] < b[1] || (a[1] == b[1] && a[0] < b[0]);
}

template <int KW>
__host__ __device__ constexpr int tile_keys() { return kSortThreads * (kSortItems / KW); }

// counts[d * ntiles + tile] = keys of the tile with digit d.
template <int KW>
__global__ void __launch_bounds__(kSortThreads) upsweep_kernel(const uint64_t *in, uint64_t n,
                                                               int shift, uint32_t *counts,
                                                               uint32_t ntiles) {
    __shared__ unsigned hist[kRadixBins];
    const int tid = threadIdx.x;
    hist[tid] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * tile_keys<KW>();
#pragma unroll 4
    for (int j = 0; j < kSortItems / KW; ++j) {
        uint64_t idx = base + (uint64_t)j * kSortThreads + tid;
        if (idx < n) atomicAdd(&hist[digit_of<KW>(in + idx * KW, shift)], 1u);
    }
    __syncthreads();
    counts[(uint64_t)tid * ntiles + blockIdx.x] = hist[tid];
}

// Row d of counts becomes its exclusive prefix over tiles; totals[d] = row sum.
__global__ void __launch_bounds__(kSortThreads) scan_rows_kernel(uint32_t *counts, uint32_t ntiles,
                                                                 uint32_t *totals) {
    uint32_t *row = counts + (uint64_t)blockIdx.x * ntiles;
    uint32_t carry = 0;
    for (uint32_t s0 = 0; s0 < ntiles; s0 += kSortThreads * 4) {
        uint32_t v[4], sum = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t idx = s0 + threadIdx.x * 4 + j;
            v[j] = idx < ntiles ? row[idx] : 0u;
            sum += v[j];
        }
        uint32_t tot;
        uint32_t pre = block_exclusive_scan<uint32_t, kSortThreads>(sum, tot) + carry;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t idx = s0 + threadIdx.x * 4 + j;
            if (idx < ntiles) row[idx] = pre;
            pre += v[j];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// The scatter of one pass: the same tiles as upsweep_kernel.  One-word keys
// take 512 threads, 8 keys each (two blocks of 16 warps fit an SM's
// registers; 256 threads x 16 keys needed 118 registers); two-word keys
// take 256 threads, 8 keys each, which measured faster than 512 x 4.
template <int KW>
__host__ __device__ constexpr int down_threads() { return KW == 1 ? 512 : 256; }

template <int KW>
__global__ void __launch_bounds__(down_threads<KW>(), KW == 1 ? 2 : 3) downsweep_kernel(
    const uint64_t *in, uint64_t *out, uint64_t n, int shift, const uint32_t *counts,
    const uint32_t *totals, uint32_t ntiles) {
    constexpr int NT = down_threads<KW>();
    constexpr int TILE = tile_keys<KW>();
    constexpr int ITEMS = TILE / NT;
    constexpr int NW = NT / 32;
    static_assert(kRadixBins <= NT, "one thread per digit");
    __shared__ uint16_t wcnt[NW][kRadixBins];   // a tile's counts and offsets stay below 2^16
    __shared__ uint32_t tstart[kRadixBins];
    __shared__ uint64_t gofs[kRadixBins];
    __shared__ uint64_t stage[TILE * KW];
    static_assert(TILE < 65536, "16-bit warp counts");

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t tile_base = (uint64_t)blockIdx.x * TILE;
    for (int d = lane; d < kRadixBins; d += 32) wcnt[warp][d] = 0;

    uint64_t key[ITEMS][KW];
    unsigned dig[ITEMS], rank[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        uint64_t idx = tile_base + (uint64_t)warp * (32 * ITEMS) + j * 32 + lane;
        if (idx < n) {
#pragma unroll
            for (int w = 0; w < KW; ++w) key[j][w] = in[idx * KW + w];
            dig[j] = digit_of<KW>(key[j], shift);
        } else {
#pragma unroll
            for (int w = 0; w < KW; ++w) key[j][w] = 0;
            dig[j] = kRadixBins - 1;   // past the end: ranked last, never stored
        }
    }
    __syncwarp();
    // stable rank within the warp: items in (j, lane) order
    const unsigned lt = (1u << lane) - 1;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        // lanes holding the same digit: one ballot per digit bit
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < kRadixBits; ++b) {
            const bool bit = (dig[j] >> b) & 1u;
            const unsigned bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
        const unsigned prev = wcnt[warp][dig[j]];
        __syncwarp();
        if (lane == __ffs(peers) - 1) wcnt[warp][dig[j]] = (uint16_t)(prev + __popc(peers));
        __syncwarp();
        rank[j] = prev + __popc(peers & lt);
    }
    __syncthreads();

    // per digit: offsets of each warp within the tile, tile start of the digit
    {
        const int d = tid;
        uint32_t run = 0;
        uint64_t t64 = 0;
        if (d < kRadixBins) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                uint32_t c = wcnt[w][d];
                wcnt[w][d] = (uint16_t)run;
                run += c;
            }
            t64 = totals[d];
        }
        uint32_t tot;
        const uint32_t ts = block_exclusive_scan<uint32_t, NT>(run, tot);
        uint64_t dtot;
        const uint64_t dbase = block_exclusive_scan<uint64_t, NT>(t64, dtot);
        if (d < kRadixBins) {
            tstart[d] = ts;
            gofs[d] = dbase + counts[(uint64_t)d * ntiles + blockIdx.x];
        }
    }
    __syncthreads();

#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        uint64_t idx = tile_base + (uint64_t)warp * (32 * ITEMS) + j * 32 + lane;
        if (idx < n) {
            const unsigned pos = tstart[dig[j]] + wcnt[warp][dig[j]] + rank[j];
#pragma unroll
            for (int w = 0; w < KW; ++w) stage[pos * KW + w] = key[j][w];
        }
    }
    __syncthreads();

    const uint64_t left = n - tile_base;
    const unsigned valid = left < (uint64_t)TILE ? (unsigned)left : (unsigned)TILE;
    for (unsigned i = tid; i < valid; i += NT) {
        const unsigned d = digit_of<KW>(stage + i * KW, shift);
        const uint64_t o = gofs[d] + (i - tstart[d]);
#pragma unroll
        for (int w = 0; w < KW; ++w) out[o * KW + w] = stage[i * KW + w];
    }
}

// QcountBF-II (Algorithm 5) per key.
template <int KW>
__global__ void query_kernel(const uint64_t *keys, uint64_t n, int K, Geometry G, uint32_t *est) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t klo = keys[i * KW];
        const uint64_t khi = KW == 2 ? keys[i * KW + 1] : 0;
        const uint64_t k1m = KW == 1 ? premix8(klo) : 0;
        // k_h counters in groups of four, the four loads in flight together;
        // the minimum, or 0 as soon as one counter is 0 (Algorithm 5)
        uint64_t best = ~0ull;
        for (int a0 = 0; a0 < G.nhash && best; a0 += 4) {
            uint64_t cell[4], word[4];
            unsigned sh[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                cell[j] = 0;
                sh[j] = 0;
                if (a0 + j < G.nhash) {
                    uint64_t h1, h2;
                    if (KW == 1)
                        murmur8(k1m, (uint32_t)(a0 + j), h1, h2);
                    else
                        murmur16(klo, khi, (uint32_t)(a0 + j), h1, h2);
                    unsigned slot;
                    address(G, h1, cell[j], slot);
                    sh[j] = slot * (unsigned)G.alpha;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (a0 + j < G.nhash) word[j] = __ldg(G.cells + cell[j]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (a0 + j < G.nhash) {
                    const uint64_t v = (word[j] >> sh[j]) & G.maxc;
                    best = v < best ? v : best;
                }
            }
        }
        est[i] = (uint32_t)best;
        (void)K;
    }
}

// Algorithm 5 as far as Algorithm 2 needs it.  The split asks only whether
// est > tau, and est is the minimum of the key's k_h counters, so the first
// counter at or below tau decides "erroneous": the remaining counters of that
// key are not read.  est[i] is then exact for every trustworthy key (all k_h
// counters read) and, for an erroneous key, the minimum of the counters read
// so far, which is at most tau; Algorithm 5's 0 for an empty counter is that
// minimum too.  Each lane works through its keys one counter per iteration
// (a finished key makes room for the lane's next key at once), so every
// iteration keeps one random counter read per lane in flight.
template <int KW>
__global__ void __launch_bounds__(256) classify_query_kernel(const uint64_t *keys, uint64_t n,
                                                             Geometry G, uint32_t tau,
                                                             uint32_t *est) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t klo = keys[i * KW], khi = KW == 2 ? keys[i * KW + 1] : 0;
    uint64_t k1m = KW == 1 ? premix8(klo) : 0;
    unsigned j = 0;
    uint64_t best = ~0ull;
    for (;;) {
        uint64_t h1, h2, cell;
        unsigned slot;
        if (KW == 1)
            murmur8(k1m, j, h1, h2);
        else
            murmur16(klo, khi, j, h1, h2);
        address(G, h1, cell, slot);
        const uint64_t v = (__ldg(G.cells + cell) >> (slot * (unsigned)G.alpha)) & G.maxc;
        best = v < best ? v : best;
        if (++j < (unsigned)G.nhash && best > tau) continue;
        est[i] = (uint32_t)best;
        i += stride;
        if (i >= n) break;
        klo = keys[i * KW];
        khi = KW == 2 ? keys[i * KW + 1] : 0;
        k1m = KW == 1 ? premix8(klo) : 0;
        j = 0;
        best = ~0ull;
    }
}

// Trusted keys per split tile.  A tile of kSplitTile keys is read in 16
// rounds of kSortThreads consecutive keys (coalesced), key tile0 + 256j + tid.
__global__ void __launch_bounds__(kSortThreads) split_count_kernel(const uint32_t *est, uint64_t n,
                                                                   uint32_t tau, uint64_t *tile_cnt) {
    const uint64_t tile0 = (uint64_t)blockIdx.x * kSplitTile;
    unsigned c = 0;
#pragma unroll
    for (int j = 0; j < kSplitTile / kSortThreads; ++j) {
        const uint64_t i = tile0 + (uint64_t)j * kSortThreads + threadIdx.x;
        c += (i < n) && est[i] > tau;
    }
    unsigned long long tot;
    block_exclusive_scan<unsigned long long, kSortThreads>(c, tot);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = tot;
}

// Exclusive scan of tile counts in place (one block); total -> ctr->trusted.
__global__ void __launch_bounds__(kSortThreads) split_scan_kernel(uint64_t *tile_cnt,
                                                                  uint64_t ntiles, DevCounters *ctr) {
    unsigned long long carry = 0;
    for (uint64_t s0 = 0; s0 < ntiles; s0 += kSortThreads) {
        const uint64_t idx = s0 + threadIdx.x;
        unsigned long long v = idx < ntiles ? tile_cnt[idx] : 0ull, tot;
        unsigned long long pre = block_exclusive_scan<unsigned long long, kSortThreads>(v, tot) + carry;
        if (idx < ntiles) tile_cnt[idx] = pre;
        carry += tot;
    }
    if (threadIdx.x == 0) ctr->trusted = carry;
}

// Stable split of one tile: trustworthy keys (est > tau) go after the
// trustworthy keys of earlier tiles, erroneous keys after all trustworthy
// keys and the erroneous keys of earlier tiles, both in key order.  The tile
// is read in 16 coalesced rounds; a key's rank comes from its warp's ballot
// and the counts of the (round, warp) segments before it.
template <int KW>
__global__ void __launch_bounds__(kSortThreads) split_scatter_kernel(const uint64_t *keys,
                                                                     const uint32_t *est, uint64_t n,
                                                                     uint32_t tau,
                                                                     const uint64_t *tile_pre,
                                                                     const DevCounters *ctr,
                                                                     uint64_t *out) {
    constexpr int kRounds = kSplitTile / kSortThreads;
    __shared__ unsigned seg[kRounds * kWarps];   // trusted keys per (round, warp), then their prefix
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t tile0 = (uint64_t)blockIdx.x * kSplitTile;
    unsigned bal[kRounds];
#pragma unroll
    for (int j = 0; j < kRounds; ++j) {
        const uint64_t i = tile0 + (uint64_t)j * kSortThreads + threadIdx.x;
        bal[j] = __ballot_sync(0xffffffffu, i < n && est[i] > tau);
        if (lane == 0) seg[j * kWarps + warp] = __popc(bal[j]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // segments in key order: round-major, then warp
        unsigned acc = 0;
        for (int q = 0; q < kRounds * kWarps; ++q) {
            const unsigned v = seg[q];
            seg[q] = acc;
            acc += v;
        }
    }
    __syncthreads();
    const uint64_t T = ctr->trusted;
    const uint64_t tpre = tile_pre[blockIdx.x];   // trusted keys before this tile
    const unsigned lt = (1u << lane) - 1;
#pragma unroll
    for (int j = 0; j < kRounds; ++j) {
        const uint64_t i = tile0 + (uint64_t)j * kSortThreads + threadIdx.x;
        if (i >= n) continue;
        const uint64_t off = i - tile0;   // keys of the tile before this one
        const uint64_t tr_before = seg[j * kWarps + warp] + __popc(bal[j] & lt);
        const uint64_t o = (bal[j] >> lane) & 1u ? tpre + tr_before
                                                : T + (tile0 - tpre) + (off - tr_before);
#pragma unroll
        for (int w = 0; w < KW; ++w) out[o * KW + w] = keys[i * KW + w];
    }
}

// dst = counter-wise min(dst + src, 2^alpha - 1)
__global__ void merge_kernel(uint64_t *dst, const uint64_t *src, Geometry G) {
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < G.words;
         w += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = dst[w], b = src[w];
        uint64_t r = 0;
        for (int l = 0; l < G.eta; ++l) {
            const unsigned sh = (unsigned)(l * G.alpha);
            uint64_t s = ((a >> sh) & G.maxc) + ((b >> sh) & G.maxc);
            if (s > G.maxc) s = G.maxc;
            r |= s << sh;
        }
        dst[w] = r;
    }
}

__global__ void count_saturated_kernel(Geometry G, DevCounters *ctr) {
    unsigned long long c = 0;
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < G.words;
         w += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = G.cells[w];
        for (int l = 0; l < G.eta; ++l) c += ((v >> (unsigned)(l * G.alpha)) & G.maxc) == G.maxc;
    }
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&ctr->saturated, c);
}

// ---------------------------------------------------------------- bucket sort
// Partial histograms of key >> shift over kHistBins bins: block b counts the
// keys of its tile (at most 65,535) in 16-bit shared counters and writes them
// to partial[b * kHistBins ...].
__global__ void __launch_bounds__(512) bucket_hist_kernel(const uint64_t *keys, uint64_t n,
                                                          int shift, unsigned short *partial) {
    extern __shared__ unsigned hh32[];   // kHistBins 16-bit counters, two per word
    unsigned short *hh = (unsigned short *)hh32;
    for (unsigned i = threadIdx.x; i < kHistBins / 2; i += blockDim.x) hh32[i] = 0;
    __syncthreads();
    const uint64_t t0 = (uint64_t)blockIdx.x * kHistTile;
    const unsigned cnt = (unsigned)min((uint64_t)kHistTile, n - t0);
    for (unsigned i = threadIdx.x; i < cnt; i += blockDim.x) {
        const unsigned b = (unsigned)(keys[t0 + i] >> shift);
        atomicAdd(&hh32[b >> 1], 1u << (16 * (b & 1)));   // a 16-bit lane never exceeds 65,535
    }
    __syncthreads();
    unsigned short *out = partial + (uint64_t)blockIdx.x * kHistBins;
    for (unsigned i = threadIdx.x; i < kHistBins; i += blockDim.x) out[i] = hh[i];
}

// hist[i] = sum over blocks of partial[b][i].
__global__ void bucket_hist_reduce_kernel(const unsigned short *partial, unsigned nblocks,
                                          unsigned *hist) {
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kHistBins) return;
    unsigned s = 0;
    for (unsigned b = 0; b < nblocks; ++b) s += partial[(uint64_t)b * kHistBins + i];
    hist[i] = s;
}

// One tile of keys per block: count per super-bucket, reserve each
// super-bucket's run with one global atomic, then place the keys (order
// within a super-bucket is arbitrary; each is sorted afterwards).  Keys are
// read eight per thread at a time so that the loads overlap.
__global__ void __launch_bounds__(256) bucket_scatter_kernel(const uint64_t *keys, uint64_t n,
                                                             int shift, const unsigned *map,
                                                             unsigned nsuper,
                                                             unsigned long long *cursor,
                                                             uint64_t *out) {
    extern __shared__ unsigned sc[];
    unsigned *h = sc, *base = sc + nsuper;
    const uint64_t t0 = (uint64_t)blockIdx.x * kScatterTile;
    const unsigned cnt = (unsigned)min((uint64_t)kScatterTile, n - t0);
    for (unsigned i = threadIdx.x; i < nsuper; i += blockDim.x) h[i] = 0;
    __syncthreads();
    constexpr unsigned kB = 8, kStride = 256;
    for (unsigned i0 = 0; i0 < cnt; i0 += kB * kStride) {
        uint64_t k[kB];
#pragma unroll
        for (unsigned q = 0; q < kB; ++q) {
            const unsigned i = i0 + q * kStride + threadIdx.x;
            k[q] = i < cnt ? __ldg(keys + t0 + i) : 0;
        }
#pragma unroll
        for (unsigned q = 0; q < kB; ++q)
            if (i0 + q * kStride + threadIdx.x < cnt) atomicAdd(&h[__ldg(map + (k[q] >> shift))], 1u);
    }
    __syncthreads();
    for (unsigned b = threadIdx.x; b < nsuper; b += blockDim.x) {
        if (h[b]) base[b] = (unsigned)atomicAdd(cursor + b, (unsigned long long)h[b]);
        h[b] = 0;
    }
    __syncthreads();
    for (unsigned i0 = 0; i0 < cnt; i0 += kB * kStride) {
        uint64_t k[kB];
#pragma unroll
        for (unsigned q = 0; q < kB; ++q) {
            const unsigned i = i0 + q * kStride + threadIdx.x;
            k[q] = i < cnt ? __ldg(keys + t0 + i) : 0;
        }
#pragma unroll
        for (unsigned q = 0; q < kB; ++q) {
            if (i0 + q * kStride + threadIdx.x < cnt) {
                const unsigned b = __ldg(map + (k[q] >> shift));
                out[base[b] + atomicAdd(&h[b], 1u)] = k[q];
            }
        }
    }
}

// The same placement with the tile's keys first grouped by super-bucket in
// shared memory, so that each super-bucket's keys of the tile leave as one
// contiguous run (coalesced stores).  For at most kSortedScatterMax
// super-buckets; the tile is kSortedScatterTile keys, 1,024 threads.
constexpr int kSortedScatterTile = 16384;
constexpr int kSortedScatterMax = 4096;

__global__ void __launch_bounds__(1024) bucket_scatter_sorted_kernel(
    const uint64_t *keys, uint64_t n, int shift, const unsigned *map, unsigned nsuper,
    unsigned long long *cursor, uint64_t *out) {
    extern __shared__ unsigned long long ss[];
    uint64_t *tile = (uint64_t *)ss;
    unsigned *h = (unsigned *)(ss + kSortedScatterTile);
    unsigned *lst = h + nsuper, *fill = lst + nsuper, *base = fill + nsuper;
    constexpr unsigned kT = 1024, kPer = kSortedScatterTile / kT;
    const uint64_t t0 = (uint64_t)blockIdx.x * kSortedScatterTile;
    const unsigned cnt = (unsigned)min((uint64_t)kSortedScatterTile, n - t0);
    const unsigned tid = threadIdx.x;
    for (unsigned i = tid; i < nsuper; i += kT) {
        h[i] = 0;
        fill[i] = 0;
    }
    __syncthreads();
    uint64_t k[kPer];
    unsigned bk[kPer];
#pragma unroll
    for (unsigned q = 0; q < kPer; ++q) {
        const unsigned i = q * kT + tid;
        k[q] = i < cnt ? __ldg(keys + t0 + i) : 0;
    }
#pragma unroll
    for (unsigned q = 0; q < kPer; ++q) {
        bk[q] = __ldg(map + (k[q] >> shift));
        if (q * kT + tid < cnt) atomicAdd(&h[bk[q]], 1u);
    }
    __syncthreads();
    // tile-local starts (exclusive scan of h, a run of entries per thread)
    // and one global reservation per super-bucket present in the tile
    {
        const unsigned per = (nsuper + kT - 1) / kT, b0 = tid * per;
        unsigned sum = 0;
        for (unsigned j = 0; j < per && b0 + j < nsuper; ++j) sum += h[b0 + j];
        unsigned tot;
        unsigned pre = block_exclusive_scan<unsigned, kT>(sum, tot);
        for (unsigned j = 0; j < per && b0 + j < nsuper; ++j) {
            const unsigned b = b0 + j, m = h[b];
            lst[b] = pre;
            pre += m;
            if (m) base[b] = (unsigned)atomicAdd(cursor + b, (unsigned long long)m);
        }
    }
    __syncthreads();
#pragma unroll
    for (unsigned q = 0; q < kPer; ++q)
        if (q * kT + tid < cnt) tile[lst[bk[q]] + atomicAdd(&fill[bk[q]], 1u)] = k[q];
    __syncthreads();
    for (unsigned i = tid; i < cnt; i += kT) {
        const uint64_t key = tile[i];
        const unsigned b = __ldg(map + (key >> shift));
        out[base[b] + (i - lst[b])] = key;
    }
}

// Sort of one super-bucket (at most kBucketCap keys) in shared memory: a
// counting sort on the 12 bits below the super-bucket's common range
// (sub = (key - lo) >> rsh), then an insertion sort of each small
// sub-bucket.  When the keys cluster so that a sub-bucket holds more than
// kSubMax keys, the block bitonic-sorts the whole super-bucket instead.
__global__ void __launch_bounds__(kBucketThreads, 2) bucket_sort_kernel(
    uint64_t *data, const unsigned long long *start, const unsigned long long *lo,
    const int *rsh) {
    extern __shared__ unsigned long long sm[];
    unsigned long long *B = sm;   // the keys stay in registers until placed here
    unsigned *hist = (unsigned *)(sm + kBucketCap);
    unsigned *st = hist + kSubBins, *fill = st + kSubBins;
    constexpr unsigned kPer = kBucketCap / kBucketThreads;
    __shared__ unsigned maxsub;
    const unsigned long long s0 = start[blockIdx.x];
    const unsigned n = (unsigned)(start[blockIdx.x + 1] - s0);
    if (n <= 1 || n > (unsigned)kBucketCap) return;
    const unsigned long long base = lo[blockIdx.x];
    const int r = rsh[blockIdx.x];
    const unsigned tid = threadIdx.x;
    for (unsigned i = tid; i < kSubBins; i += kBucketThreads) hist[i] = 0;
    if (tid == 0) maxsub = 0;
    __syncthreads();
    unsigned long long key[kPer];
#pragma unroll
    for (unsigned q = 0; q < kPer; ++q) {
        const unsigned i = q * kBucketThreads + tid;
        key[q] = i < n ? data[s0 + i] : 0ull;
        if (i < n) atomicAdd(&hist[min((unsigned)((key[q] - base) >> r), (unsigned)kSubBins - 1)], 1u);
    }
    __syncthreads();
    // exclusive scan of the kSubBins counts: 4 per thread
    {
        unsigned v[4], sum = 0, mx = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = hist[tid * 4 + j];
            sum += v[j];
            mx = max(mx, v[j]);
        }
        unsigned tot;
        unsigned pre = block_exclusive_scan<unsigned, kBucketThreads>(sum, tot);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            st[tid * 4 + j] = pre;
            fill[tid * 4 + j] = pre;
            pre += v[j];
        }
        atomicMax(&maxsub, mx);
    }
    __syncthreads();
#pragma unroll
    for (unsigned q = 0; q < kPer; ++q) {
        if (q * kBucketThreads + tid < n) {
            const unsigned long long k = key[q];
            B[atomicAdd(&fill[min((unsigned)((k - base) >> r), (unsigned)kSubBins - 1)], 1u)] = k;
        }
    }
    __syncthreads();
    if (maxsub <= (unsigned)kSubMax) {
        for (unsigned b = tid; b < kSubBins; b += kBucketThreads) {
            const unsigned a0 = st[b], m = hist[b];
            for (unsigned i = 1; i < m; ++i) {
                const unsigned long long k = B[a0 + i];
                unsigned j = i;
                while (j > 0 && B[a0 + j - 1] > k) {
                    B[a0 + j] = B[a0 + j - 1];
                    --j;
                }
                B[a0 + j] = k;
            }
        }
    } else {
        unsigned P = 2;
        while (P < n) P <<= 1;
        for (unsigned i = n + tid; i < P; i += kBucketThreads) B[i] = ~0ull;
        __syncthreads();
        for (unsigned k = 2; k <= P; k <<= 1) {
            for (unsigned j = k >> 1; j > 0; j >>= 1) {
                for (unsigned i = tid; i < P; i += kBucketThreads) {
                    const unsigned ixj = i ^ j;
                    if (ixj > i) {
                        const unsigned long long a = B[i], b = B[ixj];
                        if ((a > b) == ((i & k) == 0)) {
                            B[i] = b;
                            B[ixj] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
    }
    __syncthreads();
    for (unsigned i = tid; i < n; i += kBucketThreads) data[s0 + i] = B[i];
}

// ------------------------------------------------------ top-bits + segments
// Sort of a large key set in two steps.  Three stable radix passes on the
// top kTopBits key bits order the keys by those bits; the array is then cut
// into segments that begin where the top bits change, near every multiple
// of half a segment's capacity, and each segment is sorted in shared memory
// (a counting sort on 12 more bits, then an insertion or bitonic sort with
// the whole key as the comparison).  A segment too large for shared memory
// (one run of equal top bits longer than that) is listed for a radix sort of
// its own.
constexpr int kTopBits = kTopSortBits;
constexpr unsigned kRankMax = 256;   // largest sub-bin rank-sorted in a segment
constexpr unsigned kMaxLarge = 8;     // larger sub-bins sorted one by one; more: the whole segment

template <int KW>
__host__ __device__ constexpr int seg_cap() { return KW == 1 ? kBucketCap : kBucketCap / 2; }

// Top kTopBits bits of a key of `bits` bits.
template <int KW>
__device__ __forceinline__ uint32_t top_bits(const uint64_t *k, int bits) {
    return (uint32_t)(bits_from<KW>(k, bits - kTopBits) & ((1u << kTopBits) - 1));
}

// b[j], j < nb: the first index at or after j * H where the top bits differ
// from those of key j * H - 1 (b[0] = 0, and n once past the end), by a
// binary search over the keys sorted by their top bits.
template <int KW>
__global__ void seg_bounds_kernel(const uint64_t *keys, uint64_t n, int bits, uint64_t H,
                                  uint64_t nb, unsigned long long *b) {
    const uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (j >= nb) return;
    const uint64_t at = j * H;
    if (j == 0 || at >= n) {
        b[j] = j == 0 ? 0 : n;
        return;
    }
    const uint32_t t = top_bits<KW>(keys + (at - 1) * KW, bits);
    uint64_t lo = at, hi = n;   // the answer is in [lo, hi]
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (top_bits<KW>(keys + mid * KW, bits) > t)
            hi = mid;
        else
            lo = mid + 1;
    }
    b[j] = lo;
}

// Segment j = [b[j], b[j + 1]) of `data` sorted in place by one block.
// Segments above seg_cap<KW>() keys go to the `big` list (begin, count)
// instead; nbig counts them.  The keys are loaded before anything else: the
// segment's top-bit range comes from its first and last key as loaded.
// Each key's sub-bin is computed once and kept beside it in shared memory.
template <int KW>
__device__ __forceinline__ unsigned rank_in_subbin(const uint64_t *B, unsigned a0, unsigned m,
                                                   const uint64_t *k) {
    unsigned r = 0;
    if (KW == 1) {
        for (unsigned j = a0; j < a0 + m; ++j) r += B[j] < k[0] ? 1u : 0u;
    } else {   // one 16-byte shared load per key: x the low word, y the high word
        const ulonglong2 *B2 = (const ulonglong2 *)B;
        for (unsigned j = a0; j < a0 + m; ++j) {
            const ulonglong2 v = B2[j];
            r += (v.y < k[1] || (v.y == k[1] && v.x < k[0])) ? 1u : 0u;
        }
    }
    return r;
}

template <int KW>
__global__ void __launch_bounds__(kBucketThreads, 2) segment_sort_kernel(
    uint64_t *data, int bits, const unsigned long long *b, unsigned long long *big,
    unsigned long long *nbig) {
    constexpr int C = seg_cap<KW>();
    constexpr unsigned kPer = C / kBucketThreads;
    extern __shared__ __align__(16) unsigned long long sm[];
    uint64_t *B = (uint64_t *)sm;                  // C keys of KW words
    unsigned *cnt = (unsigned *)(sm + C * KW);     // per sub-bin: count, then fill cursor
    unsigned *st = cnt + kSubBins;                 // per sub-bin: first place
    uint16_t *SB = (uint16_t *)(st + kSubBins);    // sub-bin of the key at B[i]
    __shared__ unsigned maxsub, nlarge;
    __shared__ unsigned large[kMaxLarge];   // sub-bins above kRankMax keys
    __shared__ uint32_t tops[2];            // top bits of the first and the last key
    const uint64_t s0 = b[blockIdx.x], e0 = b[blockIdx.x + 1];
    if (e0 <= s0 + 1) return;   // empty or one key
    const uint64_t nn = e0 - s0;
    if (nn > (uint64_t)C) {
        if (threadIdx.x == 0) {
            const unsigned long long q = atomicAdd(nbig, 1ull);
            big[2 * q] = s0;
            big[2 * q + 1] = nn;
        }
        return;
    }
    const unsigned n = (unsigned)nn;
    const unsigned tid = threadIdx.x;
    uint64_t key[kPer][KW];
#pragma unroll
    for (unsigned q = 0; q < kPer; ++q) {
        const unsigned i = q * kBucketThreads + tid;
#pragma unroll
        for (int w = 0; w < KW; ++w) key[q][w] = i < n ? data[(s0 + i) * KW + w] : 0ull;
    }
    for (unsigned i = tid; i < kSubBins; i += kBucketThreads) cnt[i] = 0;
    if (tid == 0) {
        maxsub = 0;
        nlarge = 0;
        tops[0] = top_bits<KW>(key[0], bits);
    }
#pragma unroll
    for (unsigned q = 0; q < kPer; ++q)
        if (q * kBucketThreads + tid == n - 1) tops[1] = top_bits<KW>(key[q], bits);
    __syncthreads();
    // the segment's top-bit range [t0, t1] maps onto kSubBins sub-bins of
    // the key's top min(bits, 64) bits
    const int pb = bits < 64 ? bits : 64;
    const uint32_t t0 = tops[0], t1 = tops[1];
    const int below = pb - kTopBits;                      // prefix bits under the top bits
    int span = 0;
    while ((1ull << span) < (uint64_t)(t1 - t0 + 1)) ++span;
    int r = span + below - 12;
    if (r < 0) r = 0;
    const uint64_t base = (uint64_t)t0 << below;
    // sub-bin of a key (computed again for the scatter: registers hold the keys)
    auto sub_of = [&](const uint64_t *k) {
        return (unsigned)min((bits_from<KW>(k, bits - pb) - base) >> r, (uint64_t)kSubBins - 1);
    };
#pragma unroll
    for (unsigned q = 0; q < kPer; ++q)
        if (q * kBucketThreads + tid < n) atomicAdd(&cnt[sub_of(key[q])], 1u);
    __syncthreads();
    {
        unsigned v[4], sum = 0, mx = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = cnt[tid * 4 + j];
            sum += v[j];
            mx = max(mx, v[j]);
        }
        unsigned tot;
        unsigned pre = block_exclusive_scan<unsigned, kBucketThreads>(sum, tot);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            st[tid * 4 + j] = pre;
            cnt[tid * 4 + j] = pre;   // fill cursor; after the scatter, the sub-bin's end
            pre += v[j];
            if (v[j] > kRankMax) {
                const unsigned q = atomicAdd(&nlarge, 1u);
                if (q < kMaxLarge) large[q] = tid * 4 + j;
            }
        }
        atomicMax(&maxsub, mx);
    }
    __syncthreads();
#pragma unroll
    for (unsigned q = 0; q < kPer; ++q) {
        if (q * kBucketThreads + tid < n) {
            const unsigned bin = sub_of(key[q]);
            const unsigned at = atomicAdd(&cnt[bin], 1u);
#pragma unroll
            for (int w = 0; w < KW; ++w) B[at * KW + w] = key[q][w];
            SB[at] = (uint16_t)bin;
        }
    }
    __syncthreads();
    if (maxsub > (unsigned)kRankMax && nlarge <= kMaxLarge) {
        // a few clustered sub-bins: each sorted in place by the whole block
        // with a bitonic network for any length (every compare-exchange puts
        // the smaller key first; a partner past the end stands for +infinity
        // and is skipped), the others rank sorted as below
        for (unsigned q = 0; q < nlarge; ++q) {
            const unsigned a0 = st[large[q]], m = cnt[large[q]] - a0;
            uint64_t *X = B + (uint64_t)a0 * KW;
            unsigned P = 2;
            while (P < m) P <<= 1;
            for (unsigned k = 2; k <= P; k <<= 1) {
                for (unsigned j = k >> 1; j > 0; j >>= 1) {
                    for (unsigned p = tid; p < P / 2; p += kBucketThreads) {
                        unsigned i, x;
                        if (j == (k >> 1)) {   // the flip: i against its mirror in the k-block
                            const unsigned blk = p / j, off = p % j;
                            i = blk * k + off;
                            x = blk * k + (k - 1 - off);
                        } else {
                            i = (p / j) * 2 * j + (p % j);
                            x = i + j;
                        }
                        if (x < m && key_less<KW>(X + x * KW, X + i * KW)) {
#pragma unroll
                            for (int w = 0; w < KW; ++w) {
                                const uint64_t t = X[i * KW + w];
                                X[i * KW + w] = X[x * KW + w];
                                X[x * KW + w] = t;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (unsigned i = tid; i < m * KW; i += kBucketThreads) data[(s0 + a0) * KW + i] = X[i];
        }
    }
    if (maxsub <= (unsigned)kRankMax || nlarge <= kMaxLarge) {
        // rank sort inside each sub-bin: a key's place is the number of keys
        // of its sub-bin below it (the keys are distinct); neighbouring
        // threads mostly share a sub-bin, so the loop reads are broadcasts.
        // Each key goes straight to its place in global memory.  Sub-bins
        // above kRankMax keys were placed above.
        for (unsigned i = tid; i < n; i += kBucketThreads) {
            uint64_t k[KW];
#pragma unroll
            for (int w = 0; w < KW; ++w) k[w] = B[i * KW + w];
            const unsigned bin = SB[i];
            const unsigned a0 = st[bin], m = cnt[bin] - a0;
            if (m > kRankMax) continue;
            const unsigned rk = rank_in_subbin<KW>(B, a0, m, k);
#pragma unroll
            for (int w = 0; w < KW; ++w) data[(s0 + a0 + rk) * KW + w] = k[w];
        }
        return;
    }
    // many clustered sub-bins: bitonic sort of the whole segment (all-ones
    // pads sort last)
    unsigned P = 2;
    while (P < n) P <<= 1;
    for (unsigned i = n + tid; i < P; i += kBucketThreads)
#pragma unroll
        for (int w = 0; w < KW; ++w) B[i * KW + w] = ~0ull;
    __syncthreads();
    for (unsigned k = 2; k <= P; k <<= 1) {
        for (unsigned j = k >> 1; j > 0; j >>= 1) {
            for (unsigned i = tid; i < P; i += kBucketThreads) {
                const unsigned ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    if (key_less<KW>(B + ixj * KW, B + i * KW) == up) {
#pragma unroll
                        for (int w = 0; w < KW; ++w) {
                            const uint64_t t = B[i * KW + w];
                            B[i * KW + w] = B[ixj * KW + w];
                            B[ixj * KW + w] = t;
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    for (unsigned i = tid; i < n * KW; i += kBucketThreads) data[s0 * KW + i] = B[i];
}

// Segments above seg_cap<KW>() keys (runs of equal top bits), one block each:
// a stable LSD radix sort of the segment in global memory, ping-ponging with
// the same range of `alt`.  When the whole segment shares its top bits only
// the bits below them are sorted.  Per pass: the segment's digit histogram
// and its scan, then its tiles of kBigTile keys in order, each key ranked
// stably among the equal digits of its warp (one ballot per digit bit) and
// of the warps before it, and stored behind the keys of earlier tiles with
// the same digit.  Segments above kBigSegMax keys are left to the caller.
constexpr int kBigThreads = 1024;
constexpr uint64_t kBigSegMax = 1ull << 22;

template <int KW>
__global__ void __launch_bounds__(kBigThreads, 1) big_segment_sort_kernel(
    uint64_t *data, uint64_t *alt, int bits, const unsigned long long *big,
    const unsigned long long *nbig) {
    constexpr int NW = kBigThreads / 32;
    __shared__ unsigned hist[kRadixBins];
    __shared__ unsigned long long gbase[kRadixBins];
    __shared__ uint16_t wcnt[NW][kRadixBins];
    const unsigned long long seg = blockIdx.x;
    if (seg >= *nbig) return;
    const uint64_t begin = big[2 * seg], n = big[2 * seg + 1];
    if (n > kBigSegMax) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t t0 = top_bits<KW>(data + begin * KW, bits);
    const uint32_t t1 = top_bits<KW>(data + (begin + n - 1) * KW, bits);
    const int low = t0 == t1 ? bits - kTopBits : bits;
    const int passes = (low + kRadixBits - 1) / kRadixBits;
    uint64_t *src = data + begin * KW, *dst = alt + begin * KW;
    const unsigned lt = (1u << lane) - 1;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * kRadixBits;
        for (int d = tid; d < kRadixBins; d += kBigThreads) hist[d] = 0;
        __syncthreads();
        for (uint64_t i = tid; i < n; i += kBigThreads) atomicAdd(&hist[digit_of<KW>(src + i * KW, shift)], 1u);
        __syncthreads();
        if (tid < 32) {   // exclusive scan of the 256 counts by one warp, 8 per lane
            unsigned v[kRadixBins / 32], sum = 0;
#pragma unroll
            for (int j = 0; j < kRadixBins / 32; ++j) {
                v[j] = hist[lane * (kRadixBins / 32) + j];
                sum += v[j];
            }
            unsigned incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            unsigned long long pre = incl - sum;
#pragma unroll
            for (int j = 0; j < kRadixBins / 32; ++j) {
                gbase[lane * (kRadixBins / 32) + j] = pre;
                pre += v[j];
            }
        }
        __syncthreads();
        for (uint64_t t = 0; t < n; t += kBigThreads) {
            const uint64_t i = t + tid;
            const bool in = i < n;
            uint64_t key[KW];
#pragma unroll
            for (int w = 0; w < KW; ++w) key[w] = in ? src[i * KW + w] : 0;
            const unsigned dg = in ? digit_of<KW>(key, shift) : kRadixBins - 1;
            unsigned peers = __ballot_sync(0xffffffffu, in);
#pragma unroll
            for (int b = 0; b < kRadixBits; ++b) {
                const bool bit = (dg >> b) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, bit);
                peers &= bit ? bal : ~bal;
            }
            for (int d = lane; d < kRadixBins; d += 32) wcnt[warp][d] = 0;
            __syncwarp();
            if (in && lane == __ffs(peers) - 1) wcnt[warp][dg] = (uint16_t)__popc(peers);
            __syncthreads();
            // per digit: keys of the warps before each warp (in place), and the
            // digit's count in this tile
            if (tid < kRadixBins) {
                unsigned run = 0;
#pragma unroll 4
                for (int w = 0; w < NW; ++w) {
                    const unsigned c = wcnt[w][tid];
                    wcnt[w][tid] = (uint16_t)run;
                    run += c;
                }
                hist[tid] = run;
            }
            __syncthreads();
            if (in) {
                const uint64_t o = gbase[dg] + wcnt[warp][dg] + __popc(peers & lt);
#pragma unroll
                for (int w = 0; w < KW; ++w) dst[o * KW + w] = key[w];
            }
            __syncthreads();
            if (tid < kRadixBins) gbase[tid] += hist[tid];
            __syncthreads();
        }
        uint64_t *tmp = src;
        src = dst;
        dst = tmp;
    }
    if (passes & 1) {   // the result is in alt: back into place
        __syncthreads();
        for (uint64_t i = tid; i < n * KW; i += kBigThreads) data[begin * KW + i] = alt[begin * KW + i];
    }
}

uint32_t sort_tiles(uint64_t n, int kw) {
    const uint64_t t = kw == 1 ? (uint64_t)tile_keys<1>() : (uint64_t)tile_keys<2>();
    return (uint32_t)((n + t - 1) / t);
}

unsigned grid_for(uint64_t n, unsigned threads, unsigned cap) {
    uint64_t b = (n + threads - 1) / threads;
    if (b > cap) b = cap;
    return b ? (unsigned)b : 1u;
}

}  // namespace

uint64_t bucket_hist_blocks(uint64_t n) { return (n + kHistTile - 1) / kHistTile; }

cudaError_t bucket_histogram(const uint64_t *keys, uint64_t n, int shift, unsigned short *partial,
                             unsigned *hist, cudaStream_t s) {
    const uint64_t nb = bucket_hist_blocks(n);
    const int smem = kHistBins * 2;
    cudaError_t e = cudaFuncSetAttribute(bucket_hist_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    bucket_hist_kernel<<<(unsigned)nb, 512, smem, s>>>(keys, n, shift, partial);
    bucket_hist_reduce_kernel<<<(kHistBins + 255) / 256, 256, 0, s>>>(partial, (unsigned)nb, hist);
    return cudaGetLastError();
}

cudaError_t bucket_place_and_sort(const uint64_t *in, uint64_t *out, uint64_t n, int shift,
                                  const unsigned *map, unsigned nsuper,
                                  const unsigned long long *start, const unsigned long long *lo,
                                  const int *rsh, unsigned long long *cursor, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(cursor, start, nsuper * sizeof(unsigned long long),
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    if (nsuper <= (unsigned)kSortedScatterMax) {
        const int smem = (int)(kSortedScatterTile * sizeof(uint64_t) + 4 * nsuper * sizeof(unsigned));
        e = cudaFuncSetAttribute(bucket_scatter_sorted_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        bucket_scatter_sorted_kernel<<<(unsigned)((n + kSortedScatterTile - 1) / kSortedScatterTile),
                                       1024, smem, s>>>(in, n, shift, map, nsuper, cursor, out);
    } else {
        const int smem = (int)(2 * nsuper * sizeof(unsigned));
        e = cudaFuncSetAttribute(bucket_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem);
        if (e != cudaSuccess) return e;
        bucket_scatter_kernel<<<(unsigned)((n + kScatterTile - 1) / kScatterTile), 256, smem, s>>>(
            in, n, shift, map, nsuper, cursor, out);
    }
    const int ssmem = kBucketCap * 8 + 3 * kSubBins * 4;
    e = cudaFuncSetAttribute(bucket_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ssmem);
    if (e != cudaSuccess) return e;
    bucket_sort_kernel<<<nsuper, kBucketThreads, ssmem, s>>>(out, start, lo, rsh);
    return cudaGetLastError();
}

uint64_t sort_scratch_words(uint64_t n, int kw) {
    return (uint64_t)kRadixBins * sort_tiles(n, kw) + kRadixBins;
}

cudaError_t radix_pass(const uint64_t *src, uint64_t *dst, uint64_t n, int kw, int shift,
                       uint32_t *counts, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint32_t ntiles = sort_tiles(n, kw);
    uint32_t *totals = counts + (uint64_t)kRadixBins * ntiles;
    if (kw == 1) {
        upsweep_kernel<1><<<ntiles, kSortThreads, 0, s>>>(src, n, shift, counts, ntiles);
        scan_rows_kernel<<<kRadixBins, kSortThreads, 0, s>>>(counts, ntiles, totals);
        downsweep_kernel<1><<<ntiles, down_threads<1>(), 0, s>>>(src, dst, n, shift, counts, totals,
                                                            ntiles);
    } else {
        upsweep_kernel<2><<<ntiles, kSortThreads, 0, s>>>(src, n, shift, counts, ntiles);
        scan_rows_kernel<<<kRadixBins, kSortThreads, 0, s>>>(counts, ntiles, totals);
        downsweep_kernel<2><<<ntiles, down_threads<2>(), 0, s>>>(src, dst, n, shift, counts, totals,
                                                            ntiles);
    }
    return cudaGetLastError();
}

uint64_t seg_half(int kw) { return (uint64_t)(kw == 1 ? seg_cap<1>() : seg_cap<2>()) / 2; }

uint64_t seg_bounds_entries(uint64_t n, int kw) { return (n + seg_half(kw) - 1) / seg_half(kw) + 2; }

cudaError_t top_segment_sort(uint64_t *data, uint64_t n, int kw, int bits, unsigned long long *b,
                             unsigned long long *big, unsigned long long *nbig, cudaStream_t s) {
    if (bits < kTopBits + 12) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(nbig, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    const uint64_t H = seg_half(kw);
    const uint64_t nb = (n + H - 1) / H + 1;   // b[0..nb-1], the last one n
    const unsigned g = (unsigned)((nb + 255) / 256);
    if (kw == 1)
        seg_bounds_kernel<1><<<g, 256, 0, s>>>(data, n, bits, H, nb, b);
    else
        seg_bounds_kernel<2><<<g, 256, 0, s>>>(data, n, bits, H, nb, b);
    // keys, two arrays per sub-bin, one 16-bit sub-bin per key
    const int smem1 = seg_cap<1>() * (8 + 2) + 2 * kSubBins * 4;
    const int smem2 = seg_cap<2>() * (16 + 2) + 2 * kSubBins * 4;
    if (kw == 1) {
        e = cudaFuncSetAttribute(segment_sort_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem1);
        if (e != cudaSuccess) return e;
        segment_sort_kernel<1><<<(unsigned)(nb - 1), kBucketThreads, smem1, s>>>(data, bits, b, big,
                                                                               nbig);
    } else {
        e = cudaFuncSetAttribute(segment_sort_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem2);
        if (e != cudaSuccess) return e;
        segment_sort_kernel<2><<<(unsigned)(nb - 1), kBucketThreads, smem2, s>>>(data, bits, b, big,
                                                                               nbig);
    }
    return cudaGetLastError();
}

cudaError_t big_segment_sort(uint64_t *data, uint64_t *alt, uint64_t n, int kw, int bits,
                             const unsigned long long *big, const unsigned long long *nbig,
                             cudaStream_t s) {
    // at most one segment per seg_cap keys; blocks past *nbig return at once
    const uint64_t most = n / (uint64_t)(kw == 1 ? seg_cap<1>() : seg_cap<2>()) + 1;
    if (kw == 1)
        big_segment_sort_kernel<1><<<(unsigned)most, kBigThreads, 0, s>>>(data, alt, bits, big, nbig);
    else
        big_segment_sort_kernel<2><<<(unsigned)most, kBigThreads, 0, s>>>(data, alt, bits, big, nbig);
    return cudaGetLastError();
}

uint64_t big_segment_max() { return kBigSegMax; }

cudaError_t radix_sort(const uint64_t *in, uint64_t *alt0, uint64_t *alt1, uint64_t n, int kw,
                       int bits, uint32_t *counts, const uint64_t **result, cudaStream_t s) {
    *result = in;
    if (n <= 1) return cudaSuccess;
    const uint32_t ntiles = sort_tiles(n, kw);
    uint32_t *totals = counts + (uint64_t)kRadixBins * ntiles;
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    const uint64_t *src = in;
    for (int p = 0; p < passes; ++p) {
        uint64_t *dst = (p & 1) ? alt1 : alt0;
        const int shift = p * kRadixBits;
        if (kw == 1) {
            upsweep_kernel<1><<<ntiles, kSortThreads, 0, s>>>(src, n, shift, counts, ntiles);
            scan_rows_kernel<<<kRadixBins, kSortThreads, 0, s>>>(counts, ntiles, totals);
            downsweep_kernel<1><<<ntiles, down_threads<1>(), 0, s>>>(src, dst, n, shift, counts, totals,
                                                                ntiles);
        } else {
            upsweep_kernel<2><<<ntiles, kSortThreads, 0, s>>>(src, n, shift, counts, ntiles);
            scan_rows_kernel<<<kRadixBins, kSortThreads, 0, s>>>(counts, ntiles, totals);
            downsweep_kernel<2><<<ntiles, down_threads<2>(), 0, s>>>(src, dst, n, shift, counts, totals,
                                                                ntiles);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        src = dst;
    }
    *result = src;
    return cudaSuccess;
}

cudaError_t launch_query(const uint64_t *keys, uint64_t n, int kw, int K, Geometry G,
                         uint32_t *est, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned g = grid_for(n, 256, 152 * 64);
    if (kw == 1)
        query_kernel<1><<<g, 256, 0, s>>>(keys, n, K, G, est);
    else
        query_kernel<2><<<g, 256, 0, s>>>(keys, n, K, G, est);
    return cudaGetLastError();
}

cudaError_t launch_classify_query(const uint64_t *keys, uint64_t n, int kw, Geometry G,
                                  uint32_t tau, uint32_t *est, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned g = grid_for(n, 256, 152 * 8);
    if (kw == 1)
        classify_query_kernel<1><<<g, 256, 0, s>>>(keys, n, G, tau, est);
    else
        classify_query_kernel<2><<<g, 256, 0, s>>>(keys, n, G, tau, est);
    return cudaGetLastError();
}

uint64_t split_scratch_words(uint64_t n) { return (n + kSplitTile - 1) / kSplitTile + 1; }

cudaError_t launch_split(const uint64_t *keys, const uint32_t *est, uint64_t n, int kw,
                         uint32_t tau, uint64_t *out, uint64_t *scratch, DevCounters *ctr,
                         cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(&ctr->trusted, 0, sizeof(ctr->trusted), s);
    const uint64_t ntiles = (n + kSplitTile - 1) / kSplitTile;
    split_count_kernel<<<(unsigned)ntiles, kSortThreads, 0, s>>>(est, n, tau, scratch);
    split_scan_kernel<<<1, kSortThreads, 0, s>>>(scratch, ntiles, ctr);
    if (kw == 1)
        split_scatter_kernel<1><<<(unsigned)ntiles, kSortThreads, 0, s>>>(keys, est, n, tau, scratch,
                                                                          ctr, out);
    else
        split_scatter_kernel<2><<<(unsigned)ntiles, kSortThreads, 0, s>>>(keys, est, n, tau, scratch,
                                                                          ctr, out);
    return cudaGetLastError();
}

// pos[i] = number of keys of the sorted array below probe i (lower bound).
template <int KW>
__global__ void lower_bound_kernel(const uint64_t *keys, uint64_t n, const uint64_t *probes,
                                   uint64_t np, uint64_t *pos) {
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (key_less<KW>(keys + mid * KW, probes + i * KW))
            lo = mid + 1;
        else
            hi = mid;
    }
    pos[i] = lo;
}

cudaError_t launch_lower_bound(const uint64_t *keys, uint64_t n, int kw, const uint64_t *probes,
                               uint64_t np, uint64_t *pos, cudaStream_t s) {
    if (np == 0) return cudaSuccess;
    const unsigned g = (unsigned)((np + 255) / 256);
    if (kw == 1)
        lower_bound_kernel<1><<<g, 256, 0, s>>>(keys, n, probes, np, pos);
    else
        lower_bound_kernel<2><<<g, 256, 0, s>>>(keys, n, probes, np, pos);
    return cudaGetLastError();
}

cudaError_t launch_merge(uint64_t *dst, const uint64_t *src, Geometry G, cudaStream_t s) {
    merge_kernel<<<grid_for(G.words, 256, 152 * 16), 256, 0, s>>>(dst, src, G);
    return cudaGetLastError();
}

cudaError_t launch_count_saturated(Geometry G, DevCounters *ctr, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&ctr->saturated, 0, sizeof(ctr->saturated), s);
    if (e != cudaSuccess) return e;
    count_saturated_kernel<<<grid_for(G.words, 256, 152 * 16), 256, 0, s>>>(G, ctr);
    return cudaGetLastError();
}

}  // namespace countbf

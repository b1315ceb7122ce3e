// Insertion phase of KmerCo (Algorithm 1 with the countBF insert of
// Algorithm 3) on sm_103a.
//
// Work unit: a chunk of consecutive window starts of the flat bases array
// (kChunk, or kPartChunk in the partitioned design), regardless of read
// boundaries, so long and short reads balance the same way.  Per chunk a
// block
//   1. stages the chunk's bases (plus K-1 halo) in shared memory with
//      16-byte streaming loads, and marks the read starts inside it in a
//      break bitmap (no breaks when the reads are one sequence),
//   2. packs the bases to 2-bit codes (A=0 C=1 G=2 T=3, first base most
//      significant) with an invalid-base bitmap,
//   3. keeps the window starts whose K bases are valid and lie in one read,
//   4. per window: the canonical key (the smaller of forward and reverse
//      complement by value, or by H_0; Sections 2.2-2.3), k_h MurmurHash3
//      hashes, one saturating counter increment per hash (Algorithm 3), and
//      an insert into the distinct-key set (open addressing, linear
//      probing); keys new to the set are staged in shared memory and
//      appended to the distinct list with one global atomic per chunk.
//
// Two designs apply the counter increments of step 4:
//  - atomic: each increment is a compare-and-swap on its 64-bit cell in
//    global memory;
//  - partitioned (k_h <= 4, at most 2^30 cells): each increment is emitted
//    as a 32-bit code (cell within its coarse region, counter within the
//    cell); the chunk's codes are counting-sorted in shared memory into 64
//    coarse countBF regions and appended to per-region buffers with one
//    cursor atomic per region and chunk.  repartition_kernel splits every
//    region into slices, and one block per slice applies its increments in
//    shared memory: apply_count_kernel (alpha <= 15) counts them in 32-bit
//    lanes and adds the counts with saturation (the repartition then writes
//    each increment as its 16-bit lane index), apply_kernel uses
//    shared-memory compare-and-swap on the cells.  Either writes the slice
//    back once.  Increments that do not fit a buffer fall back to the global
//    compare-and-swap.
// Saturating increments commute, so both designs give the same countBF.
#include "kmerco_internal.cuh"

namespace countbf {
namespace {

// Staging sizes for a chunk of CHUNK window starts.
template <int CHUNK>
struct ChunkDims {
    static constexpr int kPack32 = CHUNK / 16 + 8;   // 16 bases per 32-bit word; chunk + 128 bases
};

template <int KW, int CHUNK, int PART>
struct __align__(16) InsertSmem {
    uint32_t pk[ChunkDims<CHUNK>::kPack32];     // codes; word t at t ^ 1 so pairs read as u64
    uint16_t inv[ChunkDims<CHUNK>::kPack32];    // bit j of inv[t]: base 16t + j is not ACGTacgt
    uint32_t brk[ChunkDims<CHUNK>::kPack32 / 2];  // bit q: a read starts at base q of the chunk
    uint16_t vpos[CHUNK];                       // valid window starts
    uint64_t fresh[CHUNK * KW];                 // keys new to the distinct set
    // partitioned design: the chunk's counter-increment codes
    uint32_t staged[PART ? CHUNK * kPartMaxHash : 1];
    uint32_t sorted[PART ? CHUNK * kPartMaxHash : 1];
    uint8_t sbin[PART == 2 ? CHUNK * kPartMaxHash : 1];   // coarse region of staged[i]
    unsigned hist[PART ? kCoarseBins : 1];
    unsigned start[PART ? kCoarseBins : 1];
    unsigned fill[PART ? kCoarseBins : 1];
    unsigned long long base[PART ? kCoarseBins : 1];
    unsigned nvalid;
    unsigned nfresh;
    unsigned nupd;
    unsigned long long fresh_base;
};

// 64 bits of a bitmap starting at bit p.
__device__ __forceinline__ uint64_t bits_at(const uint64_t *bm, unsigned p) {
    unsigned w = p >> 6, s = p & 63;
    uint64_t v = bm[w] >> s;
    if (s) v |= bm[w + 1] << (64 - s);
    return v;
}

__device__ __forceinline__ uint64_t load_cg(const uint64_t *p) { return __ldcg(p); }

// L2 eviction-priority policies.  The countBF is kept (evict_last) while
// the distinct set, touched once per window at random over a region much
// larger than L2, is let go first.
__device__ __forceinline__ uint64_t policy_keep() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_stream() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// 64-bit load that bypasses L1 (the value may be changed by other SMs'
// atomics) with an L2 eviction policy.
__device__ __forceinline__ uint64_t load_hint(const uint64_t *a, uint64_t pol) {
    uint64_t v;
    asm volatile("ld.global.cg.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(a), "l"(pol) : "memory");
    return v;
}

// 128-bit compare-and-swap (sm_90+), returns the previous slot contents.
__device__ __forceinline__ void cas128(uint64_t *addr, uint64_t cmp_lo, uint64_t cmp_hi,
                                       uint64_t new_lo, uint64_t new_hi, uint64_t &old_lo,
                                       uint64_t &old_hi) {
    asm volatile(
        "{\n\t.reg .b128 d, b, c;\n\t"
        "mov.b128 b, {%3, %4};\n\t"
        "mov.b128 c, {%5, %6};\n\t"
        "atom.global.cas.b128 d, [%2], b, c;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(old_lo), "=l"(old_hi)
        : "l"(addr), "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi)
        : "memory");
}

// Saturating increment of the counter at `shift` in cell `c`
// (Algorithm 3: extract, add one unless at 2^alpha - 1, write back).  `old`
// is a recent read of the cell; a failed CAS refreshes it.
__device__ __forceinline__ void sat_increment(uint64_t *cells, uint64_t c, unsigned shift,
                                              uint64_t maxc, uint64_t old, uint32_t limit,
                                              unsigned *err) {
    const uint64_t inc = 1ull << shift;
    for (uint32_t it = 0;; ++it) {
        if (((old >> shift) & maxc) == maxc) return;   // saturated: stays at the maximum
        uint64_t prev = atomicCAS((unsigned long long *)(cells + c), (unsigned long long)old,
                                  (unsigned long long)(old + inc));
        if (prev == old) return;
        old = prev;
        if (it >= limit) {
            atomicOr(err, kErrCasLimit);
            return;
        }
    }
}

// Insert a key into the distinct set; true when the key was not there yet.
// A slot stores the key with the set's generation tag in the unused top bits
// of its top word (SetTag): a slot whose tag differs from the current one is
// free, so a reset only moves to the next tag instead of clearing the table.
// Without spare bits (mask 0) a free slot is all ones, cleared at reset.
// For one-word keys `first` is an already loaded value of the home slot
// (kEmptyKey - 1 when none was loaded, a value no slot holds).
__device__ __forceinline__ bool slot_free(uint64_t top, const SetTag &t) {
    return t.mask ? (top & t.mask) != t.tag : top == kEmptyKey;
}

template <int KW>
__device__ __forceinline__ bool set_insert(uint64_t *table, uint64_t cap, uint64_t th,
                                           uint64_t klo, uint64_t khi, const SetTag &t,
                                           uint32_t limit, unsigned *err, uint64_t pol,
                                           uint64_t first = kEmptyKey - 1) {
    uint64_t slot = __umul64hi(th, cap);
    for (uint32_t it = 0;; ++it) {
        if (KW == 1) {
            const uint64_t want = klo | t.tag;
            uint64_t v = (it == 0 && first != kEmptyKey - 1) ? first : load_hint(table + slot, pol);
            for (;;) {   // settle this slot
                if (v == want) return false;
                if (!slot_free(v, t)) break;   // another key
                const uint64_t prev = atomicCAS((unsigned long long *)(table + slot),
                                                (unsigned long long)v, (unsigned long long)want);
                if (prev == v) return true;
                v = prev;                      // written meanwhile: look again
            }
        } else {
            // A plain 16-byte load settles most probes without an atomic: the
            // key itself, or another key (a different top word: each slot is
            // written once per generation).  A free slot, or one showing our
            // top word with another low word (a different key, or ours half
            // written), is decided by the 128-bit compare-and-swap, whose
            // result is the slot's real contents.
            const uint64_t whi = khi | t.tag;
            ulonglong2 v = __ldcg((const ulonglong2 *)(table + 2 * slot));
            for (;;) {
                if (v.x == klo && v.y == whi) return false;
                const bool free = t.mask ? slot_free(v.y, t) : (v.x == kEmptyKey || v.y == kEmptyKey);
                if (!free && v.y != whi) break;
                const uint64_t elo = free ? v.x : kEmptyKey, ehi = free ? v.y : kEmptyKey;
                uint64_t olo, ohi;
                cas128(table + 2 * slot, elo, ehi, klo, whi, olo, ohi);
                if (olo == elo && ohi == ehi) return true;
                if (!free && olo == v.x && ohi == v.y) break;   // a different key, settled
                v.x = olo;
                v.y = ohi;
            }
        }
        if (++slot == cap) slot = 0;
        if (it >= limit) {
            atomicOr(err, kErrProbeLimit);
            return false;
        }
    }
}

// One chunk of CHUNK window starts (steps 1-5 above) for the sample
// described by `a`; counts its windows into my_windows / my_skipped.
template <int KW, int CHUNK, int PART>
__device__ __forceinline__ void process_chunk(const InsertArgs &a, uint64_t chunk,
                                              InsertSmem<KW, CHUNK, PART> &S, uint64_t pol_keep,
                                              uint64_t pol_stream,
                                              unsigned long long &my_windows,
                                              unsigned long long &my_skipped) {
    constexpr int kPack32 = ChunkDims<CHUNK>::kPack32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = a.K;
    const uint64_t total = a.last - a.first;
    const Geometry &G = a.G;
    const uint64_t c0 = chunk * (uint64_t)CHUNK;
    const uint64_t e = min(c0 + (uint64_t)(CHUNK + K - 1), total);
    const unsigned nb = (unsigned)(e - c0);
    const uintptr_t src = (uintptr_t)(a.bases + c0);
    const unsigned head = (unsigned)(src & 15);
    const uintptr_t abase = src - head;

    // 1. read starts inside the chunk's span (none when the reads are one
    //    sequence); S.brk is zero on entry
    for (uint64_t r = (uint64_t)a.first_read[chunk] + tid; !a.whole_file && r < a.nreads;
         r += kInsertThreads) {
        uint64_t s = a.offsets[r] - a.first;
        if (s >= c0 + nb) break;
        if (s < c0) continue;   // only with decreasing offsets, which the host rejects
        unsigned q = (unsigned)(s - c0);
        if (q > 0) atomicOr(&S.brk[q >> 5], 1u << (q & 31));
    }
    if (tid == 0) {
        S.nvalid = 0;
        S.nfresh = 0;
        S.nupd = 0;
    }
    if (PART && tid < kCoarseBins) {
        S.hist[tid] = 0;
        S.fill[tid] = 0;
    }
    // 2. bases [16t, 16t + 16) of the span straight from global memory (the
    //    two 16-byte vectors holding them: whole ones with streaming loads,
    //    the partial ones at the span's ends bytewise, 'N' outside it), then
    //    2-bit codes + invalid bits
    for (int t = tid; t < kPack32; t += kInsertThreads) {
        uint32_t w[8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned lo = (unsigned)(t + h) << 4;
            if (lo >= head && lo + 16 <= head + nb) {
                const uint4 v = __ldcs((const uint4 *)(abase + lo));
                w[4 * h] = v.x;
                w[4 * h + 1] = v.y;
                w[4 * h + 2] = v.z;
                w[4 * h + 3] = v.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t word = 0;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const unsigned b = lo + 4 * q + k;
                        const unsigned c = b >= head && b < head + nb
                                               ? *(const uint8_t *)(abase + b) : (unsigned)'N';
                        word |= c << (8 * k);
                    }
                    w[4 * h + q] = word;
                }
            }
        }
        // the 16 bytes start `head` bytes into the 32 loaded ones
        const unsigned hb = (head & 3) * 8;
        uint32_t x[4];
        switch (head >> 2) {
        case 0:
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = __funnelshift_r(w[i], w[i + 1], hb);
            break;
        case 1:
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = __funnelshift_r(w[i + 1], w[i + 2], hb);
            break;
        case 2:
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = __funnelshift_r(w[i + 2], w[i + 3], hb);
            break;
        default:
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = __funnelshift_r(w[i + 3], w[i + 4], hb);
            break;
        }
        uint32_t code = 0, bad = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const unsigned c = (x[j >> 2] >> (8 * (j & 3))) & 0xFFu;
            const unsigned u = c | 0x20u;
            const bool ok = (u == 'a') | (u == 'c') | (u == 'g') | (u == 't');
            const unsigned cd = ((c >> 1) ^ (c >> 2)) & 3u;   // A,a->0 C,c->1 G,g->2 T,t->3
            code = (code << 2) | (ok ? cd : 0u);
            bad |= (ok ? 0u : 1u) << j;
        }
        S.pk[t ^ 1] = code;
        S.inv[t] = (uint16_t)bad;
    }
    __syncthreads();

    // 3. window starts: inside one read, K valid bases
    const uint64_t *inv64 = (const uint64_t *)S.inv;
    const uint64_t *brk64 = (const uint64_t *)S.brk;
    const uint64_t maskK = K == 64 ? ~0ull : ((1ull << K) - 1);
    const uint64_t maskK1 = (1ull << (K - 1)) - 1;
    for (int p0 = 0; p0 < CHUNK; p0 += kInsertThreads) {
        unsigned p = (unsigned)(p0 + tid);
        bool window = p + (unsigned)K <= nb && (bits_at(brk64, p + 1) & maskK1) == 0;
        bool valid = window && (bits_at(inv64, p) & maskK) == 0;
        my_windows += window;
        my_skipped += window && !valid;
        unsigned bal = __ballot_sync(0xffffffffu, valid);
        unsigned base = 0;
        if (lane == 0 && bal) base = atomicAdd(&S.nvalid, (unsigned)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (valid) S.vpos[base + __popc(bal & ((1u << lane) - 1))] = (uint16_t)p;
    }
    __syncthreads();

    // 4. per valid window: canonical key, hashes, counter updates, set insert
    for (int i = tid; i < kPack32 / 2; i += kInsertThreads) S.brk[i] = 0;   // for the next chunk
    const unsigned nvalid = S.nvalid;
    const uint64_t *pk64 = (const uint64_t *)S.pk;
    for (unsigned i0 = (unsigned)warp * 32; i0 < nvalid; i0 += kInsertThreads) {
        const unsigned i = i0 + lane;
        const bool active = i < nvalid;
        uint64_t klo = 0, khi = 0;
        if (active) {
            const unsigned p = S.vpos[i];
            const unsigned w = p >> 5, s = (p & 31) * 2;
            const uint64_t x0 = pk64[w], x1 = pk64[w + 1];
            const uint64_t t0 = s ? (x0 << s) | (x1 >> (64 - s)) : x0;
            if (KW == 1) {
                const uint64_t fwd = t0 >> (64 - 2 * K);
                klo = fwd;
                if (a.canonical == 1) {
                    const uint64_t rc = revcomp64(fwd, K);
                    klo = rc < fwd ? rc : fwd;
                } else if (a.canonical == 2) {   // the strand with the smaller H_0
                    const uint64_t rc = revcomp64(fwd, K);
                    uint64_t hf, hr, t;
                    murmur8(premix8(fwd), 0u, hf, t);
                    murmur8(premix8(rc), 0u, hr, t);
                    klo = hf < hr ? fwd : rc;
                }
            } else {
                const uint64_t x2 = pk64[w + 2];
                const uint64_t t1 = s ? (x1 << s) | (x2 >> (64 - s)) : x1;
                const int r = 128 - 2 * K;   // 0..62
                uint64_t fhi, flo;
                if (r == 0) {
                    fhi = t0;
                    flo = t1;
                } else {
                    flo = (t1 >> r) | (t0 << (64 - r));
                    fhi = t0 >> r;
                }
                klo = flo;
                khi = fhi;
                if (a.canonical) {
                    uint64_t rhi, rlo;
                    revcomp128(fhi, flo, K, rhi, rlo);
                    bool take_rc;
                    if (a.canonical == 2) {   // the strand with the smaller H_0
                        uint64_t hf, hr, t;
                        murmur16(flo, fhi, 0u, hf, t);
                        murmur16(rlo, rhi, 0u, hr, t);
                        take_rc = !(hf < hr);
                    } else {
                        take_rc = rhi < fhi || (rhi == fhi && rlo < flo);
                    }
                    if (take_rc) {
                        klo = rlo;
                        khi = rhi;
                    }
                }
            }
        }

        uint64_t table_hash = 0, table_first = kEmptyKey - 1;
        const uint64_t k1m = KW == 1 ? premix8(klo) : 0;
        if (PART) {
            // Partitioned design: stage one 32-bit code per increment, the
            // cell within its coarse region (up to 24 bits) above the counter
            // within the cell (6 bits), the region itself beside it.  A
            // window's k_h codes sit together: one reservation per warp.  The
            // hashes go two per loop trip (a smaller loop body measured
            // faster than all k_h at once); the distinct-set home slot is
            // loaded as soon as the first hash gives it.
            const unsigned nh = (unsigned)G.nhash;   // at most kPartMaxHash
            const unsigned bal = __ballot_sync(0xffffffffu, active);
            unsigned base = 0;
            if (lane == 0 && bal) base = atomicAdd(&S.nupd, nh * (unsigned)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            base += nh * (unsigned)__popc(bal & ((1u << lane) - 1));
            if (active) {
#pragma unroll 2
                for (unsigned j = 0; j < nh; ++j) {
                    uint64_t h1, h2, cell;
                    unsigned slot;
                    if (KW == 1)
                        murmur8(k1m, j, h1, h2);
                    else
                        murmur16(klo, khi, j, h1, h2);
                    if (j == 0) {
                        table_hash = h2;
                        if (KW == 1)
                            table_first = load_hint(a.table + __umul64hi(table_hash, a.cap),
                                                    pol_stream);
                    }
                    address(G, h1, cell, slot);
                    const unsigned bin = (unsigned)(cell >> a.coarse_shift);
                    const uint32_t code =
                        ((uint32_t)(cell & ((1ull << a.coarse_shift) - 1)) << 6) | slot;
                    if (PART == 2) {   // region beside the code
                        S.staged[base + j] = code;
                        S.sbin[base + j] = (uint8_t)bin;
                    } else {           // region in the top 6 bits (coarse_shift <= 20)
                        S.staged[base + j] = (bin << 26) | code;
                    }
                    atomicAdd(&S.hist[bin], 1u);
                }
            }
        }
        // Atomic design: all loads of a group of four hashes (and, in the
        // first group, the distinct-set home slot) are issued together, then
        // all first compare-and-swap attempts; only failed attempts retry.
        for (int a0 = 0; !PART && a0 < G.nhash; a0 += 4) {
            uint64_t cell[4], cur[4], prev[4];
            unsigned sh[4], slot[4];
            bool use[4], need[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                use[j] = active && (a0 + j < G.nhash);
                cell[j] = 0;
                sh[j] = 0;
                slot[j] = 0;
                if (use[j]) {
                    uint64_t h1, h2;
                    if (KW == 1)
                        murmur8(k1m, (uint32_t)(a0 + j), h1, h2);
                    else
                        murmur16(klo, khi, (uint32_t)(a0 + j), h1, h2);
                    if (a0 + j == 0) table_hash = h2;
                    address(G, h1, cell[j], slot[j]);
                    sh[j] = slot[j] * (unsigned)G.alpha;
                }
            }
            if (KW == 1 && a0 == 0 && active)
                table_first = load_hint(a.table + __umul64hi(table_hash, a.cap), pol_stream);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (use[j]) cur[j] = load_hint(G.cells + cell[j], pol_keep);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                need[j] = use[j] && ((cur[j] >> sh[j]) & G.maxc) != G.maxc;
                prev[j] = cur[j];
                if (need[j])
                    prev[j] = atomicCAS((unsigned long long *)(G.cells + cell[j]),
                                        (unsigned long long)cur[j],
                                        (unsigned long long)(cur[j] + (1ull << sh[j])));
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (need[j] && prev[j] != cur[j])
                    sat_increment(G.cells, cell[j], sh[j], G.maxc, prev[j], G.cas_limit,
                                  &a.ctr->error);
        }

        bool isnew = false;
        if (active)
            isnew = set_insert<KW>(a.table, a.cap, table_hash, klo, khi, a.set_tag,
                                   G.probe_limit, &a.ctr->error, pol_stream, table_first);
        const unsigned bal = __ballot_sync(0xffffffffu, isnew);
        unsigned base = 0;
        if (lane == 0 && bal) base = atomicAdd(&S.nfresh, (unsigned)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (isnew) {
            const unsigned slot = base + __popc(bal & ((1u << lane) - 1));
            S.fresh[slot * KW] = klo;
            if (KW == 2) S.fresh[slot * KW + 1] = khi;
        }
    }
    __syncthreads();

    // 4b. reservations, all in one phase: the distinct-list run of this
    //     chunk's new keys, and (partitioned design) one cursor atomic per
    //     coarse region for the chunk's increment codes
    const unsigned nfresh = S.nfresh;
    if (tid == kCoarseBins && nfresh) {
        unsigned long long b = atomicAdd(&a.ctr->distinct, (unsigned long long)nfresh);
        if (b + nfresh > a.dlist_cap) {
            atomicOr(&a.ctr->error, kErrListFull);
            b = ~0ull;
        }
        S.fresh_base = b;
    }
    if (PART) {
        const unsigned nupd = S.nupd;
        if (tid < kCoarseBins) {   // warps 0 and 1: prefix over the regions
            const unsigned n = S.hist[tid];
            unsigned incl = n, below = 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (unsigned)o) incl += t;
            }
            if (tid >= 32) {   // warp 1 starts after all of warp 0's regions
                below = S.hist[tid - 32];
#pragma unroll
                for (int o = 16; o; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
            }
            S.start[tid] = below + incl - n;
            unsigned long long b0 = ~0ull;
            if (n) {
                b0 = atomicAdd(a.coarse_cursor + tid, (unsigned long long)n);
                if (b0 + n > a.coarse_cap)
                    b0 = ~0ull;   // region full: these go to the global fallback
                else
                    atomicAdd(a.coarse_written + tid, (unsigned long long)n);
            }
            S.base[tid] = b0;
        }
        __syncthreads();
        // 4c. counting sort of the codes by coarse region in shared memory
        for (unsigned i = tid; i < nupd; i += kInsertThreads) {
            if (PART == 2) {
                const unsigned bin = S.sbin[i];
                S.sorted[S.start[bin] + atomicAdd(&S.fill[bin], 1u)] = S.staged[i];
            } else {
                const uint32_t c = S.staged[i];
                const unsigned bin = c >> 26;
                S.sorted[S.start[bin] + atomicAdd(&S.fill[bin], 1u)] = c & 0x3FFFFFFu;
            }
        }
        __syncthreads();
        // 4d. one warp per region run: contiguous stores into the region
        for (unsigned bin = warp; bin < kCoarseBins; bin += kInsertThreads / 32) {
            const unsigned n = S.hist[bin], s0 = S.start[bin];
            const unsigned long long b0 = S.base[bin];
            uint32_t *dst = b0 != ~0ull ? a.coarse + (uint64_t)bin * a.coarse_cap + b0 : nullptr;
            for (unsigned i = lane; i < n; i += 32) {
                const uint32_t code = S.sorted[s0 + i];
                if (dst) {
                    __stcs(dst + i, code);
                } else {
                    const uint64_t cell = ((uint64_t)bin << a.coarse_shift) | (code >> 6);
                    const unsigned shift = (code & 63u) * (unsigned)G.alpha;
                    sat_increment(G.cells, cell, shift, G.maxc, load_cg(G.cells + cell),
                                  G.cas_limit, &a.ctr->error);
                }
            }
        }
    } else {
        __syncthreads();
    }

    // 5. this chunk's new keys into the distinct list
    if (nfresh) {
        const unsigned long long b = S.fresh_base;
        if (b != ~0ull)
            for (unsigned i = tid; i < nfresh * KW; i += kInsertThreads)
                a.dlist[b * KW + i] = S.fresh[i];
    }
    __syncthreads();
}

// Warp totals of windows and skipped windows into a sample's counters.
__device__ __forceinline__ void flush_totals(DevCounters *ctr, unsigned long long &w,
                                             unsigned long long &k) {
    for (int o = 16; o; o >>= 1) {
        w += __shfl_down_sync(0xffffffffu, w, o);
        k += __shfl_down_sync(0xffffffffu, k, o);
    }
    if ((threadIdx.x & 31) == 0 && w) {
        atomicAdd(&ctr->windows, w);
        atomicAdd(&ctr->skipped, k);
        atomicAdd(&ctr->inserted, w - k);
    }
    w = 0;
    k = 0;
}

template <int KW, int CHUNK, int PART>
__global__ void __launch_bounds__(kInsertThreads, 4) insert_kernel(InsertArgs a) {
    // dynamic: the partitioned variants need more than 48 KiB
    extern __shared__ __align__(16) unsigned char insert_smem[];
    InsertSmem<KW, CHUNK, PART> &S = *reinterpret_cast<InsertSmem<KW, CHUNK, PART> *>(insert_smem);
    for (int i = threadIdx.x; i < ChunkDims<CHUNK>::kPack32 / 2; i += kInsertThreads) S.brk[i] = 0;
    __syncthreads();
    const uint64_t pol_keep = policy_keep(), pol_stream = policy_stream();
    unsigned long long my_windows = 0, my_skipped = 0;
    for (uint64_t chunk = a.chunk_begin + blockIdx.x; chunk < a.nchunks; chunk += gridDim.x)
        process_chunk<KW, CHUNK, PART>(a, chunk, S, pol_keep, pol_stream, my_windows, my_skipped);
    flush_totals(a.ctr, my_windows, my_skipped);
}

// Many samples in one persistent launch (atomic update design): the chunks
// of all samples form one index space, sample s owning chunks
// [chunk_end[s-1], chunk_end[s]).  A block walks its chunks in increasing
// order, so the sample only moves forward; its arguments are kept in
// shared memory and its totals are flushed when it changes.
template <int KW, int CHUNK>
__global__ void __launch_bounds__(kInsertThreads, 4) insert_batch_kernel(
    const InsertArgs *args, const unsigned long long *chunk_end, int nsamples,
    unsigned long long total_chunks) {
    __shared__ InsertSmem<KW, CHUNK, 0> S;
    __shared__ InsertArgs A;
    const uint64_t pol_keep = policy_keep(), pol_stream = policy_stream();
    unsigned long long my_windows = 0, my_skipped = 0;
    for (int i = threadIdx.x; i < ChunkDims<CHUNK>::kPack32 / 2; i += kInsertThreads) S.brk[i] = 0;
    int s = -1;
    unsigned long long s_begin = 0;
    for (unsigned long long chunk = blockIdx.x; chunk < total_chunks; chunk += gridDim.x) {
        int t = s < 0 ? 0 : s;
        while (t < nsamples && chunk >= chunk_end[t]) ++t;   // uniform across the block
        if (t != s) {
            if (s >= 0) flush_totals(A.ctr, my_windows, my_skipped);
            __syncthreads();
            if (threadIdx.x == 0) A = args[t];
            s = t;
            s_begin = t ? chunk_end[t - 1] : 0;
            __syncthreads();
        }
        process_chunk<KW, CHUNK, 0>(A, chunk - s_begin, S, pol_keep, pol_stream, my_windows,
                                        my_skipped);
    }
    if (s >= 0) flush_totals(A.ctr, my_windows, my_skipped);
}

// Sum over reads of max(0, len - K + 1); flags decreasing offsets.
__global__ void window_bound_kernel(const uint64_t *offsets, uint64_t nreads, int K,
                                    DevCounters *ctr) {
    unsigned long long sum = 0;
    bool bad = false;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < nreads;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t s = offsets[r], e = offsets[r + 1];
        if (e < s) {
            bad = true;
            continue;
        }
        if (e - s >= (uint64_t)K) sum += e - s - K + 1;
    }
    for (int o = 16; o; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&ctr->bound, sum);
    if (bad) atomicOr(&ctr->bad_offsets, 1u);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctr->first = offsets[0];
        ctr->last = offsets[nreads];
    }
}

// first_read[c] = smallest r in [0, nreads] with offsets[r] - first >= c * chunk.
__global__ void first_read_kernel(const uint64_t *offsets, uint64_t nreads, uint64_t first,
                                  uint64_t nchunks, uint64_t chunk, uint32_t *first_read) {
    uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (c >= nchunks) return;
    const uint64_t target = first + c * chunk;
    uint64_t lo = 0, hi = nreads;   // answer in [lo, hi]
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (offsets[mid] >= target)
            hi = mid;
        else
            lo = mid + 1;
    }
    first_read[c] = (uint32_t)lo;
}

// Window bound of many samples in one launch: block (x, s) scans reads of
// sample s.  out[s] = {sum of max(0, len - K + 1), first offset, last offset,
// decreasing-offsets flag}.
struct BoundOut {
    unsigned long long bound, first, last, bad;
};
__global__ void window_bound_batch_kernel(const uint64_t *const *offsets, const uint64_t *nreads,
                                          int K, BoundOut *out) {
    const int smp = blockIdx.y;
    const uint64_t *off = offsets[smp];
    const uint64_t n = nreads[smp];
    unsigned long long sum = 0;
    bool bad = false;
    for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
         r += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = off[r], b = off[r + 1];
        if (b < a) {
            bad = true;
            continue;
        }
        if (b - a >= (uint64_t)K) sum += b - a - K + 1;
    }
    for (int o = 16; o; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&out[smp].bound, sum);
    if (bad) atomicOr(&out[smp].bad, 1ull);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[smp].first = off[0];
        out[smp].last = off[n];
    }
}

// first_read of every sample's chunks in one launch (chunk index space as in
// insert_batch_kernel).
__global__ void first_read_batch_kernel(const InsertArgs *args, const unsigned long long *chunk_end,
                                        int nsamples, unsigned long long total_chunks,
                                        uint64_t chunk) {
    const unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    if (c >= total_chunks) return;
    int lo = 0, hi = nsamples - 1;   // sample owning chunk c
    while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (c < chunk_end[mid])
            hi = mid;
        else
            lo = mid + 1;
    }
    const InsertArgs &a = args[lo];
    const unsigned long long local = c - (lo ? chunk_end[lo - 1] : 0);
    const uint64_t target = a.first + local * chunk;
    uint64_t rlo = 0, rhi = a.nreads;
    while (rlo < rhi) {
        const uint64_t mid = rlo + (rhi - rlo) / 2;
        if (a.offsets[mid] >= target)
            rhi = mid;
        else
            rlo = mid + 1;
    }
    const_cast<uint32_t *>(a.first_read)[local] = (uint32_t)rlo;
}

// Re-insert keys into a distinct set (growing a set, or merging another
// handle's keys).  With dlist != nullptr keys new to the set are appended.
template <int KW>
__global__ void reinsert_kernel(const uint64_t *keys, uint64_t n, uint64_t *table, uint64_t cap,
                                SetTag tag, uint64_t *dlist, uint64_t dlist_cap, DevCounters *ctr,
                                uint32_t probe_limit) {
    const int lane = threadIdx.x & 31;
    for (uint64_t i0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull; i0 < n;
         i0 += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = i0 + lane;
        bool isnew = false;
        uint64_t klo = 0, khi = 0;
        if (i < n) {
            klo = keys[i * KW];
            khi = KW == 2 ? keys[i * KW + 1] : 0;
            uint64_t h1, h2;
            if (KW == 1)
                murmur8(premix8(klo), 0, h1, h2);
            else
                murmur16(klo, khi, 0, h1, h2);
            isnew = set_insert<KW>(table, cap, h2, klo, khi, tag, probe_limit, &ctr->error,
                                   policy_stream());
        }
        if (dlist) {
            const unsigned bal = __ballot_sync(0xffffffffu, isnew);
            unsigned long long base = 0;
            if (lane == 0 && bal) base = atomicAdd(&ctr->distinct, (unsigned long long)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (isnew) {
                const uint64_t slot = base + __popc(bal & ((1u << lane) - 1));
                if (slot < dlist_cap) {
                    dlist[slot * KW] = klo;
                    if (KW == 2) dlist[slot * KW + 1] = khi;
                } else {
                    atomicOr(&ctr->error, kErrListFull);
                }
            }
        }
    }
}

// Exclusive prefix sum of v[0..n) into out[0..n), n <= E * kRepartThreads,
// by the whole block (E entries per thread).
template <int E>
__device__ __forceinline__ void repart_scan(const unsigned *v, unsigned *out, unsigned n) {
    const unsigned tid = threadIdx.x;
    unsigned x[E], sum = 0;
#pragma unroll
    for (int q = 0; q < E; ++q) {
        x[q] = E * tid + q < n ? v[E * tid + q] : 0u;
        sum += x[q];
    }
    unsigned tot;
    unsigned off = block_exclusive_scan<unsigned, kRepartThreads>(sum, tot);
#pragma unroll
    for (int q = 0; q < E; ++q) {
        if (E * tid + q < n) out[E * tid + q] = off;
        off += x[q];
    }
}

// Split each coarse region's increment codes into slices of 2^slice_shift
// cells.  Block (x, y) takes tile x of coarse region y.  MAXF bounds the
// slices per region (2^(coarse_shift - slice_shift)).  With LANES a slice
// code is the 16-bit counting lane (counter << slice_shift) | cell of the
// counting apply, else the 32-bit (cell << 6) | counter.
template <int MAXF, bool LANES>
__global__ void __launch_bounds__(kRepartThreads, 3) repartition_kernel(PartArgs p) {
    extern __shared__ uint32_t sorted[];   // the tile's codes grouped by slice
    __shared__ unsigned hist[MAXF], start[MAXF], fill[MAXF];
    __shared__ unsigned long long base[MAXF];
    const unsigned b = blockIdx.y, tid = threadIdx.x;
    const uint64_t n = p.coarse_written[b];
    const uint64_t t0 = (uint64_t)blockIdx.x * kRepartTile;
    if (t0 >= n) return;
    const unsigned cnt = (unsigned)min((uint64_t)kRepartTile, n - t0);
    const int fsh = 6 + p.slice_shift;                            // code >> fsh = slice
    const unsigned fpc = 1u << (p.coarse_shift - p.slice_shift);  // slices per coarse region
    for (unsigned f = tid; f < fpc; f += kRepartThreads) {
        hist[f] = 0;
        fill[f] = 0;
    }
    __syncthreads();
    // 16 codes per thread, all loads issued before use (the region is 16-byte
    // aligned: coarse_cap is a multiple of 4 and t0 of kRepartTile)
    const uint32_t *src = p.coarse + (uint64_t)b * p.coarse_cap + t0;
    uint32_t c16[16];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned i = 4 * (tid + j * kRepartThreads);
        if (i + 4 <= cnt) {
            const uint4 v = __ldcs((const uint4 *)(src + i));
            c16[4 * j] = v.x;
            c16[4 * j + 1] = v.y;
            c16[4 * j + 2] = v.z;
            c16[4 * j + 3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) c16[4 * j + q] = i + q < cnt ? src[i + q] : 0u;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned i = 4 * (tid + j * kRepartThreads);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (i + q < cnt) atomicAdd(&hist[c16[4 * j + q] >> fsh], 1u);
    }
    __syncthreads();
    if (MAXF <= 64) {
        if (tid < fpc) {
            unsigned pre = 0;
            for (unsigned f = 0; f < tid; ++f) pre += hist[f];
            start[tid] = pre;
        }
    } else {
        repart_scan<(MAXF + kRepartThreads - 1) / kRepartThreads>(hist, start, fpc);
    }
    for (unsigned f = tid; f < fpc; f += kRepartThreads) {
        const unsigned m = hist[f];
        unsigned long long b0 = ~0ull;
        if (m) {
            const uint64_t F = (uint64_t)b * fpc + f;
            b0 = atomicAdd(p.fine_cursor + F, (unsigned long long)m);
            if (b0 + m > p.fine_cap)
                b0 = ~0ull;
            else
                atomicAdd(p.fine_written + F, (unsigned long long)m);
        }
        base[f] = b0;
    }
    __syncthreads();
    // group the codes by slice, straight from registers
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const unsigned i = 4 * (tid + j * kRepartThreads);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (i + q < cnt) {
                const unsigned f = c16[4 * j + q] >> fsh;
                sorted[start[f] + atomicAdd(&fill[f], 1u)] = c16[4 * j + q];
            }
        }
    }
    __syncthreads();
    const uint32_t smask = (1u << p.slice_shift) - 1;
    for (unsigned i = tid; i < cnt; i += kRepartThreads) {
        const uint32_t code = sorted[i];
        const uint32_t word = code >> 6;
        const unsigned f = word >> p.slice_shift;
        const unsigned long long b0 = base[f];
        if (b0 != ~0ull) {
            const uint64_t F = (uint64_t)b * fpc + f;
            const uint64_t at = F * p.fine_cap + b0 + (i - start[f]);
            if (LANES)
                __stcs((unsigned short *)p.fine + at,
                       (unsigned short)(((code & 63u) << p.slice_shift) | (word & smask)));
            else
                __stcs((uint32_t *)p.fine + at, ((word & smask) << 6) | (code & 63u));
        } else {
            const uint64_t cell = ((uint64_t)b << p.coarse_shift) | word;
            sat_increment(p.G.cells, cell, (code & 63u) * (unsigned)p.G.alpha, p.G.maxc,
                          load_cg(p.G.cells + cell), p.G.cas_limit, &p.ctr->error);
        }
    }
}

// One slice of 2^slice_shift cells per block: load it into shared memory,
// apply its increment codes with shared-memory compare-and-swap (saturating
// at 2^alpha - 1), write it back.  LIMITED takes the retry bound from the
// handle (a retry limit set for testing); the default bound is a constant,
// which keeps the retry loop measurably faster.  With HALF (alpha divides
// 32, so no counter straddles the middle of a cell) each update is a 32-bit
// compare-and-swap on the half-cell that holds the counter.  Slices are
// 64 KiB, three blocks per SM, so one block's slice load and store overlap
// the other blocks' updates.
template <bool LIMITED, bool HALF>
__global__ void __launch_bounds__(kCasApplyThreads, 3) apply_kernel(ApplyArgs p) {
    extern __shared__ unsigned long long cells_s[];
    const uint64_t s = blockIdx.x;
    const uint64_t w0 = s << p.slice_shift;
    const uint64_t slice = 1ull << p.slice_shift;
    const unsigned nw = (unsigned)min(slice, p.G.words - w0);
    const uint64_t n = p.written[s];
    if (n == 0) return;   // no increments for this slice
    for (unsigned i = threadIdx.x; i < nw; i += kCasApplyThreads) cells_s[i] = p.G.cells[w0 + i];
    __syncthreads();
    const uint32_t *src = (const uint32_t *)p.codes + s * p.cap;   // 16-byte aligned: cap is a multiple of 4
    const uint32_t wmask = (uint32_t)(slice - 1);
    const uint64_t maxc = p.G.maxc;
    const unsigned alpha = (unsigned)p.G.alpha;
    // eight codes per thread in flight (two 16-byte loads), then their updates
    constexpr unsigned kStep = kCasApplyThreads * 8;
    for (uint64_t i0 = 0; i0 < n; i0 += kStep) {
        uint32_t code[8];
        unsigned valid = 0;
        const uint64_t i = i0 + threadIdx.x * 4ull;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint64_t j = i + (uint64_t)h * kCasApplyThreads * 4;
            if (j + 4 <= n) {
                const uint4 v = __ldcs((const uint4 *)(src + j));
                code[4 * h] = v.x;
                code[4 * h + 1] = v.y;
                code[4 * h + 2] = v.z;
                code[4 * h + 3] = v.w;
                valid |= 0xFu << (4 * h);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    code[4 * h + q] = j + q < n ? src[j + q] : 0u;
                    valid |= (j + q < n ? 1u : 0u) << (4 * h + q);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (!((valid >> q) & 1u)) continue;   // past the end
            const unsigned w = (code[q] >> 6) & wmask;
            const unsigned shift = (code[q] & 63u) * alpha;
            if (HALF) {   // the little-endian half-cell holding the counter
                unsigned *h32 = (unsigned *)cells_s + 2 * w + (shift >> 5);
                const unsigned sh = shift & 31u, mc = (unsigned)maxc;
                unsigned old = *h32;
                for (uint32_t it = 0;; ++it) {
                    if (((old >> sh) & mc) == mc) break;
                    const unsigned prev = atomicCAS(h32, old, old + (1u << sh));
                    if (prev == old) break;
                    old = prev;
                    if (it >= (LIMITED ? p.G.cas_limit : kCasLimit)) {
                        atomicOr(&p.ctr->error, kErrCasLimit);
                        break;
                    }
                }
                continue;
            }
            unsigned long long old = cells_s[w];
            for (uint32_t it = 0;; ++it) {
                if (((old >> shift) & maxc) == maxc) break;
                const unsigned long long prev = atomicCAS(cells_s + w, old, old + (1ull << shift));
                if (prev == old) break;
                old = prev;
                if (it >= (LIMITED ? p.G.cas_limit : kCasLimit)) {
                    atomicOr(&p.ctr->error, kErrCasLimit);
                    break;
                }
            }
        }
    }
    __syncthreads();
    for (unsigned i = threadIdx.x; i < nw; i += kCasApplyThreads) p.G.cells[w0 + i] = cells_s[i];
}

// Counting apply (alpha <= 15): one slice of 2^slice_shift cells per block.
// The slice's increments are counted in 32-bit shared-memory lanes, counter
// (cell, l) at lane l * 2^slice_shift + cell (a pass stages at most 2^31
// increments, so a lane cannot wrap).  Then every counter becomes
// min(old + count, 2^alpha - 1) and the slice is written back once.  With
// LANES the codes are the 16-bit lanes themselves, else 32-bit
// (cell << 6) | counter codes.
template <bool LANES>
__global__ void __launch_bounds__(kApplyThreads, 2) apply_count_kernel(ApplyArgs p) {
    extern __shared__ uint32_t lanes[];   // one 32-bit count per counter of the slice
    const uint64_t s = blockIdx.x;
    const uint64_t n = p.written[s];
    if (n == 0) return;   // no increments for this slice
    const int ssh = p.slice_shift;
    const uint64_t w0 = s << ssh;
    const uint64_t slice = 1ull << ssh;
    const unsigned nw = (unsigned)min(slice, p.G.words - w0);
    const unsigned eta = (unsigned)p.G.eta;
    const unsigned nwords = eta << ssh;
    for (unsigned i = threadIdx.x; i < nwords; i += kApplyThreads) lanes[i] = 0;
    __syncthreads();
    // 16 bytes per load: 8 lane codes or 4 cell codes; two loads per thread in flight
    constexpr unsigned kPer = LANES ? 8 : 4;
    constexpr unsigned kStep = kApplyThreads * 2 * kPer;
    const uint32_t wmask = (uint32_t)(slice - 1);
    // each slice's codes start 16-byte aligned (cap: a multiple of 8 lanes, 4 cells)
    const uint16_t *src16 = (const uint16_t *)p.codes + s * p.cap;
    const uint32_t *src32 = (const uint32_t *)p.codes + s * p.cap;
    for (uint64_t i0 = 0; i0 < n; i0 += kStep) {
        uint32_t code[2 * kPer];
        unsigned valid = 0;
        const uint64_t i = i0 + threadIdx.x * (uint64_t)kPer;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint64_t j = i + (uint64_t)h * kApplyThreads * kPer;
            if (j + kPer <= n) {
                const uint4 v = __ldcs(LANES ? (const uint4 *)(src16 + j) : (const uint4 *)(src32 + j));
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (LANES) {
                        code[kPer * h + 2 * q] = w[q] & 0xFFFFu;
                        code[kPer * h + 2 * q + 1] = w[q] >> 16;
                    } else {
                        code[kPer * h + q] = w[q];
                    }
                }
                valid |= ((1u << kPer) - 1) << (kPer * h);
            } else {
#pragma unroll
                for (unsigned q = 0; q < kPer; ++q) {
                    const bool in = j + q < n;
                    code[kPer * h + q] = !in ? 0u : LANES ? (uint32_t)src16[j + q] : src32[j + q];
                    valid |= (in ? 1u : 0u) << (kPer * h + q);
                }
            }
        }
#pragma unroll
        for (unsigned q = 0; q < 2 * kPer; ++q) {
            if (!((valid >> q) & 1u)) continue;   // past the end
            const unsigned c = LANES ? code[q] : ((code[q] & 63u) << ssh) | ((code[q] >> 6) & wmask);
            atomicAdd(lanes + c, 1u);
        }
    }
    __syncthreads();
    const uint32_t *cnt = lanes;
    const unsigned alpha = (unsigned)p.G.alpha;
    const uint64_t maxc = p.G.maxc;
    for (unsigned i = threadIdx.x; i < nw; i += kApplyThreads) {
        const uint64_t old = p.G.cells[w0 + i];
        uint64_t out = 0;
        for (unsigned l = 0; l < eta; ++l) {
            const uint64_t v = ((old >> (l * alpha)) & maxc) + cnt[((uint64_t)l << ssh) | i];
            out |= (v < maxc ? v : maxc) << (l * alpha);
        }
        p.G.cells[w0 + i] = out;
    }
}

// Launch insert_kernel<KW, CHUNK, PART> (g blocks), or with g == 0 report its
// resident blocks per SM in *per_sm.
template <int KW, int CHUNK, int PART>
cudaError_t insert_variant(const InsertArgs *a, unsigned g, cudaStream_t s, int *per_sm) {
    const int smem = (int)sizeof(InsertSmem<KW, CHUNK, PART>);
    cudaError_t e = cudaFuncSetAttribute(insert_kernel<KW, CHUNK, PART>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (per_sm)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, insert_kernel<KW, CHUNK, PART>,
                                                             kInsertThreads, smem);
    insert_kernel<KW, CHUNK, PART><<<g, kInsertThreads, smem, s>>>(*a);
    return cudaGetLastError();
}

// part: 0 atomic design; 1 partitioned, region bits inside the codes
// (coarse_shift <= 20); 2 partitioned, regions beside the codes.
cudaError_t dispatch_insert(const InsertArgs *a, int kw, int part, unsigned g, cudaStream_t s,
                            int *per_sm, int chunk = kChunk) {
    if (part == 0 && chunk == kSmallChunk)
        return kw == 1 ? insert_variant<1, kSmallChunk, 0>(a, g, s, per_sm)
                       : insert_variant<2, kSmallChunk, 0>(a, g, s, per_sm);
    if (part == 1 && kw == 1) return insert_variant<1, kPartChunk, 1>(a, g, s, per_sm);
    if (part == 1) return insert_variant<2, kPartChunk, 1>(a, g, s, per_sm);
    if (part == 2 && kw == 1) return insert_variant<1, kPartChunk, 2>(a, g, s, per_sm);
    if (part == 2) return insert_variant<2, kPartChunk, 2>(a, g, s, per_sm);
    if (kw == 1) return insert_variant<1, kChunk, 0>(a, g, s, per_sm);
    return insert_variant<2, kChunk, 0>(a, g, s, per_sm);
}

}  // namespace

int insert_blocks_per_sm(int kw, int part) {
    int n = 0;
    if (dispatch_insert(nullptr, kw, part, 0, 0, &n) != cudaSuccess) n = 0;
    return n > 0 ? n : 1;
}

cudaError_t launch_window_bound(const uint64_t *offsets, uint64_t nreads, int K, DevCounters *ctr,
                                cudaStream_t s) {
    uint64_t blocks = (nreads + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks == 0) blocks = 1;
    window_bound_kernel<<<(unsigned)blocks, 256, 0, s>>>(offsets, nreads, K, ctr);
    return cudaGetLastError();
}

cudaError_t launch_first_read(const uint64_t *offsets, uint64_t nreads, uint64_t first,
                              uint64_t nchunks, uint64_t chunk, uint32_t *first_read,
                              cudaStream_t s) {
    if (nchunks == 0) return cudaSuccess;
    first_read_kernel<<<(unsigned)((nchunks + 255) / 256), 256, 0, s>>>(offsets, nreads, first,
                                                                         nchunks, chunk, first_read);
    return cudaGetLastError();
}

int insert_batch_blocks_per_sm(int kw, int chunk) {
    int n = 0;
    if (kw == 1 && chunk == 1024)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, insert_batch_kernel<1, 1024>, kInsertThreads, 0);
    else if (kw == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, insert_batch_kernel<1, 2048>, kInsertThreads, 0);
    else if (chunk == 1024)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, insert_batch_kernel<2, 1024>, kInsertThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, insert_batch_kernel<2, 2048>, kInsertThreads, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_window_bound_batch(const uint64_t *const *offsets, const uint64_t *nreads,
                                      int n, int K, void *out, uint64_t max_reads, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)n * sizeof(BoundOut), s);
    if (e != cudaSuccess || n == 0) return e;
    uint64_t bx = (max_reads + 255) / 256;
    if (bx > 256) bx = 256;
    if (bx == 0) bx = 1;
    window_bound_batch_kernel<<<dim3((unsigned)bx, (unsigned)n), 256, 0, s>>>(offsets, nreads, K,
                                                                              (BoundOut *)out);
    return cudaGetLastError();
}

cudaError_t launch_insert_batch(const InsertArgs *args, const unsigned long long *chunk_end,
                                int nsamples, unsigned long long total_chunks, int kw, int chunk,
                                int grid, cudaStream_t s) {
    if (total_chunks == 0) return cudaSuccess;
    first_read_batch_kernel<<<(unsigned)((total_chunks + 255) / 256), 256, 0, s>>>(
        args, chunk_end, nsamples, total_chunks, (uint64_t)chunk);
    const unsigned g = (unsigned)(total_chunks < (unsigned long long)grid ? total_chunks : grid);
    if (kw == 1 && chunk == 1024)
        insert_batch_kernel<1, 1024><<<g, kInsertThreads, 0, s>>>(args, chunk_end, nsamples, total_chunks);
    else if (kw == 1)
        insert_batch_kernel<1, 2048><<<g, kInsertThreads, 0, s>>>(args, chunk_end, nsamples, total_chunks);
    else if (chunk == 1024)
        insert_batch_kernel<2, 1024><<<g, kInsertThreads, 0, s>>>(args, chunk_end, nsamples, total_chunks);
    else
        insert_batch_kernel<2, 2048><<<g, kInsertThreads, 0, s>>>(args, chunk_end, nsamples, total_chunks);
    return cudaGetLastError();
}

cudaError_t launch_repartition(const PartArgs &p, cudaStream_t s) {
    const uint64_t tiles = (p.coarse_cap + kRepartTile - 1) / kRepartTile;
    if (tiles == 0) return cudaSuccess;
    if (p.coarse_shift - p.slice_shift > kMaxCoarseShift - kSliceShift ||
        p.coarse_shift <= p.slice_shift)
        return cudaErrorInvalidValue;
    const int smem = kRepartTile * (int)sizeof(uint32_t);
    const dim3 grid((unsigned)tiles, kCoarseBins);
    if (p.lane_codes && ((uint64_t)p.G.eta << p.slice_shift) > (uint64_t)kCountLanes)
        return cudaErrorInvalidValue;   // a lane must fit 16 bits
    // slices per coarse region: up to 64, 1,024 or kMaxFine (2,048)
    const int fbits = p.coarse_shift - p.slice_shift;
    void (*k)(PartArgs) =
        fbits <= 6    ? (p.lane_codes ? repartition_kernel<64, true> : repartition_kernel<64, false>)
        : fbits <= 10 ? (p.lane_codes ? repartition_kernel<1024, true>
                                      : repartition_kernel<1024, false>)
                      : (p.lane_codes ? repartition_kernel<kMaxFine, true>
                                      : repartition_kernel<kMaxFine, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kRepartThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_apply(const ApplyArgs &p, uint64_t nslices, cudaStream_t s) {
    if (nslices == 0) return cudaSuccess;
    if (p.lane_codes || p.cap % 4) return cudaErrorInvalidValue;   // 32-bit codes, 16-byte aligned
    const size_t smem = (size_t)8 << p.slice_shift;
    const bool half = 32 % p.G.alpha == 0;
    void (*k)(ApplyArgs) = p.G.cas_limit == kCasLimit
                               ? (half ? apply_kernel<false, true> : apply_kernel<false, false>)
                               : (half ? apply_kernel<true, true> : apply_kernel<true, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(8 << kSliceShift));
    if (e != cudaSuccess) return e;
    k<<<(unsigned)nslices, kCasApplyThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_apply_count(const ApplyArgs &p, uint64_t nslices, cudaStream_t s) {
    if (nslices == 0) return cudaSuccess;
    const size_t smem = ((size_t)p.G.eta << p.slice_shift) * 4;
    if (smem > (size_t)kCountLanes * 4 || p.G.alpha > 15) return cudaErrorInvalidValue;
    if (p.cap % (p.lane_codes ? 8 : 4)) return cudaErrorInvalidValue;   // 16-byte aligned slices
    void (*k)(ApplyArgs) = p.lane_codes ? apply_count_kernel<true> : apply_count_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kCountLanes * 4);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)nslices, kApplyThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_insert(const InsertArgs &a, int grid, int chunk, cudaStream_t s) {
    if (a.nchunks <= a.chunk_begin) return cudaSuccess;
    const uint64_t n = a.nchunks - a.chunk_begin;
    const uint64_t g = n < (uint64_t)grid ? n : (uint64_t)grid;
    const int part = !a.part ? 0 : a.coarse_shift <= 20 ? 1 : 2;
    if ((part ? kPartChunk : chunk) != chunk) return cudaErrorInvalidValue;
    return dispatch_insert(&a, a.K <= 32 ? 1 : 2, part, (unsigned)g, s, nullptr, chunk);
}

cudaError_t launch_reinsert(const uint64_t *keys, uint64_t n, int kw, uint64_t *table,
                            uint64_t cap, SetTag tag, uint64_t *dlist, uint64_t dlist_cap,
                            DevCounters *ctr, uint32_t probe_limit, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    if (kw == 1)
        reinsert_kernel<1><<<(unsigned)blocks, 256, 0, s>>>(keys, n, table, cap, tag, dlist, dlist_cap,
                                                             ctr, probe_limit);
    else
        reinsert_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(keys, n, table, cap, tag, dlist, dlist_cap,
                                                             ctr, probe_limit);
    return cudaGetLastError();
}

}  // namespace countbf

/*
 * KmerCo oracle: a plain, single-threaded CPU statement of what the countBF
 * K-mer counter computes (arXiv 2305.07545, KmerCo).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link
 * or call this file; only the test-suite, the smoke check and the timed CPU
 * baseline of the benchmark load it.  It shares no code, header, table or
 * constant generator with the CUDA library: every step below is written
 * again here from the paper's definitions, in the slow obvious way.
 *
 * Notation follows the paper (Table 1, Section 2.1):
 *   K      K-mer length                          (Table 1)
 *   k_h    number of hash functions  (nhash)     (Table 1)
 *   tau    trustworthiness threshold             (Table 1, Algorithm 2)
 *   alpha  counter bit length                    (Section 2.1)
 *   beta   cell bit length, fixed at 64          (Section 2.1)
 *   eta    counters per cell = floor(64 / alpha) (Section 2.1, supplement
 *          counter-length table)
 *   m      number of counters; W = ceil(m / eta) cells ("words")
 *
 * Readings of the paper adopted where it is silent or garbled (each one is
 * repeated beside the function that depends on it):
 *   - windows never cross read boundaries; a window holding any byte other
 *     than ACGT/acgt is skipped (Section 1.1 gives the window count
 *     len-K+1 per sequence);
 *   - canonical K-mer = the smaller of forward and reverse complement as
 *     2-bit packed integers, i.e. lexicographic order with A<C<G<T
 *     (Section 2.3, first sentence);
 *   - the hash family H_a is MurmurHash3_x64_128 with seed a (0-based),
 *     first 64-bit output (Section 3 names "murmur" without a variant);
 *   - flat addressing g = h mod m, cell g / eta, counter g mod eta
 *     (generalises Algorithm 3's i = h%x, j = h%y, l = h%eta);
 *   - a counter that would exceed 2^alpha - 1 stays at 2^alpha - 1 and the
 *     loop goes on with the next hash (Algorithm 3's overflow branch read
 *     per counter);
 *   - Algorithm 5 uses l = h mod eta (its "h % tau" is a typo);
 *   - est > tau is trustworthy, est <= tau erroneous (Table 1, Algorithm 2).
 *
 * Parity pins (tests that tie this code to something other than itself):
 *   murmur3_x64_128  the published SMHasher verification value and a
 *                    published test vector, plus an independent Python
 *                    implementation;
 *   extraction, RC   the worked examples of Section 1.1 (Fig. 1) and
 *                    Section 2.2, and brute force on ASCII strings;
 *   counters         the mask example of Section 2.1, the eta table of the
 *                    supplement, closed form == sequential Algorithm 3,
 *                    permutation and strand invariance;
 *   query / split    no-underestimate against exact counts, exact estimates
 *                    where no collision occurs, the tau boundary.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* MurmurHash3, x64 128-bit variant (Austin Appleby, public domain),         */
/* restated from its published description: 16-byte blocks mixed into two   */
/* 64-bit lanes, a tail of up to 15 bytes, then the 64-bit finaliser.        */
/* ------------------------------------------------------------------------ */

static uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

static uint64_t fmix64(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

static uint64_t load_le64(const uint8_t *p, int nbytes)
{
    uint64_t v = 0;
    for (int i = 0; i < nbytes; ++i) v |= (uint64_t)p[i] << (8 * i);
    return v;
}

void oracle_murmur3_x64_128(const uint8_t *data, uint64_t len, uint32_t seed,
                            uint64_t out[2])
{
    const uint64_t c1 = 0x87c37b91114253d5ULL;
    const uint64_t c2 = 0x4cf5ad432745937fULL;
    uint64_t h1 = seed, h2 = seed;
    uint64_t nblocks = len / 16;

    for (uint64_t b = 0; b < nblocks; ++b) {
        uint64_t k1 = load_le64(data + 16 * b, 8);
        uint64_t k2 = load_le64(data + 16 * b + 8, 8);

        k1 *= c1; k1 = rotl64(k1, 31); k1 *= c2; h1 ^= k1;
        h1 = rotl64(h1, 27); h1 += h2; h1 = h1 * 5 + 0x52dce729ULL;

        k2 *= c2; k2 = rotl64(k2, 33); k2 *= c1; h2 ^= k2;
        h2 = rotl64(h2, 31); h2 += h1; h2 = h2 * 5 + 0x38495ab5ULL;
    }

    /* Tail: bytes 8..14 form the second lane, bytes 0..7 the first. */
    const uint8_t *tail = data + 16 * nblocks;
    int rest = (int)(len & 15);
    if (rest > 8) {
        uint64_t k2 = load_le64(tail + 8, rest - 8);
        k2 *= c2; k2 = rotl64(k2, 33); k2 *= c1; h2 ^= k2;
    }
    if (rest > 0) {
        uint64_t k1 = load_le64(tail, rest > 8 ? 8 : rest);
        k1 *= c1; k1 = rotl64(k1, 31); k1 *= c2; h1 ^= k1;
    }

    h1 ^= len; h2 ^= len;
    h1 += h2; h2 += h1;
    h1 = fmix64(h1); h2 = fmix64(h2);
    h1 += h2; h2 += h1;
    out[0] = h1;
    out[1] = h2;
}

/* ------------------------------------------------------------------------ */
/* Bases and K-mers (Section 1.1, Section 2.2, Section 2.3)                  */
/* ------------------------------------------------------------------------ */

/* 2-bit code of a nucleotide: A=0, C=1, G=2, T=3 (upper or lower case);
 * -1 for anything else (N and the other IUPAC letters). */
int oracle_base_code(uint8_t c)
{
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    default: return -1;
    }
}

/* Pack a sequence of K codes into a 128-bit integer (hi, lo), first base
 * most significant: value = sum_i code_i * 4^(K-1-i). */
static void pack_codes(const int *codes, int K, uint64_t *hi, uint64_t *lo)
{
    uint64_t h = 0, l = 0;
    for (int i = 0; i < K; ++i) {
        h = (h << 2) | (l >> 62);
        l = (l << 2) | (uint64_t)codes[i];
    }
    *hi = h;
    *lo = l;
}

/* Reverse complement (Section 2.2): complement every base (A<->T, C<->G,
 * i.e. code -> 3 - code), then reverse the order. */
static void reverse_complement_codes(const int *codes, int K, int *rc)
{
    for (int i = 0; i < K; ++i) rc[K - 1 - i] = 3 - codes[i];
}

static int u128_less(uint64_t ahi, uint64_t alo, uint64_t bhi, uint64_t blo)
{
    return ahi < bhi || (ahi == bhi && alo < blo);
}

uint64_t oracle_kmer_hash(int K, uint64_t hi, uint64_t lo, uint32_t a);

/*
 * Window extraction (Section 1.1 / Fig. 1: a sequence of length len has
 * len-K+1 K-mers; Algorithm 1 takes each in turn), reverse complement and
 * canonical choice (Section 2.3).
 *
 * Reads are CSR: read r is bases[offsets[r] .. offsets[r+1]).  Every window
 * of K consecutive bases inside one read is visited in input order; with
 * whole_file != 0 the reads are instead taken as one sequence
 * bases[offsets[0] .. offsets[nreads]) and windows run across read
 * boundaries (the reading under which the paper's 55-mer totals are its
 * 28-mer totals minus 27).  A window with any non-ACGT byte is skipped and
 * counted in *n_skipped.  For each valid window the key is written to
 * hi[n], lo[n] when those are non-NULL:
 *   canonical == 0  the forward K-mer as read;
 *   canonical == 1  the smaller of forward and reverse complement as packed
 *                   integers (lexicographic, A < C < G < T);
 *   canonical == 2  the strand with the smaller hash H_0 -- Section 2.3's
 *                   equation with h = H_0: forward when
 *                   H_0(forward) < H_0(reverse complement), else the
 *                   reverse complement.
 * *n_windows receives the number of windows (sum over reads of
 * max(0, len-K+1)).  Returns the number of valid windows.
 */
uint64_t oracle_extract_ex(const uint8_t *bases, const uint64_t *offsets,
                           uint64_t nreads, int K, int canonical, int whole_file,
                           uint64_t *hi, uint64_t *lo,
                           uint64_t *n_windows, uint64_t *n_skipped)
{
    int codes[64], rc[64];
    uint64_t n = 0, windows = 0, skipped = 0;
    uint64_t nseq = whole_file ? (nreads > 0) : nreads;
    for (uint64_t r = 0; r < nseq; ++r) {
        uint64_t start = offsets[r], end = whole_file ? offsets[nreads] : offsets[r + 1];
        if (end < start + (uint64_t)K) continue;
        for (uint64_t p = start; p + (uint64_t)K <= end; ++p) {
            ++windows;
            int ok = 1;
            for (int i = 0; i < K; ++i) {
                codes[i] = oracle_base_code(bases[p + i]);
                if (codes[i] < 0) ok = 0;
            }
            if (!ok) { ++skipped; continue; }
            uint64_t fh, fl, rh, rl;
            pack_codes(codes, K, &fh, &fl);
            uint64_t kh = fh, kl = fl;
            if (canonical) {
                reverse_complement_codes(codes, K, rc);
                pack_codes(rc, K, &rh, &rl);
                int take_rc = canonical == 2
                    ? !(oracle_kmer_hash(K, fh, fl, 0) < oracle_kmer_hash(K, rh, rl, 0))
                    : u128_less(rh, rl, fh, fl);
                if (take_rc) { kh = rh; kl = rl; }
            }
            if (hi) hi[n] = kh;
            if (lo) lo[n] = kl;
            ++n;
        }
    }
    if (n_windows) *n_windows = windows;
    if (n_skipped) *n_skipped = skipped;
    return n;
}

/* Windows inside reads; canonical 0 (forward) or 1 (lexicographic). */
uint64_t oracle_extract(const uint8_t *bases, const uint64_t *offsets,
                        uint64_t nreads, int K, int canonical,
                        uint64_t *hi, uint64_t *lo,
                        uint64_t *n_windows, uint64_t *n_skipped)
{
    return oracle_extract_ex(bases, offsets, nreads, K, canonical, 0, hi, lo, n_windows,
                             n_skipped);
}

/*
 * H_a(K-mer) (Section 3; the hash step of Algorithm 3): MurmurHash3
 * x64_128 of the key's bytes with seed a, first output word.  Key bytes:
 * K <= 32 -> the 8 bytes of lo, little-endian; K > 32 -> the 8 bytes of lo
 * then the 8 bytes of hi, each little-endian.
 */
uint64_t oracle_kmer_hash(int K, uint64_t hi, uint64_t lo, uint32_t a)
{
    uint8_t bytes[16];
    int len = K <= 32 ? 8 : 16;
    for (int i = 0; i < 8; ++i) bytes[i] = (uint8_t)(lo >> (8 * i));
    for (int i = 0; i < 8; ++i) bytes[8 + i] = (uint8_t)(hi >> (8 * i));
    uint64_t out[2];
    oracle_murmur3_x64_128(bytes, (uint64_t)len, a, out);
    return out[0];
}

/* ------------------------------------------------------------------------ */
/* countBF (Section 2.1, Algorithms 3 and 5)                                 */
/* ------------------------------------------------------------------------ */

int oracle_eta(int alpha) { return 64 / alpha; }

uint64_t oracle_words(uint64_t m, int alpha)
{
    uint64_t eta = (uint64_t)oracle_eta(alpha);
    return (m + eta - 1) / eta;
}

/* Extract mask M^e_l of counter l (0-based; the paper's "1st counter" is
 * l = 0 and sits at the least significant bits, Section 2.1). */
uint64_t oracle_extract_mask(int alpha, int l)
{
    uint64_t ones = alpha == 64 ? ~0ULL : ((1ULL << alpha) - 1);
    return ones << (alpha * l);
}

/* Reset mask M^r_l = complement of the extract mask (Section 2.1). */
uint64_t oracle_reset_mask(int alpha, int l) { return ~oracle_extract_mask(alpha, l); }

/* Read counter l of cell w (Algorithm 3, extract-and-shift). */
static uint64_t read_counter(const uint64_t *filter, uint64_t w, int alpha, int l)
{
    return (filter[w] & oracle_extract_mask(alpha, l)) >> (alpha * l);
}

/*
 * Cell w and counter l that hash value h selects.
 *   Two-dimensional countBF of x * y cells (x > 0; Algorithm 3 as printed):
 *     i = h mod x, j = h mod y, l = h mod eta; the cell C[i][j] of the
 *     x-by-y array sits at w = i * y + j (row-major).
 *   Flat countBF of m counters (x == 0): g = h mod m, w = g / eta,
 *     l = g mod eta.  For x, y, eta pairwise coprime and m = x * y * eta the
 *     two are the same map up to relabelling (Chinese remainder theorem).
 */
static void address(uint64_t h, uint64_t m, uint64_t x, uint64_t y, int alpha,
                    uint64_t *w, int *l)
{
    uint64_t eta = (uint64_t)oracle_eta(alpha);
    if (x) {
        uint64_t i = h % x, j = h % y;
        *w = i * y + j;
        *l = (int)(h % eta);
    } else {
        uint64_t g = h % m;
        *w = g / eta;
        *l = (int)(g % eta);
    }
}

/*
 * Sequential IcountBF (Algorithm 3) applied to every key in input order.
 * For each hash a: the cell and counter of H_a(x) (address() above);
 * extract, add one, and write back with the reset mask -- unless the
 * counter already holds 2^alpha - 1, in which case it is left alone and the
 * loop continues with the next a (per-counter reading of the overflow
 * branch).  The filter is updated in place.
 */
static void insert_sequential(const uint64_t *hi, const uint64_t *lo, uint64_t n,
                              int K, uint64_t m, uint64_t dx, uint64_t dy, int alpha,
                              int nhash, uint64_t *filter)
{
    uint64_t maxc = (1ULL << alpha) - 1;
    for (uint64_t x = 0; x < n; ++x) {
        for (int a = 0; a < nhash; ++a) {
            uint64_t h = oracle_kmer_hash(K, hi[x], lo[x], (uint32_t)a);
            uint64_t w;
            int l;
            address(h, m, dx, dy, alpha, &w, &l);
            uint64_t value = read_counter(filter, w, alpha, l);
            if (value == maxc) continue; /* would overflow: stays saturated */
            value += 1;
            value <<= alpha * l;
            filter[w] = (filter[w] & oracle_reset_mask(alpha, l)) | value;
        }
    }
}

/* Flat countBF of m counters. */
void oracle_insert_sequential(const uint64_t *hi, const uint64_t *lo, uint64_t n,
                              int K, uint64_t m, int alpha, int nhash,
                              uint64_t *filter)
{
    insert_sequential(hi, lo, n, K, m, 0, 0, alpha, nhash, filter);
}

/* Two-dimensional countBF of dx * dy cells. */
void oracle_insert_sequential_2d(const uint64_t *hi, const uint64_t *lo, uint64_t n,
                                 int K, uint64_t dx, uint64_t dy, int alpha, int nhash,
                                 uint64_t *filter)
{
    insert_sequential(hi, lo, n, K, 0, dx, dy, alpha, nhash, filter);
}

/*
 * The same filter by its closed form: counter g holds
 *     min(2^alpha - 1, #{(x, a) : x in S, a < k_h, H_a(x) mod m == g}),
 * packed at cell g / eta, bits alpha*(g mod eta).  counts must hold m
 * zero-initialised 32-bit slots (scratch); filter receives W words.
 */
void oracle_counters_closed_form(const uint64_t *hi, const uint64_t *lo, uint64_t n,
                                 int K, uint64_t m, int alpha, int nhash,
                                 uint32_t *counts, uint64_t *filter)
{
    uint64_t eta = (uint64_t)oracle_eta(alpha);
    uint64_t maxc = (1ULL << alpha) - 1;
    for (uint64_t x = 0; x < n; ++x)
        for (int a = 0; a < nhash; ++a)
            counts[oracle_kmer_hash(K, hi[x], lo[x], (uint32_t)a) % m] += 1;
    uint64_t W = oracle_words(m, alpha);
    for (uint64_t w = 0; w < W; ++w) filter[w] = 0;
    for (uint64_t g = 0; g < m; ++g) {
        uint64_t c = counts[g] < maxc ? counts[g] : maxc;
        filter[g / eta] |= c << (alpha * (int)(g % eta));
    }
}

/*
 * QcountBF-II (Algorithm 5): for each a read counter H_a(x) mod m; return
 * 0 as soon as one is zero, otherwise the minimum over a.
 */
static uint64_t query(const uint64_t *filter, int K, uint64_t hi, uint64_t lo, uint64_t m,
                      uint64_t dx, uint64_t dy, int alpha, int nhash)
{
    uint64_t best = ~0ULL;
    for (int a = 0; a < nhash; ++a) {
        uint64_t w;
        int l;
        address(oracle_kmer_hash(K, hi, lo, (uint32_t)a), m, dx, dy, alpha, &w, &l);
        uint64_t value = read_counter(filter, w, alpha, l);
        if (value == 0) return 0;
        if (value < best) best = value;
    }
    return best;
}

uint64_t oracle_query(const uint64_t *filter, int K, uint64_t hi, uint64_t lo,
                      uint64_t m, int alpha, int nhash)
{
    return query(filter, K, hi, lo, m, 0, 0, alpha, nhash);
}

uint64_t oracle_query_2d(const uint64_t *filter, int K, uint64_t hi, uint64_t lo,
                         uint64_t dx, uint64_t dy, int alpha, int nhash)
{
    return query(filter, K, hi, lo, 0, dx, dy, alpha, nhash);
}

/*
 * Sequential distinct count of Algorithm 1: keys are taken in input order;
 * a key whose query (Algorithm 5 on the canonical key) returns 0 before its
 * own insertion counts as first seen.  Order dependent and an undercount
 * through false positives; reported, not used for parity.  filter must be
 * zero on entry and ends equal to the sequential Algorithm 3 result.
 */
uint64_t oracle_seq_distinct(const uint64_t *hi, const uint64_t *lo, uint64_t n,
                             int K, uint64_t m, int alpha, int nhash,
                             uint64_t *filter)
{
    uint64_t first_seen = 0;
    for (uint64_t x = 0; x < n; ++x) {
        if (oracle_query(filter, K, hi[x], lo[x], m, alpha, nhash) == 0) ++first_seen;
        oracle_insert_sequential(hi + x, lo + x, 1, K, m, alpha, nhash, filter);
    }
    return first_seen;
}

/* ------------------------------------------------------------------------ */
/* Distinct K-mers and classification (Algorithm 2)                          */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t hi, lo; } key128;

static int cmp_key128(const void *pa, const void *pb)
{
    const key128 *a = (const key128 *)pa, *b = (const key128 *)pb;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    return 0;
}

/*
 * Exact distinct K-mers: sort all keys ascending (as 128-bit integers) and
 * keep one of each run.  Writes the D distinct keys to dhi/dlo and, when
 * counts is non-NULL, the run length (exact frequency) of each.  Returns D.
 */
uint64_t oracle_distinct(const uint64_t *hi, const uint64_t *lo, uint64_t n,
                         uint64_t *dhi, uint64_t *dlo, uint64_t *counts)
{
    if (n == 0) return 0;
    key128 *k = (key128 *)malloc(n * sizeof(key128));
    if (!k) return ~0ULL;
    for (uint64_t i = 0; i < n; ++i) { k[i].hi = hi[i]; k[i].lo = lo[i]; }
    qsort(k, n, sizeof(key128), cmp_key128);
    uint64_t d = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (d > 0 && k[i].hi == dhi[d - 1] && k[i].lo == dlo[d - 1]) {
            if (counts) counts[d - 1] += 1;
            continue;
        }
        dhi[d] = k[i].hi;
        dlo[d] = k[i].lo;
        if (counts) counts[d] = 1;
        ++d;
    }
    free(k);
    return d;
}

/*
 * QueryKmerCo (Algorithm 2) over the distinct keys, in their order: est[i]
 * = QcountBF-II of key i; trusted[i] = 1 when est[i] > tau (frequency
 * "more than" tau), else 0 (erroneous).  Returns the number trusted.
 */
static uint64_t classify(const uint64_t *filter, const uint64_t *dhi, const uint64_t *dlo,
                         uint64_t d, int K, uint64_t m, uint64_t dx, uint64_t dy, int alpha,
                         int nhash, uint64_t tau, uint64_t *est, uint8_t *trusted)
{
    uint64_t t = 0;
    for (uint64_t i = 0; i < d; ++i) {
        est[i] = query(filter, K, dhi[i], dlo[i], m, dx, dy, alpha, nhash);
        trusted[i] = est[i] > tau;
        t += trusted[i];
    }
    return t;
}

uint64_t oracle_classify(const uint64_t *filter, const uint64_t *dhi, const uint64_t *dlo,
                         uint64_t d, int K, uint64_t m, int alpha, int nhash,
                         uint64_t tau, uint64_t *est, uint8_t *trusted)
{
    return classify(filter, dhi, dlo, d, K, m, 0, 0, alpha, nhash, tau, est, trusted);
}

uint64_t oracle_classify_2d(const uint64_t *filter, const uint64_t *dhi, const uint64_t *dlo,
                            uint64_t d, int K, uint64_t dx, uint64_t dy, int alpha, int nhash,
                            uint64_t tau, uint64_t *est, uint8_t *trusted)
{
    return classify(filter, dhi, dlo, d, K, 0, dx, dy, alpha, nhash, tau, est, trusted);
}

/*
 * Merge of two filters built over disjoint parts of the input: every
 * counter becomes min(a + b, 2^alpha - 1).  Because
 * min(min(c1, M) + min(c2, M), M) = min(c1 + c2, M), the merge of shards
 * equals the filter of the whole input.  Counter by counter, in place in dst.
 */
void oracle_merge(uint64_t *dst, const uint64_t *src, uint64_t m, int alpha)
{
    uint64_t eta = (uint64_t)oracle_eta(alpha);
    uint64_t maxc = (1ULL << alpha) - 1;
    for (uint64_t g = 0; g < m; ++g) {
        uint64_t w = g / eta;
        int l = (int)(g % eta);
        uint64_t s = read_counter(dst, w, alpha, l) + read_counter(src, w, alpha, l);
        if (s > maxc) s = maxc;
        dst[w] = (dst[w] & oracle_reset_mask(alpha, l)) | (s << (alpha * l));
    }
}

/* ------------------------------------------------------------------------ */
/* countBF sizing (Section 2.1, Eq. 1)                                       */
/* ------------------------------------------------------------------------ */

static int is_prime(uint64_t p)
{
    if (p < 2) return 0;
    for (uint64_t d = 2; d * d <= p; ++d)
        if (p % d == 0) return 0;
    return 1;
}

/*
 * Eq. 1: the standard Bloom filter size for n items at false positive
 * probability fpp is m = -n ln(fpp) / (ln 2)^2 bits; v = sqrt(m / 128);
 * X is the smallest prime greater than v and Y the third prime after X
 * (counting X's successors in the sequence of primes).  The countBF then
 * holds X * Y cells of beta = 64 bits.  Returns 0, or -1 for bad input.
 */
int oracle_paper_dims(uint64_t n, double fpp, uint64_t *X, uint64_t *Y)
{
    if (n == 0 || !(fpp > 0.0 && fpp < 1.0)) return -1;
    double m = -(double)n * log(fpp) / (log(2.0) * log(2.0));
    double v = sqrt(m / 128.0);
    uint64_t x = (uint64_t)v;
    while ((double)x <= v || !is_prime(x)) ++x;
    uint64_t y = x;
    int primes_after = 0;
    while (primes_after < 3) {
        ++y;
        if (is_prime(y)) ++primes_after;
    }
    *X = x;
    *Y = y;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 as printed (diagnostic; not a parity target)                 */
/* ------------------------------------------------------------------------ */

/* Packed value of K codes read from ASCII bases (all valid). */
static void pack_bases(const uint8_t *p, int K, int rc, uint64_t *hi, uint64_t *lo)
{
    int codes[64], r[64];
    for (int i = 0; i < K; ++i) codes[i] = oracle_base_code(p[i]);
    if (rc) {
        reverse_complement_codes(codes, K, r);
        pack_codes(r, K, hi, lo);
    } else {
        pack_codes(codes, K, hi, lo);
    }
}

/*
 * The insertion phase exactly as Algorithms 1, 3 and 4 print it, in input
 * order, with the paper's state-dependent choices kept:
 *   QcountBF-I (Algorithm 4): for a = 1..k_h compare H_a(Read) with
 *     H_a(Read_RC); Result = 0 when H_a(Read) < H_a(Read_RC), else 1; read
 *     the counter of the smaller hash and return 0 at once when it is 0;
 *     otherwise the minimum.  Result is the one of the last iteration run.
 *   Algorithm 1: the strand Result names is inserted; when the query
 *     returned 0 it is also appended to the distinct list (first seen).
 *   IcountBF (Algorithm 3): for a = 1..k_h the counter of H_a(key) is
 *     incremented, and the whole insertion stops at the first counter
 *     that cannot take one more (value + 1 > 2^alpha - 1; "Counter
 *     Overflow, return").
 * Hash index a = 1..k_h is seed a - 1 (the seeds of H_a elsewhere).
 * Flat (dx == 0, m counters) or two-dimensional (dx x dy cells) geometry.
 * Windows stay inside reads; windows with non-ACGT bytes are skipped.
 * Keys appended to the distinct list go to dhi/dlo (may be NULL).  Returns
 * the number of first-seen windows.
 */
uint64_t oracle_literal_insertion(const uint8_t *bases, const uint64_t *offsets,
                                  uint64_t nreads, int K, uint64_t m, uint64_t dx,
                                  uint64_t dy, int alpha, int nhash, uint64_t *filter,
                                  uint64_t *dhi, uint64_t *dlo)
{
    uint64_t maxc = (1ULL << alpha) - 1, first_seen = 0;
    for (uint64_t r = 0; r < nreads; ++r) {
        for (uint64_t p = offsets[r]; p + (uint64_t)K <= offsets[r + 1]; ++p) {
            int ok = 1;
            for (int i = 0; i < K; ++i)
                if (oracle_base_code(bases[p + i]) < 0) ok = 0;
            if (!ok) continue;
            uint64_t fh, fl, rh, rl;
            pack_bases(bases + p, K, 0, &fh, &fl);
            pack_bases(bases + p, K, 1, &rh, &rl);
            /* QcountBF-I */
            int result = 0;
            uint64_t freq = ~0ULL;
            for (int a = 0; a < nhash; ++a) {
                uint64_t h = oracle_kmer_hash(K, fh, fl, (uint32_t)a);
                uint64_t h1 = oracle_kmer_hash(K, rh, rl, (uint32_t)a);
                if (h < h1) {
                    result = 0;
                } else {
                    h = h1;
                    result = 1;
                }
                uint64_t w;
                int l;
                address(h, m, dx, dy, alpha, &w, &l);
                uint64_t value = read_counter(filter, w, alpha, l);
                if (value == 0) { freq = 0; break; }
                if (value < freq) freq = value;
            }
            uint64_t kh = result ? rh : fh, kl = result ? rl : fl;
            if (freq == 0) {
                if (dhi) dhi[first_seen] = kh;
                if (dlo) dlo[first_seen] = kl;
                ++first_seen;
            }
            /* IcountBF */
            for (int a = 0; a < nhash; ++a) {
                uint64_t w;
                int l;
                address(oracle_kmer_hash(K, kh, kl, (uint32_t)a), m, dx, dy, alpha, &w, &l);
                uint64_t value = read_counter(filter, w, alpha, l);
                if (value + 1 > maxc) break; /* counter overflow: insertion ends */
                filter[w] = (filter[w] & oracle_reset_mask(alpha, l)) |
                            ((value + 1) << (alpha * l));
            }
        }
    }
    return first_seen;
}

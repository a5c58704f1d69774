/*
 * Seeded synthetic corpora for the blockwise absolute-offset LZ77 decoder.
 *
 * This module holds no decoder or encoder arithmetic: it only produces input
 * bytes.  Both the CPU oracle and the GPU library are fed from it, so neither
 * depends on the other for inputs.
 *
 * Random numbers: splitmix64 seeds xoshiro256**, both written from their
 * published definitions (Vigna, "Further scramblings of Marsaglia's xorshift
 * generators", and the splitmix64 finaliser of Steele et al.).
 *
 * The corpora stand in for the paper's genome (chr1) and text corpora, which
 * are not available here (paper, Setup and Reproducibility sections).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t* x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_seed(rng_t* r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rng_next(rng_t* r) {
    uint64_t* s = r->s;
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_unif(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [lo, hi] (inclusive); the modulo bias is below 2^-40 for
 * the small ranges used here */
static inline uint64_t rng_range(rng_t* r, uint64_t lo, uint64_t hi) {
    return lo + rng_next(r) % (hi - lo + 1);
}

/*
 * Deterministic elementary functions.  libm's exp/log/cos/pow may differ in
 * the last unit in the last place between C libraries and CPU
 * architectures; the corpora must be byte-identical on every host, so these
 * use only IEEE +, -, *, / and sqrt (all correctly rounded) in a fixed
 * order.  Accuracy is about 1e-15 relative, ample for a workload generator.
 */
static double det_log(double x) {
    /* x = m * 2^e with m in [sqrt(1/2), sqrt(2)); log(m) = 2 atanh(z), z = (m-1)/(m+1) */
    int e = 0;
    double m = frexp(x, &e); /* exact: m in [0.5, 1) */
    if (m < 0.7071067811865476) { m *= 2.0; e -= 1; }
    double z = (m - 1.0) / (m + 1.0), z2 = z * z, term = z, sum = 0.0;
    for (int k = 1; k < 60; k += 2) { sum += term / (double)k; term *= z2; }
    return 2.0 * sum + (double)e * 0.6931471805599453;
}

static double det_exp(double x) {
    /* x = k ln2 + r, |r| <= ln2/2; exp(r) by its Taylor series */
    double kf = floor(x / 0.6931471805599453 + 0.5);
    double r = x - kf * 0.6931471805599453;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; k++) { term *= r / (double)k; sum += term; }
    return ldexp(sum, (int)kf);
}

static double det_cos(double x) {
    /* x in [0, 2 pi): fold to [0, pi/2] and use the Taylor series */
    const double PI = 3.141592653589793;
    double sign = 1.0;
    if (x > PI) x = 2.0 * PI - x;
    if (x > PI / 2) { x = PI - x; sign = -1.0; }
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int k = 1; k < 20; k++) { term *= -x2 / (double)((2 * k - 1) * (2 * k)); sum += term; }
    return sign * sum;
}

static double rng_normal(rng_t* r) {
    double u1 = rng_unif(r), u2 = rng_unif(r);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * det_log(u1)) * det_cos(6.283185307179586 * u2);
}

uint64_t synth_splitmix64(uint64_t seed, uint64_t* out, uint64_t n) {
    uint64_t x = seed;
    for (uint64_t i = 0; i < n; i++) out[i] = splitmix64_next(&x);
    return n;
}

uint64_t synth_xoshiro256ss(uint64_t seed, uint64_t* out, uint64_t n) {
    rng_t r;
    rng_seed(&r, seed);
    for (uint64_t i = 0; i < n; i++) out[i] = rng_next(&r);
    return n;
}

static const uint8_t BASES[4] = {'A', 'C', 'G', 'T'};

/* Per-event statistics the generator reports back (for tests). */
typedef struct {
    uint64_t n_bytes_random, n_bytes_nrun, n_bytes_copy, n_bytes_tandem;
    uint64_t n_copies, n_tandems, n_nruns, n_mutations;
} synth_dna_stats;

/*
 * DNA-like genome.  Left-to-right walk: random-base gaps (geometric) between
 * events; an event is an 'N' run (length U[10,1000]), a copy of an earlier
 * span (length lognormal(ln 7, 1) clipped to [4, 4096], distance log-uniform
 * in [len, pos], 1% point mutations to a different base), or a tandem repeat
 * (period U[1,12], length U[20,200], periodic fill).  Target coverage of the
 * output: n_frac in 'N' runs, copy_frac in copies, tandem_frac in tandem
 * repeats; the remainder is uniform {A,C,G,T}.
 */
int synth_dna(uint8_t* out, uint64_t n, uint64_t seed, double n_frac, double copy_frac,
              double tandem_frac, synth_dna_stats* st) {
    if (!out && n) return -1;
    synth_dna_stats s;
    memset(&s, 0, sizeof s);
    rng_t r;
    rng_seed(&r, seed);
    /* mean event lengths: N-run U[10,1000] -> 505; copy lognormal(ln7,1)
     * clipped -> about 11.4; tandem U[20,200] -> 110 */
    const double mean_n = 505.0, mean_copy = 11.4, mean_tandem = 110.0;
    double rate_n = n_frac / mean_n, rate_c = copy_frac / mean_copy, rate_t = tandem_frac / mean_tandem;
    double rate = rate_n + rate_c + rate_t;
    double frac_random = 1.0 - n_frac - copy_frac - tandem_frac;
    if (frac_random < 0.0) frac_random = 0.0;
    double mean_gap = rate > 0.0 ? frac_random / rate : (double)n;
    double p_n = rate > 0.0 ? rate_n / rate : 0.0, p_c = rate > 0.0 ? rate_c / rate : 0.0;
    /* geometric gap with the requested mean: P(stop) = 1/(1+mean) per byte */
    double q_gap = mean_gap > 0.0 ? 1.0 / (1.0 + mean_gap) : 1.0;
    double log1m_q = det_log(1.0 - q_gap);
    uint64_t pos = 0;
    uint64_t bits = 0;
    int nbits = 0;
    while (pos < n) {
        /* random gap */
        uint64_t gap;
        if (q_gap >= 1.0) gap = 0;
        else {
            double u = rng_unif(&r);
            if (u < 1e-300) u = 1e-300;
            gap = (uint64_t)floor(det_log(u) / log1m_q);
        }
        if (gap > n - pos) gap = n - pos;
        for (uint64_t k = 0; k < gap; k++) {
            if (nbits == 0) { bits = rng_next(&r); nbits = 32; }
            out[pos++] = BASES[bits & 3];
            bits >>= 2;
            nbits--;
        }
        s.n_bytes_random += gap;
        if (pos >= n) break;
        double u = rng_unif(&r);
        if (u < p_n) {
            uint64_t len = rng_range(&r, 10, 1000);
            if (len > n - pos) len = n - pos;
            memset(out + pos, 'N', len);
            pos += len;
            s.n_bytes_nrun += len;
            s.n_nruns++;
        } else if (u < p_n + p_c) {
            double L = det_exp(det_log(7.0) + rng_normal(&r));
            uint64_t len = (uint64_t)floor(L + 0.5);
            if (len < 4) len = 4;
            if (len > 4096) len = 4096;
            if (len > n - pos) len = n - pos;
            if (pos < len || len == 0) continue; /* no earlier span long enough yet */
            /* distance log-uniform in [len, pos] */
            double lo = det_log((double)len), hi = det_log((double)pos);
            uint64_t dist = (uint64_t)floor(det_exp(lo + (hi - lo) * rng_unif(&r)));
            if (dist < len) dist = len;
            if (dist > pos) dist = pos;
            uint64_t src = pos - dist;
            for (uint64_t k = 0; k < len; k++) {
                uint8_t c = out[src + k];
                if (rng_unif(&r) < 0.01) {
                    uint8_t m;
                    do { m = BASES[rng_next(&r) & 3]; } while (m == c);
                    c = m;
                    s.n_mutations++;
                }
                out[pos + k] = c;
            }
            pos += len;
            s.n_bytes_copy += len;
            s.n_copies++;
        } else {
            uint64_t period = rng_range(&r, 1, 12);
            uint64_t len = rng_range(&r, 20, 200);
            if (len > n - pos) len = n - pos;
            uint8_t unit[12];
            for (uint64_t k = 0; k < period; k++) unit[k] = BASES[rng_next(&r) & 3];
            for (uint64_t k = 0; k < len; k++) out[pos + k] = unit[k % period];
            pos += len;
            s.n_bytes_tandem += len;
            s.n_tandems++;
        }
    }
    if (st) *st = s;
    return 0;
}

/* ---- text ---------------------------------------------------------------- */

typedef struct {
    uint64_t n_sentences, n_repeated, n_words;
} synth_text_stats;

static uint64_t word_hash(const uint8_t* w, int len) {
    uint64_t h = 1469598103934665603ULL;
    for (int i = 0; i < len; i++) { h ^= w[i]; h *= 1099511628211ULL; }
    return h;
}

/*
 * Zipf text: a vocabulary of n_vocab distinct words (length U[2,12], letters
 * U[a-z]); word rank k drawn with probability proportional to k^-zipf_s;
 * sentences of U[5,25] words separated by spaces and ended by ". "; with
 * probability p_repeat a sentence is a verbatim copy of a uniformly chosen
 * earlier sentence.
 */
int synth_text(uint8_t* out, uint64_t n, uint64_t seed, uint32_t n_vocab, double zipf_s, double p_repeat,
               synth_text_stats* st) {
    if (!out && n) return -1;
    if (n_vocab == 0) return -1;
    synth_text_stats s;
    memset(&s, 0, sizeof s);
    rng_t r;
    rng_seed(&r, seed);
    uint8_t* words = (uint8_t*)malloc((size_t)n_vocab * 12);
    uint8_t* wlen = (uint8_t*)malloc(n_vocab);
    double* cdf = (double*)malloc(sizeof(double) * n_vocab);
    uint64_t hcap = 1;
    while (hcap < (uint64_t)n_vocab * 4) hcap <<= 1;
    uint64_t* htab = (uint64_t*)calloc(hcap, sizeof(uint64_t)); /* stores index+1 */
    uint64_t sent_cap = 1024, n_sent = 0;
    uint64_t* sent_off = (uint64_t*)malloc(sent_cap * sizeof(uint64_t));
    uint32_t* sent_len = (uint32_t*)malloc(sent_cap * sizeof(uint32_t));
    if (!words || !wlen || !cdf || !htab || !sent_off || !sent_len) {
        free(words); free(wlen); free(cdf); free(htab); free(sent_off); free(sent_len);
        return -3;
    }
    for (uint32_t i = 0; i < n_vocab;) {
        int len = (int)rng_range(&r, 2, 12);
        uint8_t* w = words + (size_t)i * 12;
        for (int k = 0; k < len; k++) w[k] = (uint8_t)('a' + rng_range(&r, 0, 25));
        uint64_t h = word_hash(w, len), slot = h & (hcap - 1);
        int dup = 0;
        while (htab[slot]) {
            uint64_t j = htab[slot] - 1;
            if (wlen[j] == len && memcmp(words + j * 12, w, (size_t)len) == 0) { dup = 1; break; }
            slot = (slot + 1) & (hcap - 1);
        }
        if (dup) continue;
        htab[slot] = (uint64_t)i + 1;
        wlen[i] = (uint8_t)len;
        i++;
    }
    double acc = 0.0;
    for (uint32_t k = 0; k < n_vocab; k++) { acc += det_exp(-zipf_s * det_log((double)(k + 1))); cdf[k] = acc; }
    for (uint32_t k = 0; k < n_vocab; k++) cdf[k] /= acc;
    uint64_t pos = 0;
    while (pos < n) {
        uint64_t start = pos;
        if (n_sent > 0 && rng_unif(&r) < p_repeat) {
            uint64_t j = rng_range(&r, 0, n_sent - 1);
            uint64_t len = sent_len[j];
            if (len > n - pos) len = n - pos;
            memmove(out + pos, out + sent_off[j], len); /* source lies before pos: no overlap */
            pos += len;
            s.n_repeated++;
        } else {
            uint64_t nw = rng_range(&r, 5, 25);
            for (uint64_t k = 0; k < nw && pos < n; k++) {
                double u = rng_unif(&r);
                uint32_t lo = 0, hi = n_vocab - 1;
                while (lo < hi) {
                    uint32_t mid = (lo + hi) / 2;
                    if (cdf[mid] > u) hi = mid; else lo = mid + 1;
                }
                const uint8_t* w = words + (size_t)lo * 12;
                for (int c = 0; c < wlen[lo] && pos < n; c++) out[pos++] = w[c];
                if (k + 1 < nw && pos < n) out[pos++] = ' ';
                s.n_words++;
            }
            if (pos < n) out[pos++] = '.';
            if (pos < n) out[pos++] = ' ';
        }
        if (n_sent == sent_cap) {
            sent_cap *= 2;
            uint64_t* o2 = (uint64_t*)realloc(sent_off, sent_cap * sizeof(uint64_t));
            uint32_t* l2 = (uint32_t*)realloc(sent_len, sent_cap * sizeof(uint32_t));
            if (!o2 || !l2) { free(o2 ? o2 : sent_off); free(l2 ? l2 : sent_len); free(words); free(wlen); free(cdf); free(htab); return -3; }
            sent_off = o2;
            sent_len = l2;
        }
        sent_off[n_sent] = start;
        sent_len[n_sent] = (uint32_t)(pos - start);
        n_sent++;
        s.n_sentences++;
    }
    free(words); free(wlen); free(cdf); free(htab); free(sent_off); free(sent_len);
    if (st) *st = s;
    return 0;
}

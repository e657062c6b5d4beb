/*
 * synth.c -- seeded synthetic key columns shaped like the paper's workloads.
 *
 * These generators only PRODUCE inputs; they hold none of the compressed key
 * sort's arithmetic.  Both the CPU oracle tests and the CUDA path (tests and
 * bench) draw their inputs from here.
 *
 * Randomness is counter-based so that any row can be generated independently
 * and the result does not depend on the thread count: every draw is
 *   mix64(base(seed, stream) + (i + 1) * 0x9E3779B97F4A7C15)
 * where mix64 is the finaliser of SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t base_of(uint64_t seed, uint64_t stream) {
    return mix64(seed * 0x9E3779B97F4A7C15ull ^ mix64(stream + 0x632BE59BD9B4E019ull));
}

static inline uint64_t draw(uint64_t base, uint64_t i) {
    return mix64(base + (i + 1) * 0x9E3779B97F4A7C15ull);
}

/* uniform double in [0, 1) */
static inline double unif(uint64_t base, uint64_t i) {
    return (double)(draw(base, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* uniform integer in [0, m) */
static inline uint64_t below(uint64_t base, uint64_t i, uint64_t m) {
    return (uint64_t)(unif(base, i) * (double)m);
}

uint64_t synth_draw(uint64_t seed, uint64_t stream, uint64_t i) { return draw(base_of(seed, stream), i); }

int synth_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- Zipf(s) over {1..N}: inverse CDF table for moderate N ---------------- */
static double* zipf_cdf(uint64_t N, double s) {
    double* cdf = (double*)malloc(sizeof(double) * N);
    double acc = 0.0;
    for (uint64_t k = 1; k <= N; ++k) { acc += pow((double)k, -s); cdf[k - 1] = acc; }
    for (uint64_t k = 0; k < N; ++k) cdf[k] /= acc;
    cdf[N - 1] = 1.0;
    return cdf;
}

static uint64_t zipf_pick(const double* cdf, uint64_t N, double u) {  /* 0-based rank */
    uint64_t lo = 0, hi = N - 1;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (cdf[mid] >= u) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* Draws n ranks (0-based) from Zipf(s) over N values with the table method. */
void synth_zipf_table(uint64_t n, uint64_t seed, uint64_t N, double s, uint32_t* out) {
    double* cdf = zipf_cdf(N, s);
    uint64_t b = base_of(seed, 11);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = (uint32_t)zipf_pick(cdf, N, unif(b, (uint64_t)i));
    free(cdf);
}

/* ---- Zipf(s) over {1..N} for huge N: rejection-inversion ------------------
 * W. Hormann and G. Derflinger, "Rejection-inversion to generate variates from
 * monotone discrete distributions", ACM TOMACS 6(3), 1996.  With h(x) = x^-s
 * and its antiderivative H(x) = (x^(1-s) - 1)/(1-s) (log x at s = 1), draw u
 * uniformly on [H(1.5) - 1, H(N + 0.5)], take x = H^-1(u), k = round(x), and
 * accept k when u >= H(k + 0.5) - h(k); the quick test k - x <= c accepts
 * without evaluating H. */
static double zH(double x, double s) {
    double lx = log(x), t = (1.0 - s) * lx;
    return fabs(t) > 1e-8 ? expm1(t) / (1.0 - s) : lx * (1.0 + 0.5 * t);
}
static double zHinv(double u, double s) {
    double t = u * (1.0 - s);
    return fabs(t) > 1e-8 ? exp(log1p(t) / (1.0 - s)) : exp(u * (1.0 - 0.5 * t));
}

void synth_zipf_rejinv(uint64_t n, uint64_t seed, double N, double s, uint64_t* out) {
    double lo = zH(1.5, s) - 1.0, hi = zH(N + 0.5, s);
    double c = 2.0 - zHinv(zH(2.5, s) - pow(2.0, -s), s);
    uint64_t b = base_of(seed, 12);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        for (uint64_t t = 0;; ++t) {
            double u = lo + unif(b, (uint64_t)i + t * n) * (hi - lo);
            double x = zHinv(u, s);
            double kd = floor(x + 0.5);
            if (kd < 1.0) kd = 1.0;
            if (kd > N) kd = N;
            if (kd - x <= c || u >= zH(kd + 0.5, s) - pow(kd, -s)) { out[i] = (uint64_t)kd; break; }
        }
    }
}

/* ---- integer column: 24 varying positions in a fixed 64-bit pattern -------
 * positions: 24 distinct bit positions of 0..63 (0 = most significant bit),
 * chosen by a seeded partial Fisher-Yates shuffle; the other 40 bits are a
 * seeded fixed pattern; the chosen bits are i.i.d. uniform per row. */
void synth_varying_bits_u64(uint64_t n, uint64_t seed, uint32_t nvary, uint32_t* positions, uint64_t* out) {
    uint32_t pool[64];
    for (uint32_t i = 0; i < 64; ++i) pool[i] = i;
    uint64_t bp = base_of(seed, 1);
    for (uint32_t i = 0; i < nvary; ++i) {
        uint32_t j = i + (uint32_t)below(bp, i, 64 - i);
        uint32_t t = pool[i]; pool[i] = pool[j]; pool[j] = t;
        positions[i] = pool[i];
    }
    uint64_t M = 0;
    for (uint32_t i = 0; i < nvary; ++i) M |= 1ull << (63 - positions[i]);
    uint64_t pattern = synth_draw(seed, 2, 0) & ~M;
    uint64_t b = base_of(seed, 3);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t r = draw(b, (uint64_t)i), v = pattern, m = M;
        while (m) {                          /* deposit low bits of r into the set bits of M */
            uint64_t low = m & (~m + 1);
            if (r & 1) v |= low;
            r >>= 1;
            m &= m - 1;
        }
        out[i] = v;
    }
}

/* ---- URL-like keys: "http://www." + name + ".com/" + path ----------------
 * nnames names of 4..12 lowercase letters; the name of each row is Zipf(s)
 * over the names; the path is 0..16 characters from [a-z0-9/].  The string is
 * truncated to W bytes and zero padded. */
void synth_urls(uint64_t n, uint64_t seed, uint32_t W, uint32_t nnames, double s, uint8_t* out) {
    char* names = (char*)malloc((size_t)nnames * 13);
    uint8_t* nlen = (uint8_t*)malloc(nnames);
    uint64_t bn = base_of(seed, 4);
    for (uint32_t k = 0; k < nnames; ++k) {
        nlen[k] = (uint8_t)(4 + below(bn, (uint64_t)k * 16, 9));
        for (uint32_t c = 0; c < nlen[k]; ++c) names[k * 13 + c] = (char)('a' + below(bn, (uint64_t)k * 16 + 1 + c, 26));
    }
    double* cdf = zipf_cdf(nnames, s);
    static const char alpha[] = "abcdefghijklmnopqrstuvwxyz0123456789/";
    uint64_t bz = base_of(seed, 5), bl = base_of(seed, 6), bc = base_of(seed, 7);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        char buf[64];
        uint32_t len = 0;
        memcpy(buf, "http://www.", 11); len = 11;
        uint64_t k = zipf_pick(cdf, nnames, unif(bz, (uint64_t)i));
        memcpy(buf + len, names + k * 13, nlen[k]); len += nlen[k];
        memcpy(buf + len, ".com/", 5); len += 5;
        uint32_t plen = (uint32_t)below(bl, (uint64_t)i, 17);
        uint64_t r = draw(bc, (uint64_t)i), r2 = draw(bc, (uint64_t)i + 0x8000000000000000ull);
        for (uint32_t c = 0; c < plen; ++c) {
            uint64_t src = (c < 10) ? r : r2;
            buf[len++] = alpha[(src >> (6 * (c % 10))) % 37];
        }
        uint8_t* row = out + (uint64_t)i * W;
        uint32_t take = len < W ? len : W;
        memcpy(row, buf, take);
        memset(row + take, 0, W - take);
    }
    free(cdf); free(names); free(nlen);
}

/* ---- DNA-alphabet keys ----------------------------------------------------
 * A share frac_prefixed of the rows starts with one of G seeded prefixes of
 * plen characters (uniform choice) followed by i.i.d. characters; the other
 * rows are i.i.d. uniform over {A,C,G,T}.  All W bytes are characters. */
void synth_dna(uint64_t n, uint64_t seed, uint32_t W, double frac_prefixed, uint32_t G, uint32_t plen, uint8_t* out) {
    static const uint8_t acgt[4] = {'A', 'C', 'G', 'T'};
    uint8_t* pre = (uint8_t*)malloc((size_t)G * plen);
    uint64_t bp = base_of(seed, 8);
    for (uint64_t k = 0; k < (uint64_t)G * plen; ++k) pre[k] = acgt[draw(bp, k) & 3];
    uint64_t bs = base_of(seed, 9), bc = base_of(seed, 10);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint8_t* row = out + (uint64_t)i * W;
        uint32_t c = 0;
        if (unif(bs, (uint64_t)i) < frac_prefixed) {
            uint64_t g = draw(bs, (uint64_t)i + 0x4000000000000000ull) % G;
            uint32_t take = plen < W ? plen : W;
            memcpy(row, pre + g * plen, take);
            c = take;
        }
        uint64_t r = 0;
        int64_t group = -1;
        for (; c < W; ++c) {                 /* 32 characters per 64-bit draw */
            if ((int64_t)(c / 32) != group) { group = c / 32; r = draw(bc, (uint64_t)i * 8 + (uint64_t)group); }
            row[c] = acgt[(r >> (2 * (c % 32))) & 3];
        }
    }
    free(pre);
}

/* ---- title-like keys: Zipf-chosen word + '_' + random letters -------------
 * nwords seeded words of 3..10 lowercase letters; each row takes word k ~
 * Zipf(s), then '_' and i.i.d. letters, to a total length L uniform on
 * [min(len+2, W-1), W-1]; zero padded to W (so every key ends in a 0 byte). */
void synth_titles(uint64_t n, uint64_t seed, uint32_t W, uint32_t nwords, double s, uint8_t* out) {
    char* words = (char*)malloc((size_t)nwords * 11);
    uint8_t* wlen = (uint8_t*)malloc(nwords);
    uint64_t bw = base_of(seed, 13);
    for (uint32_t k = 0; k < nwords; ++k) {
        wlen[k] = (uint8_t)(3 + below(bw, (uint64_t)k * 16, 8));
        for (uint32_t c = 0; c < wlen[k]; ++c) words[k * 11 + c] = (char)('a' + below(bw, (uint64_t)k * 16 + 1 + c, 26));
    }
    double* cdf = zipf_cdf(nwords, s);
    uint64_t bz = base_of(seed, 14), bl = base_of(seed, 15), bc = base_of(seed, 16);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint8_t* row = out + (uint64_t)i * W;
        memset(row, 0, W);
        uint64_t k = zipf_pick(cdf, nwords, unif(bz, (uint64_t)i));
        uint32_t lmin = wlen[k] + 2, lmax = W - 1;
        if (lmin > lmax) lmin = lmax;
        uint32_t L = lmin + (uint32_t)below(bl, (uint64_t)i, lmax - lmin + 1);
        uint32_t c = 0;
        for (; c < wlen[k] && c < L; ++c) row[c] = (uint8_t)words[k * 11 + c];
        if (c < L) row[c++] = '_';
        for (uint32_t j = 0; c < L; ++c, ++j) row[c] = (uint8_t)('a' + below(bc, (uint64_t)i * 64 + j, 26));
    }
    free(cdf); free(words); free(wlen);
}

/* ---- plain integer columns ------------------------------------------------ */
void synth_uniform_u32(uint64_t n, uint64_t seed, uint32_t* out) {
    uint64_t b = base_of(seed, 17);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = (uint32_t)(draw(b, (uint64_t)i) >> 32);
}

/* 2^32 + 256*i + U[0, 4096): ascending with noise spanning ~16 neighbours */
void synth_sequential_noise_u64(uint64_t n, uint64_t seed, uint64_t* out) {
    uint64_t b = base_of(seed, 18);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) out[i] = (1ull << 32) + 256ull * (uint64_t)i + (draw(b, (uint64_t)i) & 4095);
}

/* Zipf(s) over [1, 2^40] scattered by a seeded bijection of 40 bits, under a
 * constant 12-bit tag: key = tag << 52 | sigma(r - 1). */
void synth_zipf_tagged_u64(uint64_t n, uint64_t seed, double s, uint64_t* out) {
    synth_zipf_rejinv(n, seed, 1099511627776.0, s, out);
    const uint64_t M40 = (1ull << 40) - 1;
    uint64_t tag = (synth_draw(seed, 19, 0) & 0xFFF) | 0x800;
    uint64_t m1 = (synth_draw(seed, 19, 1) & M40) | 1, m2 = (synth_draw(seed, 19, 2) & M40) | 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
        uint64_t x = (out[i] - 1) & M40;
        x = (x * m1) & M40; x ^= x >> 21;
        x = (x * m2) & M40; x ^= x >> 19;
        out[i] = (tag << 52) | x;
    }
}


/* ---- Zipf(s, n, m) letter keys (the paper's synthetic datasets) -------------
 * n_keys keys of key_bytes bytes: in every 8-byte word of a key the first m
 * bytes hold a fixed character (one seeded printable character per position,
 * the same in all keys) and the other bytes hold lowercase letters drawn
 * independently from Zipf(s) over the 26 letters, rank 1 = 'a'. */
void synth_zipf_letters(uint64_t n_keys, uint64_t seed, uint32_t key_bytes, uint32_t m, double s, uint8_t* out) {
    double* cdf = zipf_cdf(26, s);
    const uint64_t bf = base_of(seed, 21), bz = base_of(seed, 22);
    uint8_t fixed[512];
    for (uint32_t p = 0; p < key_bytes && p < 512; ++p) fixed[p] = (uint8_t)(33 + below(bf, p, 94));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)n_keys; ++i)
        for (uint32_t p = 0; p < key_bytes; ++p)
            out[(uint64_t)i * key_bytes + p] =
                (p % 8) < m ? fixed[p]
                            : (uint8_t)('a' + zipf_pick(cdf, 26, unif(bz, (uint64_t)i * key_bytes + p)));
    free(cdf);
}

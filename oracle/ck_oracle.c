/*
 * ck_oracle.c -- plain, slow, single-threaded CPU oracle for the compressed key
 * sort hot path of Kwon et al., "Compressed Key Sort and Fast Index
 * Reconstruction" (arXiv 2009.11543).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path under
 * paper_2009_11543_gb300/, and it never calls into it.
 *
 * Every function is the paper's definition written out directly: bit loops,
 * byte compares and a library sort (qsort_r) used as a black-box step.  There
 * is no blocking, fusion or reordering beyond what the definitions state.
 *
 * Conventions (Sec. 3.1, "Definitions"):
 *   - keys are binary strings; bit position 0 is the most significant bit of
 *     byte 0, so position p is bit (7 - p % 8) of byte p / 8;
 *   - a bitmap over key positions (the D-bitmap and the variant bitmap of
 *     Sec. 4.2) is an array of uint64 words, most significant first:
 *     position p is bit (63 - p % 64) of word p / 64;
 *   - a compressed key Compress(key) (Sec. 3.2) of nbits bits is an unsigned
 *     integer whose most significant bit is the key's bit at the first (lowest)
 *     set position; it is stored right-aligned in K uint32 words, least
 *     significant word first, row-major (row r occupies out[r*K .. r*K+K-1]).
 *   - sorted order is lexicographic order of the key bytes (Sec. 3.1 and the
 *     binary comparison of Sec. 4.1); rows with equal keys keep their row-id
 *     order (the paper assumes distinct keys; ties by row id are this
 *     library's reading).
 */
#define _GNU_SOURCE
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CKO_NO_DBIT 0xFFFFu

/* ---- bit access helpers (Sec. 3.1 numbering) ---------------------------- */

static int key_bit(const uint8_t* key, uint32_t p) {
    return (key[p >> 3] >> (7 - (p & 7))) & 1;
}

static int map_test(const uint64_t* map, uint32_t p) {
    return (int)((map[p >> 6] >> (63 - (p & 63))) & 1u);
}

static void map_set(uint64_t* map, uint32_t p) {
    map[p >> 6] |= (uint64_t)1 << (63 - (p & 63));
}

/* ---- Sec. 4.1: numeric columns as binary-comparable index keys ----------
 * The index key format Sec. 4.1 takes from [LKN]: a signed integer's key is
 * its two's-complement value with the sign bit flipped; a float's key is its
 * IEEE bit pattern with every bit flipped if the sign bit is set, otherwise
 * with the sign bit flipped; in both cases written big-endian, so that
 * comparing the bytes compares the numbers.  kind: 1 uint32, 2 uint64,
 * 3 int32, 4 int64, 5 binary32, 6 binary64 (native values). */
void cko_encode_numeric(const void* in, uint64_t n, uint32_t kind, uint8_t* out) {
    const uint32_t w = (kind == 1 || kind == 3 || kind == 5) ? 4 : 8;
    const uint64_t sign = (uint64_t)1 << (8 * w - 1);
    for (uint64_t r = 0; r < n; ++r) {
        uint64_t v = 0;
        memcpy(&v, (const uint8_t*)in + r * w, w);  /* the value's bit pattern (little-endian host) */
        if (kind == 3 || kind == 4) {
            v ^= sign;
        } else if (kind == 5 || kind == 6) {
            if (v & sign) v = ~v;
            else v ^= sign;
            if (w == 4) v &= 0xFFFFFFFFull;
        }
        for (uint32_t b = 0; b < w; ++b) out[r * w + b] = (uint8_t)(v >> (8 * (w - 1 - b)));
    }
}

/* ---- Sec. 4.1: unsigned integers as binary-comparable index keys --------
 * An unsigned integer compares like its big-endian byte string ([LKN] mapping
 * referred to by Sec. 4.1).  kind 1 = uint32, kind 2 = uint64 (native values). */
void cko_uint_to_bytes(const void* in, uint64_t n, uint32_t kind, uint8_t* out) {
    uint32_t w = (kind == 1) ? 4 : 8;
    for (uint64_t r = 0; r < n; ++r) {
        uint64_t v = (kind == 1) ? ((const uint32_t*)in)[r] : ((const uint64_t*)in)[r];
        for (uint32_t b = 0; b < w; ++b)
            out[r * w + b] = (uint8_t)(v >> (8 * (w - 1 - b)));
    }
}

/* ---- Sec. 3.1: D-bit(a, b), the most significant differing position -------
 * Returns -1 when the keys are equal (the D-bit of equal keys is undefined). */
int64_t cko_dbit(const uint8_t* a, const uint8_t* b, uint32_t W) {
    for (uint32_t byte = 0; byte < W; ++byte) {
        if (a[byte] == b[byte]) continue;
        for (uint32_t p = 8 * byte; p < 8 * byte + 8; ++p)
            if (key_bit(a, p) != key_bit(b, p)) return (int64_t)p;
    }
    return -1;
}

/* ---- Sec. 3.1: sorted (lexicographic) order of the rows ------------------ */
typedef struct { const uint8_t* keys; uint32_t W; uint32_t stride; } row_ctx;

static int cmp_rows(const void* x, const void* y, void* arg) {
    const row_ctx* c = (const row_ctx*)arg;
    uint32_t i = *(const uint32_t*)x, j = *(const uint32_t*)y;
    int r = memcmp(c->keys + (uint64_t)i * c->stride, c->keys + (uint64_t)j * c->stride, c->W);
    if (r) return r;
    return (i > j) - (i < j);               /* equal keys: row-id order */
}

void cko_sort_rows(const uint8_t* keys, uint64_t n, uint32_t W, uint32_t stride, uint32_t* perm) {
    row_ctx c = {keys, W, stride};
    for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    qsort_r(perm, n, sizeof(uint32_t), cmp_rows, &c);
}

/* ---- Theorem 1: D = {D_1, ..., D_n}, D_i = D-bit(key_{i-1}, key_i) --------
 * perm lists the rows in sorted order.  Adjacent equal keys add nothing.
 * mask has ceil(8W/64) words and is overwritten. */
void cko_dmask(const uint8_t* keys, uint64_t n, uint32_t W, uint32_t stride,
               const uint32_t* perm, uint64_t* mask) {
    memset(mask, 0, sizeof(uint64_t) * ((8ull * W + 63) / 64));
    for (uint64_t i = 1; i < n; ++i) {
        int64_t p = cko_dbit(keys + (uint64_t)perm[i - 1] * stride, keys + (uint64_t)perm[i] * stride, W);
        if (p >= 0) map_set(mask, (uint32_t)p);
    }
}

/* ---- Sec. 4.2 variant bitmap, computed as in Sec. 4.3 ("DS-metadata
 * recompute", step 3): OR over all keys K of (K xor reference key). */
void cko_variant_mask(const uint8_t* keys, uint64_t n, uint32_t W, uint32_t stride,
                      const uint8_t* ref, uint64_t* mask) {
    memset(mask, 0, sizeof(uint64_t) * ((8ull * W + 63) / 64));
    for (uint64_t r = 0; r < n; ++r)
        for (uint32_t p = 0; p < 8 * W; ++p)
            if (key_bit(keys + r * stride, p) != key_bit(ref, p)) map_set(mask, p);
}

/* ---- Sec. 3.2: Compress(key) = the concatenation of the key's bits at the
 * (extended) distinction positions, in position order.  Bit j of the
 * concatenation (j = 0 first) is the key bit at the j-th set position and
 * becomes bit (nbits - 1 - j) of the right-aligned integer.
 * Returns nbits (the number of set positions), or -1 if it exceeds 32*K. */
int64_t cko_compress(const uint8_t* keys, uint64_t n, uint32_t W, uint32_t stride,
                     const uint64_t* mask, uint32_t K, uint32_t* out) {
    uint32_t nbits = 0;
    for (uint32_t p = 0; p < 8 * W; ++p) nbits += (uint32_t)map_test(mask, p);
    if (nbits > 32u * K) return -1;
    for (uint64_t r = 0; r < n; ++r) {
        const uint8_t* key = keys + r * stride;
        uint32_t* v = out + r * K;
        memset(v, 0, sizeof(uint32_t) * K);
        uint32_t j = 0;
        for (uint32_t p = 0; p < 8 * W; ++p) {
            if (!map_test(mask, p)) continue;
            uint32_t vb = nbits - 1 - j;    /* value bit of concatenation bit j */
            if (key_bit(key, p)) v[vb / 32] |= 1u << (vb % 32);
            ++j;
        }
    }
    return nbits;
}

/* ---- Sec. 3.2 "compressed key sort": sort rows by Compress value ---------- */
typedef struct { const uint32_t* ck; uint32_t K; } ck_ctx;

static int cmp_ck(const void* x, const void* y, void* arg) {
    const ck_ctx* c = (const ck_ctx*)arg;
    uint32_t i = *(const uint32_t*)x, j = *(const uint32_t*)y;
    for (uint32_t w = c->K; w-- > 0;) {     /* most significant word first */
        uint32_t a = c->ck[(uint64_t)i * c->K + w], b = c->ck[(uint64_t)j * c->K + w];
        if (a != b) return a < b ? -1 : 1;
    }
    return (i > j) - (i < j);
}

void cko_sort_compressed(const uint32_t* ck, uint64_t n, uint32_t K, uint32_t* perm) {
    ck_ctx c = {ck, K};
    for (uint64_t i = 0; i < n; ++i) perm[i] = (uint32_t)i;
    qsort_r(perm, n, sizeof(uint32_t), cmp_ck, &c);
}

/* D-bit between two compressed values, numbered as a concatenation position
 * (0 = the most significant of the nbits bits); -1 if equal. */
static int64_t ck_dbit(const uint32_t* a, const uint32_t* b, uint32_t nbits) {
    for (uint32_t j = 0; j < nbits; ++j) {
        uint32_t vb = nbits - 1 - j;
        uint32_t x = (a[vb / 32] >> (vb % 32)) & 1u, y = (b[vb / 32] >> (vb % 32)) & 1u;
        if (x != y) return (int64_t)j;
    }
    return -1;
}

/* ---- Sec. 4.3 rebuild step 1 with the D-offset array of Sec. 5.3 ----------
 * New D-bitmap = { D-offset[D-bit(Compress(key_{i-1}), Compress(key_i))] } over
 * the compressed keys in sorted order; D-offset[q] is the position of the
 * (q+1)-st 1 of the current D-bitmap.  ck is row-major n x K (as from
 * cko_compress), perm the sorted order.  new_mask gets ceil(key_bits/64) words. */
void cko_refine(const uint32_t* ck, const uint32_t* perm, uint64_t n, uint32_t K,
                const uint64_t* old_mask, uint32_t key_bits, uint64_t* new_mask) {
    uint32_t* doffset = (uint32_t*)malloc(sizeof(uint32_t) * (key_bits + 1));
    uint32_t nbits = 0;
    for (uint32_t p = 0; p < key_bits; ++p)
        if (map_test(old_mask, p)) doffset[nbits++] = p;
    memset(new_mask, 0, sizeof(uint64_t) * ((key_bits + 63) / 64));
    for (uint64_t i = 1; i < n; ++i) {
        int64_t q = ck_dbit(ck + (uint64_t)perm[i - 1] * K, ck + (uint64_t)perm[i] * K, nbits);
        if (q >= 0) map_set(new_mask, doffset[q]);
    }
    free(doffset);
}

/* ---- Sec. 5.3 bottom-up bulk load --------------------------------------
 * Canonical layout: every node at every level holds f consecutive entries
 * (the last node of a level may hold fewer); level 0 holds one entry per key
 * in sorted order; level l+1 holds one entry per node of level l; levels are
 * added until a level fits in one node (the root).
 *
 * cko_btree_shape: returns the level count and fills level_entries[l]
 * (entries at level l) for l < levels; n == 0 gives 0 levels. */
uint32_t cko_btree_shape(uint64_t n, uint32_t f, uint64_t* level_entries, uint32_t max_levels) {
    if (n == 0 || f < 2) {
        if (n == 1 && max_levels > 0) { level_entries[0] = 1; return 1; }
        return 0;
    }
    uint32_t l = 0;
    uint64_t m = n;
    while (l < max_levels) {
        level_entries[l++] = m;
        if (m <= f) break;                  /* this level is the root node */
        uint64_t nodes = 0, start = 0;
        while (start < m) { ++nodes; start += f; }   /* count the nodes of the level */
        m = nodes;
    }
    return l;
}

/* Leaf entries (Sec. 4.2 / 5.3): the D-bit of each key against the previous key
 * in sorted order, computed directly on the full keys (no D-offset); 0xFFFF for
 * the first key and for a key equal to its predecessor. */
void cko_btree_leaf_dbits(const uint8_t* keys, uint64_t n, uint32_t W, uint32_t stride,
                          const uint32_t* perm, uint16_t* dbit) {
    for (uint64_t i = 0; i < n; ++i) {
        int64_t p = (i == 0) ? -1 : cko_dbit(keys + (uint64_t)perm[i - 1] * stride, keys + (uint64_t)perm[i] * stride, W);
        dbit[i] = (p < 0) ? (uint16_t)CKO_NO_DBIT : (uint16_t)p;
    }
}

/* Non-leaf levels (Sec. 4.2 / 5.3), built bottom-up.  For every inner level l
 * (1 <= l < levels) and entry e of that level, in level order:
 *   child[e]  = e, the node of level l-1 the entry points to;
 *   high[e]   = the sorted index of the highest key in the descendant leaves
 *               of that child;
 *   dbit[e]   = D-bit of that highest key against the previous entry's highest
 *               key at the same level (0xFFFF for e = 0 or equal keys).
 * Arrays are concatenated level after level (level 1 first). */
void cko_btree_inner(const uint8_t* keys, uint64_t n, uint32_t W, uint32_t stride,
                     const uint32_t* perm, uint32_t f, uint32_t levels, const uint64_t* level_entries,
                     uint32_t* child, uint64_t* high, uint16_t* dbit) {
    (void)n;
    if (levels < 2) return;
    /* node_high: highest sorted index under each node of the current level */
    uint64_t m = level_entries[0];
    uint64_t* entry_high = (uint64_t*)malloc(sizeof(uint64_t) * m);
    for (uint64_t i = 0; i < m; ++i) entry_high[i] = i;       /* a leaf entry is one key */
    uint64_t out = 0;
    for (uint32_t l = 1; l < levels; ++l) {
        uint64_t nodes = level_entries[l];
        uint64_t* next_high = (uint64_t*)malloc(sizeof(uint64_t) * (nodes ? nodes : 1));
        for (uint64_t e = 0; e < nodes; ++e) {
            uint64_t last = (e + 1) * (uint64_t)f;            /* node e of level l-1 ends here */
            if (last > m) last = m;
            next_high[e] = entry_high[last - 1];
        }
        for (uint64_t e = 0; e < nodes; ++e, ++out) {
            child[out] = (uint32_t)e;
            high[out] = next_high[e];
            int64_t p = -1;
            if (e > 0)
                p = cko_dbit(keys + (uint64_t)perm[next_high[e - 1]] * stride,
                             keys + (uint64_t)perm[next_high[e]] * stride, W);
            dbit[out] = (p < 0) ? (uint16_t)CKO_NO_DBIT : (uint16_t)p;
        }
        free(entry_high);
        entry_high = next_high;
        m = nodes;
    }
    free(entry_high);
}

/* ---- learned CDF model (not in the paper): fp64 reference ----------------
 * y(x) = b2 + sum_j w2[j] * relu(w1[j] * x + b1[j]), j < 16, parameters packed
 * as [w1(16), b1(16), w2(16), b2] (49 values).  Loss over S samples with
 * targets t_i: L = (1/S) * sum_i (y(x_i) - t_i)^2.  Writes L and dL/dparams
 * (49 values) by the chain rule, summed over the samples in index order. */
#define CKO_HIDDEN 16
double cko_mlp_forward(const double* p, double x) {
    double y = p[3 * CKO_HIDDEN];
    for (int j = 0; j < CKO_HIDDEN; ++j) {
        double z = p[j] * x + p[CKO_HIDDEN + j];
        if (z > 0.0) y += p[2 * CKO_HIDDEN + j] * z;
    }
    return y;
}

double cko_mlp_loss_grad(const double* p, const double* x, const double* t, uint64_t S, double* grad) {
    memset(grad, 0, sizeof(double) * (3 * CKO_HIDDEN + 1));
    double loss = 0.0;
    for (uint64_t i = 0; i < S; ++i) {
        double y = cko_mlp_forward(p, x[i]);
        double r = y - t[i];
        loss += r * r;
        double dy = 2.0 * r / (double)S;                 /* dL/dy_i */
        grad[3 * CKO_HIDDEN] += dy;                      /* b2 */
        for (int j = 0; j < CKO_HIDDEN; ++j) {
            double z = p[j] * x[i] + p[CKO_HIDDEN + j];
            if (z <= 0.0) continue;                      /* relu'(z) = 0 */
            grad[2 * CKO_HIDDEN + j] += dy * z;          /* w2_j: dy/dw2_j = relu(z) */
            double dz = dy * p[2 * CKO_HIDDEN + j];      /* dL/dz_j */
            grad[j] += dz * x[i];                        /* w1_j */
            grad[CKO_HIDDEN + j] += dz;                  /* b1_j */
        }
    }
    return loss / (double)S;
}


/* ---- Sec. 4.3, "Search and Update Operations": DS-metadata under inserts --
 * Inserts the m keys of `batch` one after another, in the given order, into
 * the sorted set that starts as the n keys of `keys` (sorted order `perm`).
 * For each insert key K: search the current sorted set for the place of K,
 * between A (the largest key < K) and B (the smallest key >= K); set in the
 * D-bitmap the larger of D-bit(A, K) and D-bit(K, B) (only the defined ones:
 * a missing neighbour or an equal key has none; D-bit(A, B) is the smaller
 * one, Lemma 1, and is already set); OR (K xor reference key) into the variant
 * bitmap; then add K to the set.  dmask and vmask are updated in place.  The
 * current set is a plain sorted array of key copies, grown by memmove. */
void cko_insert_batch(const uint8_t* keys, uint64_t n, uint32_t W, const uint32_t* perm, const uint8_t* batch,
                      uint64_t m, const uint8_t* ref, uint64_t* dmask, uint64_t* vmask) {
    uint8_t* set = (uint8_t*)malloc((size_t)(n + m) * W + 1);
    for (uint64_t i = 0; i < n; ++i) memcpy(set + i * W, keys + (uint64_t)perm[i] * W, W);
    uint64_t count = n;
    for (uint64_t j = 0; j < m; ++j) {
        const uint8_t* k = batch + j * W;
        uint64_t lo = 0, hi = count;  /* first position whose key is >= K */
        while (lo < hi) {
            const uint64_t mid = (lo + hi) / 2;
            if (memcmp(set + mid * W, k, W) < 0) lo = mid + 1;
            else hi = mid;
        }
        int64_t best = -1;
        if (lo > 0) {
            const int64_t d = cko_dbit(set + (lo - 1) * W, k, W);
            if (d > best) best = d;
        }
        if (lo < count) {
            const int64_t d = cko_dbit(k, set + lo * W, W);
            if (d > best) best = d;
        }
        if (best >= 0) map_set(dmask, (uint32_t)best);
        for (uint32_t p = 0; p < 8 * W; ++p)
            if (key_bit(k, p) != key_bit(ref, p)) map_set(vmask, p);
        memmove(set + (lo + 1) * W, set + lo * W, (size_t)(count - lo) * W);
        memcpy(set + lo * W, k, W);
        ++count;
    }
    free(set);
}

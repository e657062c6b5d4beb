// ck_search.cu -- partial keys of the index tree (Sec. 4.2, after Bohannon,
// McIlroy and Rastogi's partial-key B+-tree; bit sources of Sec. 5.3) and the
// lower-bound search of Sec. 4.3 that uses them.
//
// Partial keys: one thread per tree entry, word-wide.  The pk positions after
// the entry's offset form a window; the mask positions in it have consecutive
// ranks in the extraction mask, so their bits are one run of the compressed
// key (read as a 64-bit window) deposited at those positions; the invariant
// positions take the reference key's window, any other the key row's.
//
// Search: one thread per query.  Inner nodes: binary search over the node's
// highest keys, compared as full keys; every comparison also yields the D-bit
// of the two keys, and the last highest key found below the query is the key
// just before the leaf the search lands in (the fence).  Leaf: the entries are
// scanned in order knowing d = D-bit(query, previous key), query > previous
// key.  For entry i with offset o = D-bit(key_{i-1}, key_i):
//   o < d   key_i has a 1 at o where the query (equal to key_{i-1} there) has
//           a 0: key_i is the first key >= the query.
//   o > d   key_i equals key_{i-1} at d, so the query stays above it; d holds.
//   o = d   query and key_i agree up to d; the partial key (positions o + 1 ..
//           o + pk) decides at its first differing bit, and only when it
//           equals the query's bits is the full key of entry i read.
#include "ck_internal.cuh"

#include <cstring>

namespace ck {

namespace {

constexpr int kPkThreads = 256;
constexpr int kSearchThreads = 128;

struct PkArgs {
    const uint32_t* ck;       // leaves' sorted compressed keys, word-major (NULL: read the rows)
    uint64_t ld;
    const uint32_t* high_ck;  // inner entries' compressed highest keys, entry-major
    const uint32_t* leaf_rid;
    const uint16_t* leaf_dbit;
    const uint32_t* inner_rid;
    const uint16_t* inner_dbit;
    uint64_t n, inner;
    uint64_t rows;            // rows of the key column (0: no column)
    uint32_t K, nbits, key_bits, pk;
    // big-endian 32-bit words: position 32w + i is bit 31 - i of word w
    uint32_t emask[kMaxKeyWords];
    uint32_t vmask[kMaxKeyWords];
    uint32_t ref[kMaxKeyWords];
    uint32_t erank[kMaxKeyWords];  // set positions of emask before word w
};

// Positions [start, start + pk) of a big-endian word array (two words from
// w = start / 32 on; hi and lo are words w and w + 1) as a pk-bit value, the
// first position most significant.
__device__ __forceinline__ uint32_t window_of(uint32_t hi, uint32_t lo, uint32_t start, uint32_t pk) {
    const uint64_t v = ((uint64_t)hi << 32) | lo;
    return (uint32_t)((v << (start & 31)) >> (64 - pk));
}

template <int VEC>
__global__ void __launch_bounds__(kPkThreads) partial_keys_kernel(const __grid_constant__ PkArgs a,
                                                                   const __grid_constant__ KeyDesc col,
                                                                   uint32_t* __restrict__ leaf_pk,
                                                                   uint32_t* __restrict__ inner_pk,
                                                                   unsigned long long* status) {
    __shared__ uint32_t em[kMaxKeyWords + 1], vm[kMaxKeyWords + 1], rf[kMaxKeyWords + 1], er[kMaxKeyWords + 1];
    const uint32_t words = (a.key_bits + 31) / 32;
    for (uint32_t i = threadIdx.x; i <= words; i += blockDim.x) {
        const bool in = i < words;
        em[i] = in ? a.emask[i] : 0u;
        vm[i] = in ? a.vmask[i] : 0u;
        rf[i] = in ? a.ref[i] : 0u;
        er[i] = in ? a.erank[i] : a.nbits;
    }
    __syncthreads();
    const uint32_t pk = a.pk;
    const uint32_t all = pk == 32 ? 0xFFFFFFFFu : (1u << pk) - 1u;
    const uint64_t total = a.n + a.inner;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
         g += (uint64_t)gridDim.x * blockDim.x) {
        const bool leaf = g < a.n;
        const uint64_t e = leaf ? g : g - a.n;
        const uint32_t off = leaf ? a.leaf_dbit[e] : a.inner_dbit[e];
        const uint64_t row = leaf ? a.leaf_rid[e] : a.inner_rid[e];
        const bool from_ck = leaf ? a.ck != nullptr : true;
        const uint32_t start = off == CK_NO_DBIT ? 0u : off + 1u;
        uint32_t v = 0, rest = all;
        if (start < a.key_bits) {
            const uint32_t w = start >> 5;
            const uint32_t wv = window_of(vm[w], vm[w + 1], start, pk);
            const uint32_t wr = window_of(rf[w], rf[w + 1], start, pk);
            if (from_ck) {                                    // (A) a run of the compressed key
                const uint32_t we = window_of(em[w], em[w + 1], start, pk);
                const uint32_t c = __popc(we);
                if (c) {
                    const uint32_t q0 = er[w] + ((start & 31) ? __popc(em[w] >> (32 - (start & 31))) : 0u);
                    const uint32_t lo = a.nbits - q0 - c;     // integer bit of the run's last rank
                    const uint32_t k0 = lo >> 5;
                    uint32_t x0, x1;
                    if (leaf) {
                        x0 = a.ck[(uint64_t)k0 * a.ld + e];
                        x1 = k0 + 1 < a.K ? a.ck[(uint64_t)(k0 + 1) * a.ld + e] : 0u;
                    } else {
                        x0 = a.high_ck[e * a.K + k0];
                        x1 = k0 + 1 < a.K ? a.high_ck[e * a.K + k0 + 1] : 0u;
                    }
                    const uint32_t run = (uint32_t)(((((uint64_t)x1 << 32) | x0) >> (lo & 31)) & ((1ull << c) - 1));
                    // deposit the run, first rank first, at the window's mask positions
                    uint32_t m = we;
                    for (int r = (int)c - 1; r >= 0; --r) {
                        const uint32_t top = 31u - __clz(m);
                        v |= ((run >> r) & 1u) << top;
                        m &= ~(1u << top);
                    }
                }
                rest &= ~we;
            }
            v |= wr & ~wv & rest;                             // (B) invariant: the reference key
            const uint32_t need = wv & rest;                  // (C) option b: the record's key
            if (need) {
                if (row < a.rows) {
                    const uint32_t wr0 = key_word<VEC>(col, row, w), wr1 = key_word<VEC>(col, row, w + 1);
                    v |= window_of(wr0, wr1, start, pk) & need;
                } else {                                      // no such row (or no column): read as 0
                    report(status, CK_EINVAL, row);
                }
            }
            // positions past the key's end read 0: the windows hold zeros there
        }
        if (leaf) leaf_pk[e] = v;
        else inner_pk[e] = v;
    }
}

struct SearchArgs {
    const uint32_t* leaf_rid;
    const uint16_t* leaf_dbit;
    const uint32_t* leaf_pk;
    const uint32_t* inner_child;
    const uint32_t* inner_high;
    const uint32_t* inner_rid;
    const uint16_t* inner_dbit;
    const uint32_t* inner_pk;  // NULL: inner nodes compare full keys
    uint64_t n, q;
    uint32_t f, levels, pk;
    uint64_t level_entries[CK_MAX_LEVELS];
    uint64_t offset[CK_MAX_LEVELS];
};

constexpr uint64_t kScanError = ~0ull;

// Scans entries i .. t - 1 of one level in key order (offsets dbit, partial
// keys pks, row ids rids), knowing that Q is above the key before entry i and
// that d is their D-bit.  Returns the first entry whose key is >= Q (t if
// none; kScanError after a bad row id) and sets eq when a full comparison
// found that key equal to Q.  On return d is still the D-bit of Q against the
// key before the returned entry.
template <int VEC, int QW>
__device__ __forceinline__ uint64_t scan_level(const uint16_t* dbit, const uint32_t* pks, const uint32_t* rids,
                                               uint64_t i, uint64_t t, int32_t& d, const KeyDesc& col,
                                               const QueryView<VEC, QW> Q, uint32_t pk, uint64_t n, bool& eq,
                                               uint32_t& derefs, unsigned long long* status) {
    eq = false;
    for (; i < t; ++i) {
        const uint32_t o = dbit[i];
        if (o == CK_NO_DBIT) continue;  // equal to the previous key: still below Q
        if ((int32_t)o < d) return i;
        if ((int32_t)o > d) continue;
        // o == d: compare Q's bits o + 1 .. o + pk with the partial key
        const uint32_t p0 = o + 1;
        const uint32_t qb = Q.window(p0, pk);
        const uint32_t x = qb ^ pks[i];
        if (x) {
            const uint32_t lead = __clz(x) - (32 - pk);  // first differing bit among the pk
            if ((qb >> (pk - 1 - lead)) & 1u) {
                d = (int32_t)(p0 + lead);                // Q above key_i
                continue;
            }
            return i;
        }
        const uint32_t r = rids[i];
        if (r >= n) {
            report(status, CK_EINVAL, i);
            return kScanError;
        }
        ++derefs;
        int32_t dd;
        const int c = Q.cmp(col, r, &dd);
        if (c >= 0) {
            eq = c == 0;
            return i;
        }
        d = dd;
    }
    return t;
}

template <int VEC, int QW, bool INNER_PK>
__global__ void __launch_bounds__(kSearchThreads, 10) search_kernel(const __grid_constant__ SearchArgs a,
                                                                const __grid_constant__ KeyDesc col,
                                                                const __grid_constant__ KeyDesc qk,
                                                                uint32_t* __restrict__ pos_out,
                                                                uint32_t* __restrict__ rid_out,
                                                                uint32_t* __restrict__ derefs_out,
                                                                unsigned long long* status) {
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.q; j += (uint64_t)gridDim.x * blockDim.x) {
        const QueryView<VEC, QW> Q(qk, j);
        uint64_t pos = a.n;
        bool found = false;
        uint32_t derefs = 0;
        if (a.n == 0) goto done;
        if (INNER_PK) {
            // ---- every level scanned with offsets and partial keys; the state d
            //      (Q against the key before the current node) carries down, since
            //      the key before child i's first entry is entry i - 1's highest key
            uint64_t node = 0;
            bool has_prev = false;  // false on the leftmost path: no key before the node
            int32_t d = -1;
            for (int32_t l = (int32_t)a.levels - 1; l >= 0; --l) {
                const bool inner = l >= 1;
                const uint64_t base = inner ? a.offset[l] : 0;
                const uint64_t m = inner ? a.level_entries[l] : a.n;
                const uint64_t s = node * a.f, t = min(s + a.f, m);
                const uint16_t* dbit = inner ? a.inner_dbit + base : a.leaf_dbit;
                const uint32_t* pks = inner ? a.inner_pk + base : a.leaf_pk;
                const uint32_t* rids = inner ? a.inner_rid + base : a.leaf_rid;
                uint64_t i = s;
                bool eq = false, first_ge = false;
                if (!has_prev) {  // the node's first key has no offset: compare it in full
                    const uint32_t r = rids[s];
                    if (r >= a.n) {
                        report(status, CK_EINVAL, s);
                        goto done;
                    }
                    ++derefs;
                    int32_t dd;
                    const int c = Q.cmp(col, r, &dd);
                    if (c >= 0) {
                        eq = c == 0;
                        first_ge = true;
                    } else {
                        d = dd;
                        has_prev = true;
                        i = s + 1;
                    }
                }
                if (!first_ge) {
                    i = scan_level<VEC, QW>(dbit, pks, rids, i, t, d, col, Q, a.pk, a.n, eq, derefs, status);
                    if (i == kScanError) goto done;
                }
                if (i == t) {  // Q above every key under this node: only at the root or the last leaf
                    pos = inner ? a.n : t;
                    goto done;
                }
                if (!inner) {
                    pos = i;
                    found = eq;
                    goto done;
                }
                node = a.inner_child[base + i];
            }
            goto done;
        }
        {
            // ---- inner levels compare full keys (Sec. 4.3): the first entry of
            //      the node whose highest key is >= Q, by binary search
            uint64_t node = 0;
            int64_t fence = -1;  // sorted index of the last highest key found below Q
            int32_t fence_d = -1;
            for (int32_t l = (int32_t)a.levels - 1; l >= 1; --l) {
                const uint64_t m = a.level_entries[l];
                uint64_t lo = node * a.f, hi = min(lo + a.f, m);
                const uint64_t end = hi;
                while (lo < hi) {
                    const uint64_t mid = (lo + hi) >> 1;
                    const uint64_t g = a.offset[l] + mid;
                    const uint32_t r = a.inner_rid[g];
                    if (r >= a.n) {
                        report(status, CK_EINVAL, g);
                        goto done;
                    }
                    int32_t d;
                    if (Q.cmp(col, r, &d) < 0) {
                        lo = mid + 1;
                        fence = a.inner_high[g];
                        fence_d = d;
                    } else {
                        hi = mid;
                    }
                }
                if (lo == end) goto done;  // Q is above every key
                node = a.inner_child[a.offset[l] + lo];
            }
            // ---- leaf: scan with offsets and partial keys
            const uint64_t s = node * a.f, t = min(s + a.f, a.n);
            uint64_t i = s;
            int32_t d = fence_d;
            if (s == 0 || fence != (int64_t)(s - 1)) {
                // no key before the leaf was compared: compare with it (or with the first key)
                const uint64_t prev = s == 0 ? 0 : s - 1;
                const uint32_t r = a.leaf_rid[prev];
                if (r >= a.n) {
                    report(status, CK_EINVAL, prev);
                    goto done;
                }
                ++derefs;
                const int c = Q.cmp(col, r, &d);
                if (s == 0) {
                    if (c >= 0) {
                        pos = 0;
                        found = c == 0;
                        goto done;
                    }
                    i = 1;
                }
            }
            bool eq = false;
            i = scan_level<VEC, QW>(a.leaf_dbit, a.leaf_pk, a.leaf_rid, i, t, d, col, Q, a.pk, a.n, eq, derefs,
                                    status);
            if (i == kScanError) goto done;
            pos = i;
            found = eq;
        }
    done:
        pos_out[j] = (uint32_t)pos;
        if (rid_out) rid_out[j] = found ? a.leaf_rid[pos] : CK_NO_ROW;
        if (derefs_out) derefs_out[j] = derefs;
    }
}

bool load_mask(const uint64_t* src, uint32_t key_bits, uint64_t* dst) {
    if (!src) return false;
    const uint32_t words = (key_bits + 63) / 64;
    memset(dst, 0, sizeof(uint64_t) * kMaxMaskWords);
    memcpy(dst, src, sizeof(uint64_t) * words);
    if (key_bits & 63) dst[words - 1] &= ~0ull << (64 - (key_bits & 63));
    return true;
}

bool host_bit(const uint64_t* m, uint32_t p) { return (m[p >> 6] >> (63 - (p & 63))) & 1ull; }

}  // namespace
}  // namespace ck

using namespace ck;

extern "C" {

ck_status ck_partial_key_mask(const uint64_t* dmask, const uint64_t* vmask, uint32_t key_bits, uint32_t pk,
                              uint64_t* out) {
    if (!dmask || !vmask || !out || key_bits == 0 || key_bits > kMaxKeyBits || pk == 0 ||
        pk > CK_MAX_PARTIAL_KEY_BITS)
        return CK_EINVAL;
    const uint32_t words = (key_bits + 63) / 64;
    uint64_t res[kMaxMaskWords] = {0};
    auto add_after = [&](uint32_t start) {
        for (uint32_t p = start; p < start + pk && p < key_bits; ++p)
            if (host_bit(vmask, p)) res[p >> 6] |= 1ull << (63 - (p & 63));
    };
    add_after(0);
    for (uint32_t p = 0; p < key_bits; ++p)
        if (host_bit(dmask, p)) {
            res[p >> 6] |= 1ull << (63 - (p & 63));
            add_after(p + 1);
        }
    memcpy(out, res, sizeof(uint64_t) * words);
    return CK_OK;
}

ck_status ck_partial_keys(const ck_btree* tree, const uint32_t* sorted_ck, uint32_t ck_words, const uint64_t* emask,
                          const uint64_t* vmask, const uint8_t* ref_key, const ck_column* col, uint32_t key_bytes,
                          uint32_t pk, uint32_t* leaf_pk, uint32_t* inner_pk, ck_stream stream) {
    if (!tree || !emask || !vmask || !ref_key || pk == 0 || pk > CK_MAX_PARTIAL_KEY_BITS || key_bytes == 0 ||
        key_bytes > CK_MAX_KEY_BYTES || ck_words == 0 || ck_words > kMaxKeyWords)
        return CK_EINVAL;
    const ck_btree_shape& sh = tree->shape;
    const uint64_t n = sh.n;
    if (n == 0) return CK_OK;
    if (!leaf_pk || !tree->leaf_rid || !tree->leaf_dbit) return CK_EINVAL;
    if (sh.inner_entries > 0 && (!inner_pk || !tree->inner_high_rid || !tree->inner_dbit || !tree->inner_high_ck))
        return CK_EINVAL;
    KeyDesc k;
    memset(&k, 0, sizeof(k));
    int vec = 1;
    if (col) {
        if (!make_key_desc(col, &k, &vec) || col->key_bytes != key_bytes) return CK_EINVAL;
    }
    static thread_local PkArgs a;
    memset(&a, 0, sizeof(a));
    a.key_bits = 8 * key_bytes;
    uint64_t e64[kMaxMaskWords], v64[kMaxMaskWords];
    load_mask(emask, a.key_bits, e64);
    load_mask(vmask, a.key_bits, v64);
    uint32_t nbits = 0;
    for (uint32_t w = 0; w < kMaxKeyWords; ++w) {
        const uint32_t sh = (w & 1) ? 0 : 32;
        a.emask[w] = (uint32_t)(e64[w >> 1] >> sh);
        a.vmask[w] = (uint32_t)(v64[w >> 1] >> sh);
        a.erank[w] = nbits;
        nbits += (uint32_t)__builtin_popcount(a.emask[w]);
    }
    if (nbits > 32 * ck_words) return CK_EINVAL;
    if (!sorted_ck && !col) return CK_EINVAL;  // the leaves' bits need a source
    for (uint32_t b = 0; b < key_bytes; ++b) a.ref[b >> 2] |= (uint32_t)ref_key[b] << (8 * (3 - (b & 3)));
    a.ck = sorted_ck;
    a.ld = CK_LD(n);
    a.high_ck = tree->inner_high_ck;
    a.leaf_rid = tree->leaf_rid;
    a.leaf_dbit = tree->leaf_dbit;
    a.inner_rid = tree->inner_high_rid;
    a.inner_dbit = tree->inner_dbit;
    a.n = n;
    a.inner = sh.inner_entries;
    a.rows = col ? col->n : 0;
    a.K = ck_words;
    a.nbits = nbits;
    a.pk = pk;
    unsigned long long* status = status_ptr();
    if (!status) return CK_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t total = n + sh.inner_entries;
    const uint64_t want = (total + kPkThreads - 1) / kPkThreads, cap = (uint64_t)num_sms() * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    switch (col ? vec : 1) {
        case 16: partial_keys_kernel<16><<<grid, kPkThreads, 0, s>>>(a, k, leaf_pk, inner_pk, status); break;
        case 8: partial_keys_kernel<8><<<grid, kPkThreads, 0, s>>>(a, k, leaf_pk, inner_pk, status); break;
        case 4: partial_keys_kernel<4><<<grid, kPkThreads, 0, s>>>(a, k, leaf_pk, inner_pk, status); break;
        default: partial_keys_kernel<1><<<grid, kPkThreads, 0, s>>>(a, k, leaf_pk, inner_pk, status); break;
    }
    count_launch();
    return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

ck_status ck_search(const ck_btree* tree, const ck_column* col, const uint32_t* leaf_pk, const uint32_t* inner_pk,
                    uint32_t pk, const ck_column* queries, uint32_t* pos_out, uint32_t* rid_out,
                    uint32_t* derefs_out, ck_stream stream) {
    if (!tree || pk == 0 || pk > CK_MAX_PARTIAL_KEY_BITS) return CK_EINVAL;
    KeyDesc ck_, qk;
    int vc = 1, vq = 1;
    if (!make_key_desc(col, &ck_, &vc) || !make_key_desc(queries, &qk, &vq)) return CK_EINVAL;
    if (col->key_bytes != queries->key_bytes || col->kind != queries->kind) return CK_EINVAL;
    const ck_btree_shape& sh = tree->shape;
    if (sh.n != col->n || sh.levels > CK_MAX_LEVELS) return CK_EINVAL;
    const uint64_t q = queries->n;
    if (q == 0) return CK_OK;
    if (!pos_out) return CK_EINVAL;
    if (sh.n > 0 && (!leaf_pk || !tree->leaf_rid || !tree->leaf_dbit || sh.levels == 0 || sh.entries_per_node == 0))
        return CK_EINVAL;
    if (sh.levels > 1 && (!tree->inner_child || !tree->inner_high || !tree->inner_high_rid)) return CK_EINVAL;
    if (sh.levels > 1 && inner_pk && !tree->inner_dbit) return CK_EINVAL;
    SearchArgs a;
    memset(&a, 0, sizeof(a));
    a.leaf_rid = tree->leaf_rid;
    a.leaf_dbit = tree->leaf_dbit;
    a.leaf_pk = leaf_pk;
    a.inner_child = tree->inner_child;
    a.inner_high = tree->inner_high;
    a.inner_rid = tree->inner_high_rid;
    a.inner_dbit = tree->inner_dbit;
    a.inner_pk = sh.levels > 1 ? inner_pk : nullptr;
    a.n = sh.n;
    a.q = q;
    a.f = sh.entries_per_node;
    a.levels = sh.levels;
    a.pk = pk;
    for (uint32_t l = 0; l < CK_MAX_LEVELS; ++l) {
        a.level_entries[l] = sh.level_entries[l];
        a.offset[l] = sh.inner_offset[l];
    }
    unsigned long long* status = status_ptr();
    if (!status) return CK_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t want = (q + kSearchThreads - 1) / kSearchThreads, cap = (uint64_t)num_sms() * 16;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    const int vec = vc < vq ? vc : vq;
    // the query's key words in registers up to 8 words (32-byte keys)
    const uint32_t nw = qk.nwords;
    const int qw = nw <= 1 ? 1 : nw <= 2 ? 2 : nw <= 4 ? 4 : nw <= 8 ? 8 : 0;
#define CK_SEARCH_LAUNCH(V, QW)                                                                               \
    if (a.inner_pk)                                                                                           \
        search_kernel<V, QW, true><<<grid, kSearchThreads, 0, s>>>(a, ck_, qk, pos_out, rid_out, derefs_out,   \
                                                                    status);                                  \
    else                                                                                                      \
        search_kernel<V, QW, false><<<grid, kSearchThreads, 0, s>>>(a, ck_, qk, pos_out, rid_out, derefs_out,  \
                                                                     status)
#define CK_SEARCH_QW(V)                          \
    switch (qw) {                                \
        case 1: CK_SEARCH_LAUNCH(V, 1); break;   \
        case 2: CK_SEARCH_LAUNCH(V, 2); break;   \
        case 4: CK_SEARCH_LAUNCH(V, 4); break;   \
        case 8: CK_SEARCH_LAUNCH(V, 8); break;   \
        default: CK_SEARCH_LAUNCH(V, 0); break;  \
    }
    switch (vec) {
        case 16: CK_SEARCH_QW(16) break;
        case 8: CK_SEARCH_QW(8) break;
        case 4: CK_SEARCH_QW(4) break;
        default: CK_SEARCH_QW(1) break;
    }
#undef CK_SEARCH_QW
#undef CK_SEARCH_LAUNCH
    count_launch();
    return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

}  // extern "C"

// ck_api.cu -- the extern "C" entry points of libck (declared in include/ck.h):
// argument validation, host-side plans, and the per-device status word.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>

#include "ck_internal.cuh"

namespace ck {

// One status word per device (a file-scope device variable, so the library
// allocates nothing); kernels receive its address as an argument.
__device__ unsigned long long g_status_word;

static constexpr int kMaxDevices = 64;
static std::mutex g_mu;
static unsigned long long* g_status_addr[kMaxDevices];
static int g_sms[kMaxDevices];
static std::atomic<uint64_t> g_launches{0};

static int current_device() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
    return d;
}

int num_sms() {
    const int d = current_device();
    if (d < 0) return 1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_sms[d] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0) v = 1;
        g_sms[d] = v;
    }
    return g_sms[d];
}

unsigned long long* status_ptr() {
    const int d = current_device();
    if (d < 0) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status_addr[d]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
        g_status_addr[d] = static_cast<unsigned long long*>(p);
    }
    return g_status_addr[d];
}

void count_launch(uint32_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Chooses the widest load (16/8/4 bytes) that every row allows: the pointer
// and the stride must be multiples of it, and rounding the key up to it must
// stay inside the row's stride.
bool make_key_desc(const ck_column* col, KeyDesc* d, int* vec) {
    if (!col || (col->n > 0 && !col->keys)) return false;
    if (col->n > CK_MAX_ROWS) return false;
    const uint32_t W = col->key_bytes;
    if (W == 0 || W > CK_MAX_KEY_BYTES || col->row_stride < W) return false;
    if (col->kind > CK_KIND_F64) return false;
    const bool four = col->kind == CK_KIND_U32 || col->kind == CK_KIND_I32 || col->kind == CK_KIND_F32;
    if (four && W != 4) return false;
    if (col->kind != CK_KIND_BYTES && !four && W != 8) return false;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(col->keys);
    const uint64_t stride = col->row_stride;
    if (col->kind != CK_KIND_BYTES && (addr % W != 0 || stride % W != 0)) return false;
    int v = 1;
    for (int cand : {16, 8, 4}) {
        const uint64_t rounded = ((uint64_t)W + cand - 1) / cand * cand;
        if (addr % cand == 0 && stride % cand == 0 && rounded <= stride) { v = cand; break; }
    }
    d->base = static_cast<const unsigned char*>(col->keys);
    d->stride = stride;
    d->key_bytes = W;
    d->kind = col->kind;
    d->nwords = (W + 3) / 4;
    d->tail_mask = (W % 4) ? (0xFFFFFFFFu << (8 * (4 - W % 4))) : 0xFFFFFFFFu;
    *vec = v;
    return true;
}

// Move masks of the compress network (Hacker's Delight, Sec. 7-4) for one
// 32-bit mask: round s moves, by 2^s places, the mask bits whose count of
// zeros to their right has bit s set.
static void compress_network(uint32_t m, uint32_t mv[5]) {
    uint32_t mk = ~m << 1;  // marks the zeros to the right of each position
    for (int s = 0; s < 5; ++s) {
        uint32_t mp = mk ^ (mk << 1);  // parallel suffix (prefix XOR from the right)
        mp ^= mp << 2;
        mp ^= mp << 4;
        mp ^= mp << 8;
        mp ^= mp << 16;
        const uint32_t move = mp & m;
        m = (m ^ move) | (move >> (1u << s));
        mk &= ~mp;
        mv[s] = move;
    }
}

static uint32_t apply_network(uint32_t x, uint32_t m, const uint32_t mv[5]) {
    x &= m;
    for (int s = 0; s < 5; ++s) {
        const uint32_t t = x & mv[s];
        x = (x ^ t) | (t >> (1u << s));
    }
    return x;
}

static uint32_t popcount64(const uint64_t* mask, uint32_t key_bits) {
    uint32_t c = 0;
    const uint32_t words = (key_bits + 63) / 64;
    for (uint32_t i = 0; i < words; ++i) {
        uint64_t w = mask[i];
        if (i == words - 1 && key_bits % 64) w &= ~0ull << (64 - key_bits % 64);
        c += (uint32_t)__builtin_popcountll(w);
    }
    return c;
}

static bool mask_fits(const uint64_t* mask, uint32_t key_bits) {
    const uint32_t words = (key_bits + 63) / 64;
    if (key_bits % 64 == 0) return true;
    return (mask[words - 1] & ~(~0ull << (64 - key_bits % 64))) == 0;  // no bits past the key
}

static ck_status cuda_status(cudaError_t e) { return e == cudaSuccess ? CK_OK : CK_ECUDA; }

// Program of one non-zero mask word (see WordProg): the runs form when the
// mask has at most two contiguous runs, else the network with only its
// non-zero rounds.  The appending fields (s1, s2, emit, kout) are set by the
// caller.
static WordProg word_program(uint32_t m) {
    WordProg p;
    memset(&p, 0, sizeof(p));
    p.mask = m;
    p.pc = (uint32_t)__builtin_popcount(m);
    uint32_t runs = 0, lo[2] = {0, 0}, len[2] = {0, 0};
    for (uint32_t b = 0; b < 32;) {  // runs from the least significant bit up
        if (!((m >> b) & 1u)) {
            ++b;
            continue;
        }
        uint32_t e = b;
        while (e < 32 && ((m >> e) & 1u)) ++e;
        if (runs < 2) {
            lo[runs] = b;
            len[runs] = e - b;
        }
        ++runs;
        b = e;
    }
    if (runs <= 2) {
        // run j moves down by the zeros below it; it lands at lo - zeros
        for (uint32_t j = 0; j < runs; ++j) {
            const uint32_t zeros = lo[j] - (j == 0 ? 0u : len[0]);
            const uint32_t field = len[j] == 32 ? 0xFFFFFFFFu : ((1u << len[j]) - 1u);
            p.mv[2 * j] = zeros;
            p.mv[2 * j + 1] = field << (lo[j] - zeros);
        }
        p.ctl = kProgRuns;
        return p;
    }
    compress_network(m, p.mv);
    for (int s = 0; s < 5; ++s)
        if (p.mv[s]) p.ctl |= 1u << s;
    return p;
}

// Host copy of the device's compress of one word under its program.
static uint32_t run_program(const WordProg& p, uint32_t x) {
    if (p.ctl & kProgRuns) return ((x >> p.mv[0]) & p.mv[1]) | ((x >> p.mv[2]) & p.mv[3]);
    x &= p.mask;
    for (int s = 0; s < 5; ++s)
        if (p.ctl & (1u << s)) {
            const uint32_t t = x & p.mv[s];
            x = (x ^ t) | (t >> (1u << s));
        }
    return x;
}

// Extraction plan of a D-bitmap: per 32-bit key word its program (how its
// D-bits are gathered and where they go in the output), plus the output
// padding.  With no set bit, first_word > last_word and only the leading zero
// words are written.
bool make_extract_plan(const KeyDesc& k, const uint64_t* dmask, uint32_t ck_words, ExtractPlan* plan) {
    memset(plan, 0, sizeof(*plan));
    const uint32_t nbits = popcount64(dmask, 8 * k.key_bytes);
    if (nbits > 32u * ck_words) return false;
    plan->K = ck_words;
    const uint32_t used = (nbits + 31) / 32;
    plan->lead_zero_words = ck_words - used;
    plan->pad_bits = 32 * used - nbits;
    plan->first_word = 0xFFFFFFFFu;
    plan->last_word = 0;
    uint32_t fill = plan->pad_bits, kout = used - 1;  // bits in the output word under construction; its index
    for (uint32_t w = 0; w < k.nwords; ++w) {
        const uint64_t mw = dmask[w / 2];
        const uint32_t m = (w % 2 == 0) ? (uint32_t)(mw >> 32) : (uint32_t)mw;
        if (!m) continue;
        WordProg p = word_program(m);
        const uint32_t e = fill + p.pc;
        if (e < 32) {
            p.ctl |= (32u - e) << 8;
            fill = e;
        } else {
            p.ctl |= ((e - 32u) << 8) | ((64u - e) << 16) | kProgEmit | (kout << 24);
            fill = e - 32u;
            --kout;
        }
        plan->prog[w] = p;
        if (plan->first_word == 0xFFFFFFFFu) plan->first_word = w;
        plan->last_word = w;
    }
    return true;
}

}  // namespace ck

using namespace ck;

extern "C" {

ck_status ck_variant_bits(const ck_column* col, uint64_t ref_row, uint64_t* mask_out, ck_stream stream) {
    KeyDesc k;
    int vec = 1;
    if (!make_key_desc(col, &k, &vec) || !mask_out) return CK_EINVAL;
    if (col->n > 0 && ref_row >= col->n) return CK_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(mask_out, 0, sizeof(uint64_t) * ((8ull * k.key_bytes + 63) / 64), s);
    if (e != cudaSuccess || col->n == 0) return cuda_status(e);
    return cuda_status(launch_variant(k, vec, col->n, ref_row, mask_out, s));
}

ck_status ck_distinction_bits(const ck_column* col, const uint32_t* order, uint64_t* mask_out, ck_stream stream) {
    KeyDesc k;
    int vec = 1;
    if (!make_key_desc(col, &k, &vec) || !mask_out) return CK_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(mask_out, 0, sizeof(uint64_t) * ((8ull * k.key_bytes + 63) / 64), s);
    if (e != cudaSuccess || col->n < 2) return cuda_status(e);
    return cuda_status(launch_dbits(k, vec, col->n, order, mask_out, s));
}

ck_status ck_extract(const ck_column* col, const uint64_t* dmask, uint32_t ck_words, uint32_t* ck_out,
                     ck_stream stream) {
    KeyDesc k;
    int vec = 1;
    if (!make_key_desc(col, &k, &vec) || !dmask || ck_words == 0 || (col->n > 0 && !ck_out)) return CK_EINVAL;
    const uint32_t key_bits = 8 * k.key_bytes;
    if (!mask_fits(dmask, key_bits)) return CK_EINVAL;
    const uint32_t nbits = popcount64(dmask, key_bits);
    if (nbits > 32u * ck_words) return CK_EOVERFLOW;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (col->n == 0) return CK_OK;
    if (nbits == 0)
        return cuda_status(cudaMemsetAsync(ck_out, 0, sizeof(uint32_t) * (size_t)ck_words * CK_LD(col->n), s));
    static thread_local ExtractPlan plan;  // ~3 KB; passed to the kernel by value
    make_extract_plan(k, dmask, ck_words, &plan);
    return cuda_status(launch_extract(k, vec, col->n, CK_LD(col->n), plan, ck_out, s));
}

ck_status ck_extract_hist(const ck_column* col, const uint64_t* dmask, uint32_t ck_words, uint32_t* ck_out,
                          uint32_t digit_bits, uint32_t* hist, ck_stream stream) {
    if (digit_bits == 0) digit_bits = 8;
    if (digit_bits < 4 || digit_bits > 11) return CK_EINVAL;
    KeyDesc k;
    int vec = 1;
    if (!make_key_desc(col, &k, &vec) || !dmask || ck_words == 0 || (col->n > 0 && !ck_out)) return CK_EINVAL;
    const uint32_t key_bits = 8 * k.key_bytes;
    if (!mask_fits(dmask, key_bits)) return CK_EINVAL;
    const uint32_t nbits = popcount64(dmask, key_bits);
    if (nbits > 32u * ck_words) return CK_EOVERFLOW;
    const uint32_t passes = (nbits + digit_bits - 1) / digit_bits;
    if (passes > 0 && !hist) return CK_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t hist_bytes = sizeof(uint32_t) * ((size_t)passes << digit_bits);
    if (passes > 0) {
        const cudaError_t e = cudaMemsetAsync(hist, 0, hist_bytes, s);
        if (e != cudaSuccess) return CK_ECUDA;
    }
    if (col->n == 0) return CK_OK;
    if (nbits == 0)
        return cuda_status(cudaMemsetAsync(ck_out, 0, sizeof(uint32_t) * (size_t)ck_words * CK_LD(col->n), s));
    static thread_local ExtractPlan plan;
    make_extract_plan(k, dmask, ck_words, &plan);
    if (hist_bytes <= kExtractHistMaxBytes)  // counted while extracting
        return cuda_status(launch_extract(k, vec, col->n, CK_LD(col->n), plan, ck_out, s, hist, digit_bits, passes));
    const cudaError_t e = launch_extract(k, vec, col->n, CK_LD(col->n), plan, ck_out, s);
    if (e != cudaSuccess) return CK_ECUDA;
    return cuda_status(launch_upsweep_all(ck_out, col->n, CK_LD(col->n), ck_words, nbits, digit_bits, hist, s));
}

size_t ck_sort_workspace_bytes(uint64_t n, uint32_t ck_words, uint32_t nbits, const ck_sort_opts* opts) {
    SortPlan p;
    if (!make_sort_plan(n, ck_words, nbits, opts ? opts->digit_bits : 0, &p, 0, opts ? opts->tile : 0)) return 0;
    return p.total;
}

ck_status ck_sort(const uint32_t* ck_in, const uint32_t* rid_in, uint32_t* ck_out, uint32_t* rid_out, uint64_t n,
                  uint32_t ck_words, uint32_t nbits, const ck_sort_opts* opts, void* ws, size_t ws_bytes,
                  ck_stream stream) {
    if (n > CK_MAX_ROWS || ck_words == 0 || nbits > 32u * ck_words) return CK_EINVAL;
    if (opts && ((opts->flags & ~CK_SORT_FLAGS_ALL) != 0 || opts->reserved != 0 ||
                 (opts->digit_bits != 0 && (opts->digit_bits < 4 || opts->digit_bits > 11)) ||
                 (opts->tile != 0 && opts->tile != 2048 && opts->tile != 4096 && opts->tile != 8192)))
        return CK_EINVAL;
    if (n == 0) return CK_OK;
    if (!ck_in || !ck_out || !rid_out) return CK_EINVAL;
    SortPlan p;
    if (!make_sort_plan(n, ck_words, nbits, opts ? opts->digit_bits : 0, &p, 0, opts ? opts->tile : 0))
        return CK_EINVAL;
    if (p.passes > 0 && (!ws || ws_bytes < p.total)) return CK_ENOMEM;
    if (p.passes > 0 && (reinterpret_cast<uintptr_t>(ws) & 255)) return CK_EINVAL;
    const uint32_t spin = (opts && opts->spin_limit) ? opts->spin_limit : (1u << 22);
    const uint32_t inject = opts ? opts->inject : 0u;
    const uint32_t flags = opts ? opts->flags : 0u;
    if (!status_ptr()) return CK_ECUDA;
    cudaEvent_t* ev = opts ? static_cast<cudaEvent_t*>(opts->pass_events) : nullptr;
    return cuda_status(run_sort(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin, inject, flags, ev,
                                static_cast<unsigned char*>(ws), reinterpret_cast<cudaStream_t>(stream),
                                opts ? opts->hist : nullptr));
}

ck_status ck_btree_plan(uint64_t n, uint32_t fanout, float fill, ck_btree_shape* shape) {
    if (!shape || n > CK_MAX_ROWS || !(fill > 0.0f) || fill > 1.0f) return CK_EINVAL;
    memset(shape, 0, sizeof(*shape));
    // f = floor(fanout * fill); the small epsilon absorbs the float rounding of fill
    const double prod = std::floor((double)fanout * (double)fill + 1e-6);
    const uint32_t f = prod < 1.0 ? 1u : (uint32_t)prod;
    shape->entries_per_node = f;
    shape->n = n;
    if (n == 0) return CK_OK;
    if (n > 1 && f < 2) return CK_EINVAL;
    uint64_t m = n;
    uint32_t l = 0;
    for (;;) {
        if (l >= CK_MAX_LEVELS) return CK_EINVAL;
        shape->level_entries[l] = m;
        shape->level_nodes[l] = (m + f - 1) / f;
        ++l;
        if (m <= f) break;
        m = (m + f - 1) / f;
    }
    shape->levels = l;
    uint64_t off = 0;
    for (uint32_t i = 1; i < l; ++i) {
        shape->inner_offset[i] = off;
        off += shape->level_entries[i];
    }
    shape->inner_entries = off;
    return CK_OK;
}

ck_status ck_build_index(const uint32_t* sorted_ck, const uint32_t* sorted_rid, uint64_t n, uint32_t ck_words,
                         const uint64_t* dmask, uint32_t key_bits, uint32_t fanout, float fill, ck_btree* tree,
                         uint64_t* refined_mask, ck_stream stream) {
    if (!tree || !dmask || ck_words == 0 || key_bits == 0 || key_bits > kMaxKeyBits) return CK_EINVAL;
    if (!mask_fits(dmask, key_bits)) return CK_EINVAL;
    ck_btree_shape shape;
    ck_status st = ck_btree_plan(n, fanout, fill, &shape);
    if (st != CK_OK) return st;
    const uint32_t nbits = popcount64(dmask, key_bits);
    if (nbits > 32u * ck_words) return CK_EOVERFLOW;
    if (n > 0 && (!sorted_ck || !sorted_rid || !tree->leaf_rid || !tree->leaf_dbit || !tree->leaf_high))
        return CK_EINVAL;
    if (shape.inner_entries > 0 && (!tree->inner_child || !tree->inner_high || !tree->inner_high_rid ||
                                    !tree->inner_high_ck || !tree->inner_dbit))
        return CK_EINVAL;
    tree->shape = shape;
    if (!status_ptr()) return CK_ECUDA;
    static thread_local BtreeArgs a;
    memset(&a, 0, sizeof(a));
    a.ck = sorted_ck;
    a.ld = CK_LD(n);
    a.rid = sorted_rid;
    a.n = n;
    a.K = ck_words;
    a.nbits = nbits;
    a.key_bits = key_bits;
    a.f = shape.entries_per_node;
    const uint32_t words = (key_bits + 63) / 64;
    for (uint32_t i = 0; i < words; ++i) a.dmask[i] = dmask[i];
    return cuda_status(launch_btree(a, shape, tree, refined_mask, reinterpret_cast<cudaStream_t>(stream)));
}

ck_status ck_build_index_keys(const ck_column* col, const uint32_t* sorted_rid, const uint64_t* dmask,
                              uint32_t ck_words, uint32_t fanout, float fill, ck_btree* tree, uint64_t* refined_mask,
                              ck_stream stream) {
    KeyDesc k;
    int vec = 1;
    if (!make_key_desc(col, &k, &vec) || !dmask || ck_words == 0 || !tree) return CK_EINVAL;
    const uint32_t key_bits = 8 * k.key_bytes;
    if (!mask_fits(dmask, key_bits)) return CK_EINVAL;
    if (popcount64(dmask, key_bits) > 32u * ck_words) return CK_EOVERFLOW;
    ck_btree_shape shape;
    ck_status st = ck_btree_plan(col->n, fanout, fill, &shape);
    if (st != CK_OK) return st;
    if (col->n > 0 && (!sorted_rid || !tree->leaf_rid || !tree->leaf_dbit || !tree->leaf_high)) return CK_EINVAL;
    if (shape.inner_entries > 0 && (!tree->inner_child || !tree->inner_high || !tree->inner_high_rid ||
                                    !tree->inner_high_ck || !tree->inner_dbit))
        return CK_EINVAL;
    tree->shape = shape;
    if (!status_ptr()) return CK_ECUDA;
    static thread_local ExtractPlan plan;
    make_extract_plan(k, dmask, ck_words, &plan);
    InnerLevels lv;
    memset(&lv, 0, sizeof(lv));
    lv.levels = shape.levels;
    lv.inner_entries = shape.inner_entries;
    for (uint32_t l = 0; l < CK_MAX_LEVELS; ++l) lv.offset[l] = shape.inner_offset[l];
    return cuda_status(launch_btree_keys(k, vec, col->n, sorted_rid, shape.entries_per_node, lv,
                                         shape.levels ? shape.level_nodes[0] : 0, plan, tree, refined_mask,
                                         reinterpret_cast<cudaStream_t>(stream)));
}

ck_status ck_device_status(uint64_t* detail) {
    if (cudaDeviceSynchronize() != cudaSuccess) return CK_ECUDA;
    unsigned long long v = 0;
    if (cudaMemcpyFromSymbol(&v, g_status_word, sizeof(v)) != cudaSuccess) return CK_ECUDA;
    if (detail) *detail = v >> 8;
    return static_cast<ck_status>(v & 0xFF);
}

ck_status ck_clear_device_status(void) {
    const unsigned long long zero = 0;
    if (cudaMemcpyToSymbol(g_status_word, &zero, sizeof(zero)) != cudaSuccess) return CK_ECUDA;
    return cudaDeviceSynchronize() == cudaSuccess ? CK_OK : CK_ECUDA;
}

const char* ck_status_string(ck_status status) {
    switch (status) {
        case CK_OK: return "CK_OK";
        case CK_EINVAL: return "CK_EINVAL: invalid argument";
        case CK_ENOMEM: return "CK_ENOMEM: workspace too small";
        case CK_ECUDA: return "CK_ECUDA: CUDA runtime error";
        case CK_EOVERFLOW: return "CK_EOVERFLOW: D-bitmap larger than the compressed key words";
        case CK_ETIMEOUT: return "CK_ETIMEOUT: a bounded device wait ran out";
        case CK_EVERIFY: return "CK_EVERIFY: verification failed, exact fallback used";
    }
    return "unknown ck_status";
}

uint64_t ck_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

uint32_t ck_compress_word_host(uint32_t x, uint32_t mask) {
    uint32_t mv[5];
    compress_network(mask, mv);
    return apply_network(x, mask, mv);
}

uint32_t ck_compress_word_program_host(uint32_t x, uint32_t mask) {
    if (!mask) return 0u;
    return run_program(word_program(mask), x);
}

}  // extern "C"

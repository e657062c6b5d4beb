// ck_scan.cu -- kernels that stream the key column once:
//   variant_kernel  variant bitmap (Sec. 4.2 / 4.3 step 3)
//   dbits_kernel    D-bitmap of adjacent sorted keys (Sec. 3.1, Theorem 1)
//   extract_kernel  Compress(key) (Sec. 3.2 / 5.1) by a per-word compress network
//
// One thread per row, grid-stride over rows.  Rows are read with the widest
// vector load the host found safe (16/8/4/1 bytes); a warp's loads of one chunk
// cover contiguous rows, so every DRAM sector of the column is fetched once.
// Bitmaps are accumulated in shared memory (one atomicOr per distinct position
// per warp) and merged into the global bitmap once per block.
#include "ck_internal.cuh"

namespace ck {

// Block-level merge of a shared bitmap (32-bit words, big-endian bit order)
// into the global uint64 bitmap (most significant first).
__device__ __forceinline__ void merge_bitmap(const uint32_t* sm, uint32_t nwords32, uint64_t* out) {
    for (uint32_t q = threadIdx.x; 2 * q < nwords32; q += blockDim.x) {
        uint64_t hi = sm[2 * q], lo = (2 * q + 1 < nwords32) ? sm[2 * q + 1] : 0u;
        uint64_t v = (hi << 32) | lo;
        if (v) atomicOr(reinterpret_cast<unsigned long long*>(out + q), (unsigned long long)v);
    }
}

// Records position p (or nothing for p < 0) in the shared bitmap; the warp's
// lanes agree on equal positions first so that each distinct position costs
// one shared atomic.
__device__ __forceinline__ void warp_mark(uint32_t* sm, int32_t p) {
    const uint32_t peers = __match_any_sync(kFull, p);
    const uint32_t lane = threadIdx.x & 31;
    if (p >= 0 && (__ffs(peers) - 1) == (int)lane) atomicOr(&sm[p >> 5], 0x80000000u >> (p & 31));
}

// ------------------------------------------------------------------ variant
// NW > 0 (keys of at most NW words): every thread ORs (row xor reference) into
// NW registers over all its rows, and the warp reduces them once at the end;
// NW = 0: a warp reduction and a shared atomic per word and 32 rows.
template <int VEC, int NW>
__global__ void __launch_bounds__(256) variant_kernel(const KeyDesc k, uint64_t n, uint64_t ref_row,
                                                      uint64_t* __restrict__ mask_out) {
    __shared__ uint32_t sm[kMaxKeyWords];
    for (uint32_t i = threadIdx.x; i < k.nwords; i += blockDim.x) sm[i] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nchunks = (k.nwords + 3) / 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (NW > 0) {
        constexpr int NC = NW > 0 ? (NW + 3) / 4 : 1;
        uint32_t ref[4 * NC], acc[4 * NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            uint32_t x[4];
            load_chunk<VEC>(k, ref_row, c, x);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ref[4 * c + i] = x[i];
                acc[4 * c + i] = 0u;
            }
        }
        for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                uint32_t x[4];
                load_chunk<VEC>(k, r, c, x);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[4 * c + i] |= x[i] ^ ref[4 * c + i];
            }
        }
#pragma unroll
        for (int w = 0; w < 4 * NC; ++w) {
            const uint32_t x = __reduce_or_sync(kFull, acc[w]);
            if (lane == 0 && x && (uint32_t)w < k.nwords) atomicOr(&sm[w], x);
        }
    } else {
        // warp-uniform trip count so that every lane takes part in the reductions
        for (uint64_t r0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); r0 < n; r0 += stride) {
            const uint64_t r = r0 + lane;
            const bool valid = r < n;
            for (uint32_t c = 0; c < nchunks; ++c) {
                uint32_t w[4] = {0, 0, 0, 0}, ref[4];
                load_chunk<VEC>(k, ref_row, c, ref);
                if (valid) load_chunk<VEC>(k, r, c, w);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t x = __reduce_or_sync(kFull, valid ? (w[i] ^ ref[i]) : 0u);
                    if (lane == 0 && x && 4 * c + i < k.nwords) atomicOr(&sm[4 * c + i], x);
                }
            }
        }
    }
    __syncthreads();
    merge_bitmap(sm, k.nwords, mask_out);
}

// ------------------------------------------------------------------ D-bits
// D-bit of rows a and b: the first differing position, or -1 if equal.
template <int VEC>
__device__ __forceinline__ int32_t key_dbit(const KeyDesc& k, uint64_t a, uint64_t b) {
    const uint32_t nchunks = (k.nwords + 3) / 4;
    for (uint32_t c = 0; c < nchunks; ++c) {
        uint32_t wa[4], wb[4];
        load_chunk<VEC>(k, a, c, wa);
        load_chunk<VEC>(k, b, c, wb);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t x = wa[i] ^ wb[i];
            if (x) return (int32_t)(32 * (4 * c + i) + __clz(x));
        }
    }
    return -1;
}

template <int VEC>
__global__ void __launch_bounds__(256) dbits_kernel(const KeyDesc k, uint64_t n, const uint32_t* __restrict__ order,
                                                    uint64_t* __restrict__ mask_out, unsigned long long* status) {
    __shared__ uint32_t sm[kMaxKeyWords];
    for (uint32_t i = threadIdx.x; i < k.nwords; i += blockDim.x) sm[i] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); r0 < n; r0 += stride) {
        const uint64_t i = r0 + lane;
        int32_t p = -1;
        if (i >= 1 && i < n) {
            const uint64_t a = order ? order[i - 1] : i - 1;
            const uint64_t b = order ? order[i] : i;
            if (a < n && b < n) p = key_dbit<VEC>(k, a, b);
            else report(status, CK_EINVAL, i);          // a row id past the column: skip it
        }
        warp_mark(sm, p);
    }
    __syncthreads();
    merge_bitmap(sm, k.nwords, mask_out);
}

// ------------------------------------------------------------------ extract
// Compress network (H. S. Warren, Hacker's Delight, 2nd ed., Sec. 7-4): with
// move masks mv[s] precomputed for the word's mask, the rounds
//   t = x & mv[s];  x = (x ^ t) | (t >> 2^s)
// gather the masked bits of x, in order, into its low popcount(mask) bits.
// The host plans each key word once (WordProg): only the rounds whose move
// mask is non-zero run, and a mask of at most two contiguous runs takes two
// shift-and-mask terms instead.  The compressed bits of successive key words
// are appended (most significant key word first) to the output word under
// construction, which starts with the output's leading zero padding; every
// full 32 bits leave as one output word, top word first.  The plan is copied
// once per block into shared memory so that every lookup is a broadcast
// shared load (indexing the kernel parameter with a runtime word index would
// serialise on the indexed constant cache).

// Digit counts of the compressed keys, gathered while they are extracted (the
// histograms a radix sort of them needs first): digit q of a key is bits
// [q * rb, q * rb + rb) of its compressed value and is counted when the word
// holding its lowest bit is emitted (the word above it, emitted just before,
// supplies the rest).  sm: passes * 2^rb shared counters; NULL: no counting.
struct HistSink {
    uint32_t* sm;
    uint32_t rb, passes;
};

__device__ __forceinline__ void count_digits(const HistSink& h, uint32_t k, uint32_t prev, uint32_t v) {
    if (h.rb == 8) {  // the bytes of the word, least significant first, are digits 4k .. 4k + 3
        uint32_t* base = h.sm + (k << 10);
#pragma unroll
        for (uint32_t b = 0; b < 4; ++b)
            if (4u * k + b < h.passes) atomicAdd(base + (b << 8) + ((v >> (8u * b)) & 255u), 1u);
        return;
    }
    const uint32_t lo_bit = 32u * k, bins = 1u << h.rb;
    const uint32_t q_lo = (lo_bit + h.rb - 1) / h.rb;
    uint32_t q_hi = (lo_bit + 31u) / h.rb;
    if (q_hi + 1 > h.passes) q_hi = h.passes - 1;
    const uint64_t both = ((uint64_t)prev << 32) | v;
    for (uint32_t q = q_lo; q <= q_hi && q < h.passes; ++q)
        atomicAdd(&h.sm[q * bins + ((uint32_t)(both >> (q * h.rb - lo_bit)) & (bins - 1u))], 1u);
}

// The network rounds selected by RM (bit s: round s) on R values at once.
// The moved bits t land on zeros of x ^ t, so the OR of a round is an
// addition, and t >> 2^s is the high word of t * 2^(32 - 2^s): one
// multiply-add (on the multiply pipe) in place of a shift and an OR (on the
// integer pipe, which the extraction saturates).
template <uint32_t RM, int R>
__device__ __forceinline__ void network_rounds(uint32_t (&x)[R], const WordProg& p) {
#pragma unroll
    for (int s = 0; s < 5; ++s)
        if (RM & (1u << s)) {
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const uint32_t t = x[q] & p.mv[s];
                x[q] = __umulhi(t, 1u << (32 - (1u << s))) + (x[q] ^ t);
            }
        }
}

// x[q] = compressed bits of word w[q] under program p.  ALL: run every round
// of the network (a round with a zero move mask changes nothing) instead of
// branching to the rounds the word needs; the host picks ALL when most words
// need most rounds, where the branch costs more than it saves.
template <int R, bool ALL>
__device__ __forceinline__ void compress_word(const WordProg& p, const uint32_t (&w)[R], uint32_t (&x)[R]) {
    if (p.ctl & kProgRuns) {
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = ((w[q] >> p.mv[0]) & p.mv[1]) | ((w[q] >> p.mv[2]) & p.mv[3]);
        return;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) x[q] = w[q] & p.mask;
    if (ALL) {
        network_rounds<31, R>(x, p);
        return;
    }
#define CK_ROUNDS_CASE(M) \
    case M: network_rounds<M, R>(x, p); break;
    switch (p.ctl & 31u) {
        CK_ROUNDS_CASE(0) CK_ROUNDS_CASE(1) CK_ROUNDS_CASE(2) CK_ROUNDS_CASE(3) CK_ROUNDS_CASE(4) CK_ROUNDS_CASE(5)
        CK_ROUNDS_CASE(6) CK_ROUNDS_CASE(7) CK_ROUNDS_CASE(8) CK_ROUNDS_CASE(9) CK_ROUNDS_CASE(10)
        CK_ROUNDS_CASE(11) CK_ROUNDS_CASE(12) CK_ROUNDS_CASE(13) CK_ROUNDS_CASE(14) CK_ROUNDS_CASE(15)
        CK_ROUNDS_CASE(16) CK_ROUNDS_CASE(17) CK_ROUNDS_CASE(18) CK_ROUNDS_CASE(19) CK_ROUNDS_CASE(20)
        CK_ROUNDS_CASE(21) CK_ROUNDS_CASE(22) CK_ROUNDS_CASE(23) CK_ROUNDS_CASE(24) CK_ROUNDS_CASE(25)
        CK_ROUNDS_CASE(26) CK_ROUNDS_CASE(27) CK_ROUNDS_CASE(28) CK_ROUNDS_CASE(29) CK_ROUNDS_CASE(30)
        default: network_rounds<31, R>(x, p); break;
    }
#undef CK_ROUNDS_CASE
}

// Copies the word programs of the chunks extract_rows visits (whole 16-byte
// chunks from first_word's to last_word's) into shared memory.
__device__ __forceinline__ void stage_programs(const ExtractPlan& plan, WordProg* wp) {
    if (plan.first_word > plan.last_word) return;
    const uint32_t w0 = plan.first_word & ~3u, w1 = plan.last_word | 3u;
    for (uint32_t w = w0 + threadIdx.x; w <= w1; w += blockDim.x) wp[w] = plan.prog[w];
}

// Compress of R rows at once: row q's chunks come from rows[q] (global or
// shared memory); each word's program is read once for all R rows.
template <int VEC, int R, bool HIST = false, bool ALL = false>
__device__ __forceinline__ void extract_rows(const KeyDesc& k, const unsigned char* const (&rows)[R],
                                             const uint64_t (&r)[R], const bool (&valid)[R], uint64_t ld,
                                             const ExtractPlan& plan, const WordProg* wp, uint32_t* __restrict__ out,
                                             const HistSink& hs = HistSink{nullptr, 0, 0}) {
    uint32_t prev[R], cur[R];
#pragma unroll
    for (int q = 0; q < R; ++q) prev[q] = cur[q] = 0u;
    for (uint32_t z = 0; z < plan.lead_zero_words; ++z) {
        const uint32_t kout = plan.K - 1 - z;
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (valid[q]) {
                out[(uint64_t)kout * ld + r[q]] = 0u;
                if (HIST) count_digits(hs, kout, 0u, 0u);
            }
    }
    const uint32_t c0 = plan.first_word >> 2, c1 = plan.last_word >> 2;
    for (uint32_t c = c0; c <= c1; ++c) {
        uint32_t w[R][4];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            if (valid[q]) load_chunk_row<VEC, false>(k, rows[q], c, w[q]);
            else w[q][0] = w[q][1] = w[q][2] = w[q][3] = 0;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const WordProg p = wp[4 * c + i];
            if (p.mask == 0) continue;
            uint32_t wi[R], x[R];
#pragma unroll
            for (int q = 0; q < R; ++q) wi[q] = w[q][i];
            compress_word<R, ALL>(p, wi, x);
            const uint32_t s1 = (p.ctl >> 8) & 63u;
            if (!(p.ctl & kProgEmit)) {
#pragma unroll
                for (int q = 0; q < R; ++q) cur[q] |= x[q] << s1;
                continue;
            }
            const uint32_t s2 = (p.ctl >> 16) & 63u, kout = p.ctl >> 24;
            uint32_t* o = out + (uint64_t)kout * ld;
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const uint32_t word = cur[q] | (x[q] >> s1);
                cur[q] = __funnelshift_lc(0u, x[q], s2);  // x << s2; 0 for s2 = 32
                if (valid[q]) {
                    o[r[q]] = word;
                    if (HIST) {
                        count_digits(hs, kout, prev[q], word);
                        prev[q] = word;
                    }
                }
            }
        }
    }
}

// Persistent extraction with TMA staging: block b takes row tiles b, b + G,
// b + 2G, ...; each full tile (rows_per_tile rows, contiguous in memory
// because row_stride * rows_per_tile is a multiple of 16) arrives in a ring of
// kExtractStages shared buffers by one bulk copy, issued kExtractStages tiles
// ahead.  The ragged last tile is read straight from global memory.  Each
// thread extracts kExtractRows rows of a tile together, as often as the tile
// needs.
constexpr int kExtractStages = 4;       // ring depth without digit counting
constexpr int kExtractStagesHist = 3;   // with it (room for the counters, three blocks per SM)
constexpr int kExtractThreads = 256;
constexpr int kExtractRows = 2;

template <int VEC, bool HIST, bool ALL>
__global__ void __launch_bounds__(kExtractThreads, 3) extract_kernel(const KeyDesc k, uint64_t n, uint64_t ld,
                                                                  uint32_t rows_per_tile, uint32_t staged,
                                                                  const __grid_constant__ ExtractPlan plan,
                                                                  uint32_t* __restrict__ out, uint32_t spin_limit,
                                                                  unsigned long long* status,
                                                                  uint32_t* __restrict__ hist, uint32_t rb,
                                                                  uint32_t passes) {
    constexpr int R = kExtractRows;
    constexpr int kExtractStages = HIST ? kExtractStagesHist : ck::kExtractStages;
    extern __shared__ __align__(128) unsigned char sm[];
    const uint32_t tile_bytes = staged ? rows_per_tile * (uint32_t)k.stride : 0u;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + (size_t)kExtractStages * tile_bytes);
    WordProg* wp = reinterpret_cast<WordProg*>(bar + kExtractStages);
    uint32_t* hsm = reinterpret_cast<uint32_t*>(wp + kMaxKeyWords);
    const uint32_t nctr = passes << rb;
    if constexpr (HIST)
        for (uint32_t i = threadIdx.x; i < nctr; i += kExtractThreads) hsm[i] = 0u;
    const HistSink hs{hsm, rb, passes};
    const uint64_t tiles = (n + rows_per_tile - 1) / rows_per_tile;
    const uint64_t full_tiles = staged ? n / rows_per_tile : 0;  // tiles that arrive by bulk copy
    const uint32_t tid = threadIdx.x;
    stage_programs(plan, wp);
    if (tid == 0 && staged) {
        for (int b = 0; b < kExtractStages; ++b) mbar_init(&bar[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](uint64_t i) {  // thread 0: local tile i into stage i % kExtractStages
        const uint64_t t = blockIdx.x + i * gridDim.x;
        if (t < full_tiles)
            bulk_load(sm + (size_t)(i % kExtractStages) * tile_bytes, k.base + t * rows_per_tile * k.stride,
                      tile_bytes, &bar[i % kExtractStages]);
    };
    if (tid == 0)
        for (uint64_t i = 0; i < (uint64_t)kExtractStages; ++i) issue(i);
    for (uint64_t i = 0;; ++i) {
        const uint64_t t = blockIdx.x + i * gridDim.x;
        if (t >= tiles) break;
        const uint64_t r0 = t * rows_per_tile;
        const unsigned char* base = k.base + r0 * k.stride;
        if (t < full_tiles) {
            const uint32_t st = (uint32_t)(i % kExtractStages);
            if (!mbar_wait(&bar[st], (uint32_t)(i / kExtractStages) & 1u, spin_limit))
                report(status, CK_ETIMEOUT, t);
            base = sm + (size_t)st * tile_bytes;
        }
        const uint64_t nrows = min((uint64_t)rows_per_tile, n - r0);
        for (uint32_t j0 = tid; j0 < nrows; j0 += R * kExtractThreads) {
            const unsigned char* rows[R];
            uint64_t r[R];
            bool valid[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const uint64_t j = j0 + (uint64_t)q * kExtractThreads;
                valid[q] = j < nrows;
                r[q] = r0 + j;
                rows[q] = base + (valid[q] ? j : 0) * k.stride;
            }
            extract_rows<VEC, R, HIST, ALL>(k, rows, r, valid, ld, plan, wp, out, hs);
        }
        __syncthreads();  // stage i % kExtractStages is free again
        if (tid == 0) {
            fence_proxy_async_smem();
            issue(i + kExtractStages);
        }
    }
    if constexpr (HIST) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nctr; i += kExtractThreads)
            if (hsm[i]) atomicAdd(&hist[i], hsm[i]);
    }
}

// ------------------------------------------------- bulk load from full keys
// The tree of ck_build_index, built from the key column and the sorted row
// ids alone (no sorted compressed keys): a leaf's D-bit is the D-bit of the
// two full keys it compares, gathered by row id -- by Sec. 5.3 the same value
// D-offset maps the compressed D-bit to -- and an inner entry's compressed
// highest key is extracted from its full key on the spot.
__device__ __forceinline__ void merge_bitmap_bits(const uint32_t* sm, uint32_t nwords32, uint64_t* out) {
    merge_bitmap(sm, nwords32, out);
}

template <int VEC>
__global__ void __launch_bounds__(256) leaf_keys_kernel(const KeyDesc k, uint64_t n, const uint32_t* __restrict__ rid,
                                                        uint32_t f, uint32_t* __restrict__ leaf_rid,
                                                        uint16_t* __restrict__ leaf_dbit,
                                                        uint32_t* __restrict__ leaf_high, uint64_t nodes0,
                                                        uint64_t* __restrict__ refined, unsigned long long* status) {
    __shared__ uint32_t sm[kMaxKeyWords];
    for (uint32_t i = threadIdx.x; i < k.nwords; i += blockDim.x) sm[i] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
        const uint64_t i = i0 + lane;
        int32_t p = -1;
        if (i < n) {
            const uint32_t b = rid[i];
            if (leaf_rid) leaf_rid[i] = b;  // NULL: the row ids already are the tree's
            if (i > 0) {
                const uint32_t a = rid[i - 1];
                if (a < n && b < n) p = key_dbit<VEC>(k, a, b);
                else report(status, CK_EINVAL, i);
            }
            leaf_dbit[i] = p >= 0 ? (uint16_t)p : (uint16_t)CK_NO_DBIT;
            if (i < nodes0) leaf_high[i] = (uint32_t)(min((i + 1) * (uint64_t)f, n) - 1);
        }
        if (refined) warp_mark(sm, p);
    }
    if (!refined) return;
    __syncthreads();
    merge_bitmap(sm, k.nwords, refined);
}

template <int VEC>
__global__ void __launch_bounds__(256) inner_keys_kernel(const KeyDesc k, uint64_t n, const uint32_t* __restrict__ rid,
                                                         uint32_t f, const __grid_constant__ InnerLevels lv,
                                                         const __grid_constant__ ExtractPlan plan,
                                                         uint32_t* __restrict__ child, uint32_t* __restrict__ high,
                                                         uint32_t* __restrict__ high_rid,
                                                         uint32_t* __restrict__ high_ck, uint16_t* __restrict__ dbit,
                                                         unsigned long long* status) {
    __shared__ WordProg wp[kMaxKeyWords];
    stage_programs(plan, wp);
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < lv.inner_entries; g += stride) {
        uint32_t l = 1;
        while (l + 1 < lv.levels && g >= lv.offset[l + 1]) ++l;
        const uint64_t e = g - lv.offset[l];
        uint64_t span = 1;  // f^l, capped at n (a capped span only occurs when the level has one entry)
        for (uint32_t t = 0; t < l; ++t) span = min(span * f, n);
        const uint64_t hi = min((e + 1) * span, n) - 1;
        const uint32_t r = rid[hi];
        child[g] = (uint32_t)e;
        high[g] = (uint32_t)hi;
        high_rid[g] = r;
        int32_t p = -1;
        if (r < n) {
            const unsigned char* rows[1] = {k.base + (uint64_t)r * k.stride};
            const uint64_t rr[1] = {g * plan.K};
            const bool valid[1] = {true};
            extract_rows<VEC, 1>(k, rows, rr, valid, 1, plan, wp, high_ck);  // entry-major: ld = 1
            if (e > 0) {
                const uint32_t a = rid[e * span - 1];
                if (a < n) p = key_dbit<VEC>(k, a, r);
                else report(status, CK_EINVAL, e * span - 1);
            }
        } else {
            report(status, CK_EINVAL, hi);
        }
        dbit[g] = p >= 0 ? (uint16_t)p : (uint16_t)CK_NO_DBIT;
    }
}

// ------------------------------------------------------------------ launchers
static unsigned grid_for(uint64_t n, unsigned threads) {
    const uint64_t want = (n + threads - 1) / threads;
    const uint64_t cap = (uint64_t)num_sms() * 8;
    return (unsigned)(want < cap ? (want ? want : 1) : cap);
}

#define CK_DISPATCH_VEC(vec, KERNEL, ...)                                      \
    switch (vec) {                                                             \
        case 16: KERNEL<16><<<grid, 256, 0, s>>>(__VA_ARGS__); break;          \
        case 8: KERNEL<8><<<grid, 256, 0, s>>>(__VA_ARGS__); break;            \
        case 4: KERNEL<4><<<grid, 256, 0, s>>>(__VA_ARGS__); break;            \
        default: KERNEL<1><<<grid, 256, 0, s>>>(__VA_ARGS__); break;           \
    }

template <int NW>
static void launch_variant_nw(const KeyDesc& k, int vec, uint64_t n, uint64_t ref_row, uint64_t* mask_out,
                              unsigned grid, cudaStream_t s) {
    switch (vec) {
        case 16: variant_kernel<16, NW><<<grid, 256, 0, s>>>(k, n, ref_row, mask_out); break;
        case 8: variant_kernel<8, NW><<<grid, 256, 0, s>>>(k, n, ref_row, mask_out); break;
        case 4: variant_kernel<4, NW><<<grid, 256, 0, s>>>(k, n, ref_row, mask_out); break;
        default: variant_kernel<1, NW><<<grid, 256, 0, s>>>(k, n, ref_row, mask_out); break;
    }
}

cudaError_t launch_variant(const KeyDesc& k, int vec, uint64_t n, uint64_t ref_row, uint64_t* mask_out,
                           cudaStream_t s) {
    const unsigned grid = grid_for(n, 256);
    if (k.nwords <= 4) launch_variant_nw<4>(k, vec, n, ref_row, mask_out, grid, s);
    else if (k.nwords <= 8) launch_variant_nw<8>(k, vec, n, ref_row, mask_out, grid, s);
    else launch_variant_nw<0>(k, vec, n, ref_row, mask_out, grid, s);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_dbits(const KeyDesc& k, int vec, uint64_t n, const uint32_t* order, uint64_t* mask_out,
                         cudaStream_t s) {
    const unsigned grid = grid_for(n, 256);
    CK_DISPATCH_VEC(vec, dbits_kernel, k, n, order, mask_out, status_ptr());
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_btree_keys(const KeyDesc& k, int vec, uint64_t n, const uint32_t* rid, uint32_t f,
                              const InnerLevels& lv, uint64_t nodes0, const ExtractPlan& plan, ck_btree* t,
                              uint64_t* refined, cudaStream_t s) {
    if (refined) {
        cudaError_t e = cudaMemsetAsync(refined, 0, sizeof(uint64_t) * ((8ull * k.key_bytes + 63) / 64), s);
        if (e != cudaSuccess) return e;
    }
    if (n == 0) return cudaSuccess;
    unsigned grid = grid_for(n, 256);
    uint32_t* lr = t->leaf_rid == rid ? nullptr : t->leaf_rid;
    CK_DISPATCH_VEC(vec, leaf_keys_kernel, k, n, rid, f, lr, t->leaf_dbit, t->leaf_high, nodes0, refined,
                    status_ptr());
    count_launch();
    if (lv.inner_entries > 0) {
        grid = grid_for(lv.inner_entries, 256);
        CK_DISPATCH_VEC(vec, inner_keys_kernel, k, n, rid, f, lv, plan, t->inner_child, t->inner_high,
                        t->inner_high_rid, t->inner_high_ck, t->inner_dbit, status_ptr());
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_extract(const KeyDesc& k, int vec, uint64_t n, uint64_t ld, const ExtractPlan& plan,
                           uint32_t* ck_out, cudaStream_t s, uint32_t* hist, uint32_t rb, uint32_t passes) {
    // rows per tile: a multiple of 16 (so that tiles start 16-byte aligned),
    // about 16 KB of keys (short keys: several rows per thread and tile).
    // Staging needs a 16-byte aligned column and a ring that fits shared memory.
    const bool counting = hist != nullptr && passes > 0;
    const uint32_t stages = counting ? kExtractStagesHist : kExtractStages;
    uint32_t rows = (uint32_t)(16384 / k.stride) & ~15u;
    if (rows < 16) rows = 16;
    const bool staged = (reinterpret_cast<uintptr_t>(k.base) & 15) == 0 &&
                        (uint64_t)stages * rows * k.stride <= 160 * 1024;
    if (!staged) rows = kExtractRows * kExtractThreads;
    const size_t smem = (staged ? (size_t)stages * rows * k.stride : 0) + stages * sizeof(uint64_t) +
                        sizeof(WordProg) * kMaxKeyWords + (counting ? sizeof(uint32_t) * ((size_t)passes << rb) : 0);
    const uint64_t tiles = (n + rows - 1) / rows;
    const uint64_t cap = (uint64_t)num_sms() * 3;
    const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
    cudaError_t e = cudaSuccess;
    // every network round for all words when the network words need, on
    // average, at least four of the five rounds
    uint32_t nnet = 0, rounds = 0;
    for (uint32_t w = plan.first_word; plan.first_word <= plan.last_word && w <= plan.last_word; ++w)
        if (plan.prog[w].mask && !(plan.prog[w].ctl & kProgRuns)) {
            ++nnet;
            rounds += (uint32_t)__builtin_popcount(plan.prog[w].ctl & 31u);
        }
    const bool all = nnet > 0 && rounds >= 4 * nnet;
#define CK_EXTRACT_LAUNCH(V, H, A)                                                                              \
    e = cudaFuncSetAttribute(extract_kernel<V, H, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                                             \
    extract_kernel<V, H, A><<<grid, kExtractThreads, smem, s>>>(k, n, ld, rows, staged ? 1u : 0u, plan, ck_out,  \
                                                                 kDefaultSpin, status_ptr(), hist, rb, passes);
#define CK_EXTRACT_VEC(H, A)                          \
    switch (vec) {                                    \
        case 16: CK_EXTRACT_LAUNCH(16, H, A); break;  \
        case 8: CK_EXTRACT_LAUNCH(8, H, A); break;    \
        case 4: CK_EXTRACT_LAUNCH(4, H, A); break;    \
        default: CK_EXTRACT_LAUNCH(1, H, A); break;   \
    }
    if (counting) {
        if (all) {
            CK_EXTRACT_VEC(true, true)
        } else {
            CK_EXTRACT_VEC(true, false)
        }
    } else {
        if (all) {
            CK_EXTRACT_VEC(false, true)
        } else {
            CK_EXTRACT_VEC(false, false)
        }
    }
#undef CK_EXTRACT_VEC
#undef CK_EXTRACT_LAUNCH
    count_launch();
    return cudaGetLastError();
}

}  // namespace ck

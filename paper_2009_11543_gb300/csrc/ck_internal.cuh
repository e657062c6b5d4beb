// ck_internal.cuh -- shared device helpers and host launch declarations of libck.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ck.h"

namespace ck {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kMaxKeyWords = CK_MAX_KEY_BYTES / 4;  // 32-bit key words
constexpr uint32_t kMaxMaskWords = CK_MAX_KEY_BYTES / 8;  // uint64 bitmap words
constexpr uint32_t kMaxKeyBits = CK_MAX_KEY_BYTES * 8;

// ---------------------------------------------------------------- status word
// Keeps the first error: code in bits 0..7, detail above.
__device__ __forceinline__ void report(unsigned long long* status, uint32_t code, uint64_t detail) {
    atomicCAS(status, 0ull, (unsigned long long)code | ((unsigned long long)detail << 8));
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ------------------------------------------------- TMA bulk copy + mbarrier
// One-dimensional bulk copies (global -> shared) signal an mbarrier with the
// bytes they deliver; consumers poll the barrier's phase with a bounded loop.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The calling thread arrives once on bar and announces `bytes` more bytes,
// then starts the copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) that completes them.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Tests whether the phase with the given parity has completed; a thread
// whose phase is not complete is suspended for up to about 1 us (it resumes as soon as the phase
// completes), so a waiting warp does not compete for issue slots.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "n"(1000)
        : "memory");
    return ok != 0;
}

// Waits for the phase with the given parity to complete; gives up after
// about limit / 4 suspended tries (each up to 1 us) and returns false (the
// caller records the timeout).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
    const uint32_t tries = limit / 4 + 1;
    for (uint32_t i = 0; i < tries; ++i)
        if (mbar_try_wait_sleep(bar, parity)) return true;
    return false;
}

// ------------------------------------------------------------- key loading
// A key is presented as a sequence of 32-bit words in big-endian bit order:
// word w holds key positions [32w, 32w + 32), position 32w in bit 31.
//   BYTES: word w = bytes 4w..4w+3 of the row, byte 4w most significant;
//   U32:   word 0 = the value;
//   U64:   word 0 = high half, word 1 = low half of the value;
//   I32 / I64, F32 / F64: the same for the value mapped to its order-preserving
//   form (sign bit flipped; a negative float's bits all inverted).
// Bytes at or past key_bytes read as zero.  VEC is the load width in bytes
// (16, 8, 4 or 1), chosen by the host so that every vector load stays inside
// the row's stride.
struct KeyDesc {
    const unsigned char* base;
    uint64_t stride;
    uint32_t key_bytes;
    uint32_t kind;
    uint32_t nwords;      // ceil(key_bytes / 4)
    uint32_t tail_mask;   // valid bits of the last word (big-endian order)
};

__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// Loads 16 bytes worth of words starting at word 4c of row r.  Words past the
// key read 0.  Only the word indices [4c, 4c+4) are produced.
template <int VEC, bool TAIL = true>
__device__ __forceinline__ void load_chunk_row(const KeyDesc& k, const unsigned char* row, uint32_t c,
                                               uint32_t (&w)[4]);

template <int VEC>
__device__ __forceinline__ void load_chunk(const KeyDesc& k, uint64_t r, uint32_t c, uint32_t (&w)[4]) {
    load_chunk_row<VEC>(k, k.base + r * k.stride, c, w);
}

// Same, for a row that starts at `row` (global or shared memory).  TAIL =
// false leaves the bytes past key_bytes of byte keys as loaded (for callers
// that mask them away).
template <int VEC, bool TAIL>
__device__ __forceinline__ void load_chunk_row(const KeyDesc& k, const unsigned char* row, uint32_t c,
                                               uint32_t (&w)[4]) {
    if (k.kind == CK_KIND_U64 || k.kind == CK_KIND_I64 || k.kind == CK_KIND_F64) {  // 8-byte value; chunk 0 only
        const uint2 v = *reinterpret_cast<const uint2*>(row);
        uint32_t hi = v.y, lo = v.x;
        if (k.kind == CK_KIND_I64) {
            hi ^= 0x80000000u;
        } else if (k.kind == CK_KIND_F64) {
            if (hi >> 31) {
                hi = ~hi;
                lo = ~lo;
            } else {
                hi ^= 0x80000000u;
            }
        }
        w[0] = hi; w[1] = lo; w[2] = 0; w[3] = 0;
        return;
    }
    if (k.kind != CK_KIND_BYTES) {          // 4-byte value
        uint32_t x = *reinterpret_cast<const uint32_t*>(row);
        if (k.kind == CK_KIND_I32) x ^= 0x80000000u;
        else if (k.kind == CK_KIND_F32) x = (x >> 31) ? ~x : (x ^ 0x80000000u);
        w[0] = x; w[1] = 0; w[2] = 0; w[3] = 0;
        return;
    }
    const uint32_t first = 4 * c;
    if (VEC == 16) {
        uint4 v = *reinterpret_cast<const uint4*>(row + 16 * c);
        w[0] = bswap32(v.x); w[1] = bswap32(v.y); w[2] = bswap32(v.z); w[3] = bswap32(v.w);
    } else if (VEC == 8) {
        uint2 a = *reinterpret_cast<const uint2*>(row + 16 * c);
        uint2 b = (first + 2 < k.nwords) ? *reinterpret_cast<const uint2*>(row + 16 * c + 8) : make_uint2(0, 0);
        w[0] = bswap32(a.x); w[1] = bswap32(a.y); w[2] = bswap32(b.x); w[3] = bswap32(b.y);
    } else if (VEC == 4) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            w[i] = (first + i < k.nwords) ? bswap32(*reinterpret_cast<const uint32_t*>(row + 16 * c + 4 * i)) : 0u;
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t x = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                uint32_t byte = 16 * c + 4 * i + b;
                x = (x << 8) | (byte < k.key_bytes ? (uint32_t)row[byte] : 0u);
            }
            w[i] = x;
        }
    }
    // zero the bytes past key_bytes inside the last word
    if (TAIL) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (first + i == k.nwords - 1) w[i] &= k.tail_mask;
            else if (first + i >= k.nwords) w[i] = 0;
    }
}


// A key of a column: row r of column k.
struct KeyRef {
    const KeyDesc* k;
    uint64_t r;
};

// -1, 0, 1: lexicographic comparison of two keys of equal width (Sec. 4.1).
template <int VEC>
__device__ __forceinline__ int cmp_keys(const KeyRef& a, const KeyRef& b) {
    const uint32_t nchunks = (a.k->nwords + 3) / 4;
    for (uint32_t c = 0; c < nchunks; ++c) {
        uint32_t wa[4], wb[4];
        load_chunk<VEC>(*a.k, a.r, c, wa);
        load_chunk<VEC>(*b.k, b.r, c, wb);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (wa[i] != wb[i]) return wa[i] < wb[i] ? -1 : 1;
    }
    return 0;
}

// D-bit of two keys (Sec. 3.1): the first differing position; -1 if equal.
template <int VEC>
__device__ __forceinline__ int32_t dbit_keys(const KeyRef& a, const KeyRef& b) {
    const uint32_t nchunks = (a.k->nwords + 3) / 4;
    for (uint32_t c = 0; c < nchunks; ++c) {
        uint32_t wa[4], wb[4];
        load_chunk<VEC>(*a.k, a.r, c, wa);
        load_chunk<VEC>(*b.k, b.r, c, wb);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t x = wa[i] ^ wb[i];
            if (x) return (int32_t)(32 * (4 * c + i) + __clz(x));
        }
    }
    return -1;
}


// Exclusive scan in place over count entries of arr (shared or global memory)
// by one block; returns the total.  scratch: THREADS/32 + 1 shared words.
template <int THREADS>
__device__ uint32_t block_exclusive_scan(uint32_t* arr, int count, uint32_t* scratch) {
    constexpr int WARPS = THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (count + THREADS - 1) / THREADS;
    const int beg = tid * per;
    uint32_t sum = 0;
    for (int i = 0; i < per; ++i)
        if (beg + i < count) sum += arr[beg + i];
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = lane < WARPS ? scratch[lane] : 0u;
        uint32_t vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, vi, o);
            if (lane >= o) vi += t;
        }
        if (lane < WARPS) scratch[lane] = vi - v;
        if (lane == 31) scratch[WARPS] = vi;
    }
    __syncthreads();
    uint32_t run = scratch[warp] + inc - sum;
    for (int i = 0; i < per; ++i)
        if (beg + i < count) {
            const uint32_t t = arr[beg + i];
            arr[beg + i] = run;
            run += t;
        }
    const uint32_t total = scratch[WARPS];
    __syncthreads();
    return total;
}


// Word w of row r (0 past the key).
template <int VEC>
__device__ __forceinline__ uint32_t key_word(const KeyDesc& k, uint64_t r, uint32_t w) {
    if (w >= k.nwords) return 0u;
    uint32_t c[4];
    load_chunk<VEC>(k, r, w >> 2, c);
    return c[w & 3];
}

// Sign of a - b and, when they differ, their D-bit.
template <int VEC>
__device__ __forceinline__ int cmp_dbit(const KeyRef& a, const KeyRef& b, int32_t* d) {
    const uint32_t nchunks = (a.k->nwords + 3) / 4;
    for (uint32_t c = 0; c < nchunks; ++c) {
        uint32_t wa[4], wb[4];
        load_chunk<VEC>(*a.k, a.r, c, wa);
        load_chunk<VEC>(*b.k, b.r, c, wb);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t x = wa[i] ^ wb[i];
            if (x) {
                *d = (int32_t)(32 * (4 * c + i) + __clz(x));
                return wa[i] < wb[i] ? -1 : 1;
            }
        }
    }
    *d = -1;
    return 0;
}

// The query of one thread.  QW > 0: its key words (QW >= the key's words) are
// held in registers, so a comparison loads only the other key and the
// partial-key window costs no load; QW = 0: read from the query column.
template <int VEC, int QW>
struct QueryView {
    const KeyDesc* qk;
    uint64_t j;
    uint32_t w[QW > 0 ? QW : 1];

    __device__ __forceinline__ QueryView(const KeyDesc& k, uint64_t row) : qk(&k), j(row) {
        if (QW > 0) {
#pragma unroll
            for (int c = 0; c < (QW + 3) / 4; ++c) {
                uint32_t x[4];
                load_chunk<VEC>(k, row, c, x);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (4 * c + i < QW) w[4 * c + i] = x[i];
            }
        }
    }

    // Sign of key(col, r) - query and, when they differ, their D-bit.
    __device__ __forceinline__ int cmp(const KeyDesc& col, uint64_t r, int32_t* d) const {
        if (QW == 0) return cmp_dbit<VEC>(KeyRef{&col, r}, KeyRef{qk, j}, d);
#pragma unroll
        for (int c = 0; c < (QW + 3) / 4; ++c) {
            uint32_t x[4];
            load_chunk<VEC>(col, r, c, x);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (4 * c + i >= QW) break;
                const uint32_t y = x[i] ^ w[4 * c + i];
                if (y) {
                    *d = (int32_t)(32 * (4 * c + i) + __clz(y));
                    return x[i] < w[4 * c + i] ? -1 : 1;
                }
            }
        }
        *d = -1;
        return 0;
    }

    // The query's positions p0 .. p0 + pk - 1 as a pk-bit value.
    __device__ __forceinline__ uint32_t window(uint32_t p0, uint32_t pk) const {
        const uint32_t wi = p0 >> 5;
        uint32_t hi = 0, lo = 0;
        if (QW == 0) {
            hi = key_word<VEC>(*qk, j, wi);
            lo = key_word<VEC>(*qk, j, wi + 1);
        } else {
#pragma unroll
            for (int k = 0; k < (QW > 0 ? QW : 1); ++k) {
                hi |= w[k] & (0u - (uint32_t)((uint32_t)k == wi));      // masks, not an index:
                lo |= w[k] & (0u - (uint32_t)((uint32_t)k == wi + 1));  // w stays in registers
            }
        }
        return (uint32_t)(((((uint64_t)hi << 32) | lo) << (p0 & 31)) >> (64 - pk));
    }
};

}  // namespace ck

// ------------------------------------------------------------ host helpers
namespace ck {
int num_sms();
unsigned long long* status_ptr();     // device address of the status word (current device)
void count_launch(uint32_t k = 1);
bool make_key_desc(const ck_column* col, KeyDesc* d, int* vec);

// launchers (each returns a CUDA error code of the launch)
cudaError_t launch_variant(const KeyDesc& k, int vec, uint64_t n, uint64_t ref_row, uint64_t* mask_out,
                           cudaStream_t s);
cudaError_t launch_dbits(const KeyDesc& k, int vec, uint64_t n, const uint32_t* order, uint64_t* mask_out,
                         cudaStream_t s);

// The extraction's program for one 32-bit key word, the same for every row.
// Its D-bits are gathered into the low popcount(mask) bits of a value x in one
// of two forms, then x is appended to the output word under construction.
//   network form: x = word & mask, then the rounds of the compress network
//     whose move masks are non-zero (ctl bits 0-4; mv[s] moves by 2^s);
//   runs form (ctl kProgRuns; masks of at most two contiguous runs):
//     x = ((word >> mv[0]) & mv[1]) | ((word >> mv[2]) & mv[3]).
// Appending: with e = (bits already in the output word) + popcount(mask),
//   e < 32:  cur |= x << s1;
//   e >= 32: the output word cur | (x >> s1) is complete and stored as
//            compressed word `kout` (ctl bits 24-31); cur = x << s2 (s2 = 32:
//            nothing is left over).
struct WordProg {
    uint32_t mask;   // D's positions in this word, big-endian bit order; 0: the word adds nothing
    uint32_t mv[5];  // network: move masks; runs: shift, mask, shift, mask
    uint32_t ctl;    // bits 0-4 rounds, 5 runs form, 8-13 s1, 16-21 s2, 22 emits, 24-31 kout
    uint32_t pc;     // popcount(mask)
};
constexpr uint32_t kProgRuns = 1u << 5;
constexpr uint32_t kProgEmit = 1u << 22;

struct ExtractPlan {
    uint32_t first_word, last_word;  // words with a non-zero mask
    uint32_t K;                      // output words
    uint32_t lead_zero_words;        // whole zero words at the top of the output
    uint32_t pad_bits;               // zero bits at the top of the first non-zero output word
    uint32_t pad[3];
    WordProg prog[kMaxKeyWords];     // per key word (zero outside first_word .. last_word)
};
// hist (device, passes * 2^rb counters, zeroed by the caller) != NULL: the
// digit counts of the compressed keys are added to it in the same pass.
cudaError_t launch_extract(const KeyDesc& k, int vec, uint64_t n, uint64_t ld, const ExtractPlan& plan,
                           uint32_t* ck_out, cudaStream_t s, uint32_t* hist = nullptr, uint32_t rb = 0,
                           uint32_t passes = 0);
constexpr size_t kExtractHistMaxBytes = 16 * 1024;  // counters the fused extraction keeps in shared memory
// All digit histograms of compressed keys already in memory (the sort's upsweep).
cudaError_t launch_upsweep_all(const uint32_t* ck, uint64_t n, uint64_t ld, uint32_t K, uint32_t nbits, uint32_t rb,
                               uint32_t* hist, cudaStream_t s);
constexpr uint32_t kDefaultSpin = 1u << 22;  // polls before a device wait gives up

struct InnerLevels {
    uint32_t levels;
    uint64_t inner_entries;
    uint64_t offset[CK_MAX_LEVELS];  // start of level l in the inner arrays
};
cudaError_t launch_btree_keys(const KeyDesc& k, int vec, uint64_t n, const uint32_t* rid, uint32_t f,
                              const InnerLevels& lv, uint64_t nodes0, const ExtractPlan& plan, ck_btree* t,
                              uint64_t* refined, cudaStream_t s);
bool make_extract_plan(const KeyDesc& k, const uint64_t* dmask, uint32_t ck_words, ExtractPlan* plan);

constexpr int kPassTile = (int)CK_SORT_TILE;      // pairs per onesweep tile
constexpr int kMaxPassArrays = kMaxKeyWords + 2;  // key words, row ids, one extra
constexpr uint32_t kLookbackFlagAgg = 1u << 30;

// The arrays a pass moves, in staging order.  Array 0 (and array 1 when the
// digit straddles two words) holds the digit.  A NULL source means the values
// are the input positions (row ids 0..n-1; such an array takes no ring slot);
// a NULL destination means the array is read for its digit but not carried on.
struct PassArrays {
    const uint32_t* src[kMaxPassArrays];
    uint32_t* dst[kMaxPassArrays];
};

struct PassArgs {
    uint64_t n;
    uint32_t narr;                // arrays in PassArrays
    uint32_t sh, bits, straddle;  // digit = bits [sh, sh + bits) of array 0 (spilling into array 1)
    uint32_t pass;
    uint32_t bulk;                // 1: every array is 16-byte aligned, full tiles stage by TMA
    const uint32_t* bucket_base;  // [BINS] of this pass
    uint32_t* lookback;           // [tiles][BINS] of this pass, zeroed
    uint32_t* tile_counter;       // zeroed
    uint32_t spin_limit, inject;
    unsigned long long* status;
    const uint32_t* gate;         // NULL, or: the pass runs only while *gate == gate_run (decided on the device)
    uint32_t gate_run;
    uint32_t tiles;               // set by the launcher
};

// One onesweep pass with digit width rb (4..11); tiles = ceil(n / kPassTile).
// tile: pairs per tile, kPassTile (default), 2048 or 8192.
cudaError_t launch_onesweep_pass(uint32_t rb, const PassArgs& a, const PassArrays& arrays, uint32_t tiles,
                                 cudaStream_t s, uint32_t tile = kPassTile);
// Exclusive scan, in place, of `sets` histograms of 2^rb bins (rb <= 8).
cudaError_t launch_bucket_scan(uint32_t* hist, uint32_t sets, uint32_t rb, cudaStream_t s);

struct SortPlan {
    uint32_t digit_bits, passes, tile, tiles, K;
    uint64_t ld;  // leading dimension of the word arrays (input, output and scratch)
    size_t off_hist, off_counter, off_lookback, off_alt_ck, off_alt_rid, total;
};
// ld == 0 selects CK_LD(n); a larger ld sorts a segment of wider arrays in place.
// tile: pairs per radix tile, 0 = kPassTile; 2048, 4096 and 8192 are valid.
bool make_sort_plan(uint64_t n, uint32_t K, uint32_t nbits, uint32_t digit_bits, SortPlan* p, uint64_t ld = 0,
                    uint32_t tile = 0);
// gate != NULL: every kernel of the sort returns at once unless *gate != 0
// when it runs (a sort the device decides to need; the launches are made
// either way, so the host never waits for the decision).  A gated sort must
// not be in place, must have passes > 0 and takes no hist_in.
cudaError_t run_sort(const SortPlan& p, const uint32_t* ck_in, const uint32_t* rid_in, uint32_t* ck_out,
                     uint32_t* rid_out, uint64_t n, uint32_t nbits, uint32_t spin_limit, uint32_t inject,
                     uint32_t flags, cudaEvent_t* pass_events, unsigned char* ws, cudaStream_t s,
                     const uint32_t* hist_in = nullptr, const uint32_t* gate = nullptr);

struct BtreeArgs {
    const uint32_t* ck;  // word-major, K words, leading dimension ld
    uint64_t ld;
    const uint32_t* rid;
    uint64_t n;
    uint32_t K, nbits, key_bits, f;
    uint64_t dmask[kMaxMaskWords];
};
cudaError_t launch_btree(const BtreeArgs& a, const ck_btree_shape& shape, ck_btree* t, uint64_t* refined,
                         cudaStream_t s);
}  // namespace ck

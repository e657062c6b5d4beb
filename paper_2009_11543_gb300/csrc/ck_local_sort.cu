// ck_local_sort.cu -- the second half of the learned-partition sort (not in the
// paper): after the partition every bucket is a contiguous key range of the
// output, in row-id order; here each bucket is sorted by one block in shared
// memory and checked.
//
// A bucket of m <= cap pairs is loaded once.  Its order is built over a
// composite key -- the compressed key followed by the pair's position in the
// bucket (which is its row-id order, the partition being stable) -- so every
// composite key is distinct and sorting by it is the stable sort:
//
//  1. the block takes the 32-bit window of the composite key that ends at its
//     highest varying bit, subtracts the bucket's smallest window value and
//     shifts right until the values fit F bits (2^F >= m, at most 8192 bins;
//     when the window's top byte takes few values, as for keys over a small
//     alphabet, the digit is instead the mixed-radix number of the dense codes
//     of the values its two top bytes take, which keeps the order and fills
//     far more bins):
//     one counting pass (shared-memory atomics; the scatter order inside a bin
//     does not matter, since the bin is then sorted by the composite key)
//     places almost every pair, the keys of a bucket spanning a narrow key
//     range;
//  2. the short bins are listed densely: 2 to 4 pairs are finished by one
//     thread (a sorting network over their window values in registers), 5 to
//     32 by eight lanes or a warp -- each lane holds one pair's window value
//     and counts the smaller ones by shuffles -- so the keys are read from
//     shared memory once, not at every comparison (equal windows, rare, are
//     ordered by the full composite keys).
//     A bin of 128 pairs or more is split again in the same way (its own
//     window, bins sized to it) by a quarter of the block, four such bins at
//     a time, or by the whole block from 1024 pairs on; the bins in between go
//     to warps, which repeat the split with 256 bins, until every range is
//     short.  The
//     minimum and the maximum of a range always land in different bins, so
//     every split shrinks the ranges it makes.
//
// Checks (a failure sends the whole sort to the plain radix path): adjacent
// composite keys ascend, the bucket's keys lie inside its splitter range,
// equal keys leave in increasing row-id order, and the hash of every output
// pair is added to a sum that must equal the input's.  Buckets of one key
// value (the splitter range [v, v + 1)) need no sorting and are only checked;
// large ones in a second kernel that spreads them over all blocks.
#include "ck_learned.cuh"

namespace ck {

constexpr int kLsThreads = 1024;
constexpr int kLsWarps = kLsThreads / 32;
constexpr int kLsBinBits = 13;
constexpr int kLsBins = 1 << kLsBinBits;            // 8192 bins in step 1
constexpr int kLsWarpBins = kLsBins / kLsWarps;      // 256 bins per warp in step 2
constexpr int kLsWarpBinBits = 8;
constexpr uint32_t kLsSmall = 4;                     // bins up to this length: sorted by one thread (narrow: insertion sort)
constexpr uint32_t kLsSeg = 8;                       // bins up to this length: rank sort by eight lanes
constexpr uint32_t kLsRank = 32;                     // bins up to this length: rank sort by one warp
constexpr uint32_t kLsBlockRange = 128;              // ranges from this length on are split by a block group:
constexpr uint32_t kLsGroupRange = 1024;             // a quarter of the block below this length, else the block
constexpr int kLsBlockStack = 128;                   // such ranges are disjoint: at most cap / 128
constexpr int kLsPerThread = 16;                     // register staging of row ids: cap <= 16 * 1024
constexpr uint32_t kLsMaxCap = kLsPerThread * kLsThreads;
constexpr int kLsList = 512;                         // pending ranges: disjoint, > 32 pairs each, so < cap / 33
constexpr uint32_t kConstInline = 16384;             // constant buckets up to this size are checked inline
constexpr uint32_t kConstChunk = 65536;              // chunk of the constant-bucket check
constexpr size_t kLsStaticSmem = 2 * kLsList * 4 + 11264;
constexpr size_t kSmemLimit = 227 * 1024;

static_assert(kLsWarpBins == (1 << kLsWarpBinBits), "warp bins");

size_t local_sort_smem(uint32_t cap, uint32_t K) {
    return (size_t)kLsBins * 4 + (size_t)K * cap * 4 + (size_t)cap * 4;
}

uint32_t local_sort_cap(uint32_t K) {
    const size_t avail = kSmemLimit - kLsStaticSmem - (size_t)kLsBins * 4;
    size_t cap = avail / (4 * (size_t)K + 4);
    cap = cap / 256 * 256;
    return (uint32_t)(cap < kLsMaxCap ? cap : kLsMaxCap);
}

// Shared-memory view of the bucket being sorted.  Composite word 0 is the
// pair's position e in the bucket; composite word w >= 1 is key word w - 1.
template <int KW>
struct LsView {
    static constexpr uint32_t K = KW, KC = KW + 1;
    uint32_t* keys;  // [K][cap]
    uint16_t* A;     // current order (positions)
    uint16_t* T;     // scratch order / digits
    uint32_t cap;
    __device__ __forceinline__ uint32_t key(uint32_t e, uint32_t w) const { return keys[w * cap + e]; }
    __device__ __forceinline__ uint32_t cw(uint32_t e, uint32_t w) const { return w == 0 ? e : key(e, w - 1); }
    // composite key of e < composite key of f
    __device__ __forceinline__ bool less(uint32_t e, uint32_t f) const {
#pragma unroll
        for (int w = KW - 1; w >= 0; --w) {
            const uint32_t x = key(e, w), y = key(f, w);
            if (x != y) return x < y;
        }
        return e < f;
    }
    __device__ __forceinline__ bool same_key(uint32_t e, uint32_t f) const {
        bool eq = true;
#pragma unroll
        for (int w = 0; w < KW; ++w) eq &= key(e, w) == key(f, w);
        return eq;
    }
};

// The 32 composite bits [base, base + 32).
struct LsWin {
    uint32_t lo, hi, sh;
    __device__ __forceinline__ LsWin(uint32_t base, uint32_t KC) {
        lo = base >> 5;
        sh = base & 31;
        hi = (sh && lo + 1 < KC) ? lo + 1 : lo;
    }
    template <class V>
    __device__ __forceinline__ uint32_t operator()(const V& v, uint32_t e) const {
        const uint32_t x = v.cw(e, lo);
        return sh ? __funnelshift_r(x, v.cw(e, hi), sh) : x;
    }
};

// Highest set bit over the composite words orw[0..KC), -1 if none.
template <uint32_t KC>
__device__ __forceinline__ int top_bit_of(const uint32_t* orw) {
    int top = -1;
#pragma unroll
    for (int w = 0; w < (int)KC; ++w)
        if (orw[w]) top = 32 * w + 31 - __clz(orw[w]);
    return top;
}

// One thread sorts A[p, p + len) (2 <= len <= 4) whose pairs share every
// composite bit above window W: the positions and window values are held in
// registers and put in order by a five-comparator network; equal window
// values (rare) are ordered by the full composite key.
template <class V>
__device__ __forceinline__ void small_sort(const V& v, const LsWin& W, uint32_t p, uint32_t len) {
    uint32_t e[4], x[4];
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
        e[i] = i < len ? v.A[p + i] : 0xFFFFu;  // 0xFFFF: padding, after every pair
        x[i] = i < len ? W(v, e[i]) : 0xFFFFFFFFu;
    }
    auto cs = [&](int a, int b) {
        const bool sw = x[b] < x[a] || (x[b] == x[a] && e[b] != 0xFFFFu && (e[a] == 0xFFFFu || v.less(e[b], e[a])));
        if (sw) {
            const uint32_t te = e[a], tx = x[a];
            e[a] = e[b];
            x[a] = x[b];
            e[b] = te;
            x[b] = tx;
        }
    };
    cs(0, 1);
    cs(2, 3);
    cs(0, 2);
    cs(1, 3);
    cs(1, 2);
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i)
        if (i < len) v.A[p + i] = (uint16_t)e[i];
}

// One warp sorts A[p, p + len) (2 <= len <= 32) whose pairs share every
// composite bit above window W: lane i ranks pair i among the others by
// window value and, where two window values are equal, by the full composite
// key (read from shared memory for those pairs only), so every pair gets its
// final slot at once.
template <class V>
__device__ __forceinline__ void warp_rank_sort(const V& v, const LsWin& W, uint32_t p, uint32_t len) {
    const uint32_t lane = threadIdx.x & 31;
    const bool in = lane < len;
    const uint32_t e = in ? v.A[p + lane] : 0u;
    const uint32_t w = in ? W(v, e) : 0xFFFFFFFFu;
    uint32_t rank = 0;
    for (uint32_t j = 0; j < len; ++j) {
        const uint32_t wj = __shfl_sync(kFull, w, j), ej = __shfl_sync(kFull, e, j);
        if (in && j != lane) rank += (wj < w || (wj == w && v.less(ej, e))) ? 1u : 0u;
    }
    __syncwarp();
    if (in) v.A[p + rank] = (uint16_t)e;
    __syncwarp();
}

// Eight lanes sort A[p, p + len) (len <= 8; len = 0: nothing) like
// warp_rank_sort, so a warp sorts four such bins at once.  Every lane of the
// warp calls this.
template <class V>
__device__ __forceinline__ void seg8_rank_sort(const V& v, const LsWin& W, uint32_t p, uint32_t len) {
    const uint32_t j = threadIdx.x & 7;
    const bool in = j < len;
    const uint32_t e = in ? v.A[p + j] : 0u;
    const uint32_t w = in ? W(v, e) : 0xFFFFFFFFu;
    uint32_t rank = 0;
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) {
        const uint32_t wi = __shfl_sync(kFull, w, i, 8), ei = __shfl_sync(kFull, e, i, 8);
        if (in && i < len && i != j) rank += (wi < w || (wi == w && v.less(ei, e))) ? 1u : 0u;
    }
    __syncwarp();
    if (in) v.A[p + rank] = (uint16_t)e;
    __syncwarp();
}

__device__ __forceinline__ void push_range(uint32_t* list, uint32_t* count, uint32_t p, uint32_t len,
                                           uint32_t* fail) {
    const uint32_t slot = atomicAdd(count, 1u);
    if (slot < (uint32_t)kLsList) list[slot] = p | (len << 16);
    else atomicAdd(fail, 1u);  // cannot happen (disjoint ranges of more than kLsRank pairs)
}

// A group of G consecutive threads of the block that splits one range: the
// whole block (G = kLsThreads, barrier 0), or a quarter of it (G = 256),
// which waits on its own named barrier 1 + gid so that four ranges are split
// side by side.
template <int G>
struct LsGroup {
    static constexpr uint32_t kThreads = G, kWarps = G / 32;
    uint32_t gid;
    __device__ __forceinline__ uint32_t tid() const { return threadIdx.x % G; }
    __device__ __forceinline__ void sync() const {
        if (G == kLsThreads) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(1u + gid), "r"(G) : "memory");
    }
};
using LsBlock = LsGroup<kLsThreads>;

// Group-wide exclusive prefix of one value per thread; *total = the sum.
template <int G = kLsThreads>
__device__ __forceinline__ uint32_t block_exclusive_sum(uint32_t x, uint32_t* wsum /*[kWarps + 1]*/,
                                                        uint32_t* total, LsGroup<G> grp = LsGroup<G>{0}) {
    constexpr uint32_t kWarps = LsGroup<G>::kWarps;
    const uint32_t lane = threadIdx.x & 31, warp = grp.tid() >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    grp.sync();
    if (warp == 0) {
        const uint32_t w = lane < kWarps ? wsum[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, wi, o);
            if (lane >= (uint32_t)o) wi += t;
        }
        if (lane < kWarps) wsum[lane] = wi - w;
        if (lane == 31) wsum[kWarps] = wi;
    }
    grp.sync();
    const uint32_t r = wsum[warp] + inc - x;
    *total = wsum[kWarps];
    grp.sync();
    return r;
}

// The c words (c = 0, 1, 2, 4 or 8) of h[0, c), h aligned to 4c bytes, by
// vector accesses; x[c ..] = 0.
__device__ __forceinline__ void load_chunk(const uint32_t* h, uint32_t c, uint32_t (&x)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = 0;
    if (c >= 4) {
        const uint4 u = reinterpret_cast<const uint4*>(h)[0];
        x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
        if (c == 8) {
            const uint4 w = reinterpret_cast<const uint4*>(h)[1];
            x[4] = w.x; x[5] = w.y; x[6] = w.z; x[7] = w.w;
        }
    } else if (c == 2) {
        const uint2 u = *reinterpret_cast<const uint2*>(h);
        x[0] = u.x; x[1] = u.y;
    } else if (c == 1) {
        x[0] = h[0];
    }
}
__device__ __forceinline__ void store_chunk(uint32_t* h, uint32_t c, const uint32_t (&x)[8]) {
    if (c >= 4) {
        reinterpret_cast<uint4*>(h)[0] = make_uint4(x[0], x[1], x[2], x[3]);
        if (c == 8) reinterpret_cast<uint4*>(h)[1] = make_uint4(x[4], x[5], x[6], x[7]);
    } else if (c == 2) {
        *reinterpret_cast<uint2*>(h) = make_uint2(x[0], x[1]);
    } else {
        h[0] = x[0];
    }
}

// Group-wide exclusive prefix of one 64-bit value per thread (several
// counters packed in bit fields); *total = the sum.  Ends without a barrier:
// the caller synchronises the group before wsum is written again.
template <int G = kLsThreads>
__device__ __forceinline__ uint64_t group_exclusive_sum64(uint64_t x, uint64_t* wsum /*[kWarps + 1]*/,
                                                          uint64_t* total, LsGroup<G> grp = LsGroup<G>{0}) {
    constexpr uint32_t kWarps = LsGroup<G>::kWarps;
    const uint32_t lane = threadIdx.x & 31, warp = grp.tid() >> 5;
    uint64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    grp.sync();
    if (warp == 0) {
        const uint64_t w = lane < kWarps ? wsum[lane] : 0ull;
        uint64_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(kFull, wi, o);
            if (lane >= (uint32_t)o) wi += t;
        }
        if (lane < kWarps) wsum[lane] = wi - w;
        if (lane == 31) wsum[kWarps] = wi;
    }
    grp.sync();
    *total = wsum[kWarps];
    return wsum[warp] + inc - x;
}

// Step 2: one warp splits range A[p0, p0 + r) (r > kLsRank) into 256 bins of
// its own window; short bins are finished at once, longer ones listed.
template <int KW>
__device__ void warp_split_range(const LsView<KW>& v, uint32_t p0, uint32_t r, uint32_t* wh, uint32_t* wpres,
                                 uint32_t* next, uint32_t* next_count, uint32_t* fail) {
    constexpr uint32_t KC = KW + 1;
    const uint32_t lane = threadIdx.x & 31, pe = p0 + r;
    const uint32_t e0 = v.A[p0];
    uint32_t orw[KC];
#pragma unroll
    for (uint32_t w = 0; w < KC; ++w) orw[w] = 0;
    for (uint32_t p = p0 + lane; p < pe; p += 32) {
        const uint32_t e = v.A[p];
#pragma unroll
        for (uint32_t w = 0; w < KC; ++w) orw[w] |= v.cw(e, w) ^ v.cw(e0, w);
    }
#pragma unroll
    for (uint32_t w = 0; w < KC; ++w) orw[w] = __reduce_or_sync(kFull, orw[w]);
    const int P = top_bit_of<KC>(orw);
    if (P < 0) {  // distinct composite keys always differ somewhere
        if (lane == 0) atomicAdd(fail, 1u);
        return;
    }
    const LsWin W((uint32_t)(P >= 31 ? P - 31 : 0), KC);
    // window range, and which values the window's top two bytes take (the
    // warp's 2 x 256-bit bitmaps, a value's bit set once)
    if (lane < 16) wpres[lane] = 0;
    __syncwarp();
    // each lane holds the positions and window values of its (at most four)
    // pairs of the range in registers for the three passes below
    static_assert(kLsBlockRange <= 4 * 32, "a warp's ranges fit four pairs per lane");
    uint32_t we[4], wx[4];
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    {
        volatile uint32_t* pr = wpres;
#pragma unroll
        for (uint32_t i = 0; i < 4; ++i) {
            const uint32_t p = p0 + lane + 32 * i;
            we[i] = p < pe ? v.A[p] : 0u;
            wx[i] = p < pe ? W(v, we[i]) : 0u;
            if (p >= pe) continue;
            const uint32_t x = wx[i];
            lo = min(lo, x);
            hi = max(hi, x);
            const uint32_t w1 = x >> 29, m1 = 1u << ((x >> 24) & 31u);
            const uint32_t w2 = 8u + ((x >> 21) & 7u), m2 = 1u << ((x >> 16) & 31u);
            if (!(pr[w1] & m1)) atomicOr(&wpres[w1], m1);
            if (!(pr[w2] & m2)) atomicOr(&wpres[w2], m2);
        }
    }
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    __syncwarp();
    // The digit: 8 bits of the window above its minimum, unless the top byte
    // is sparse (at most 64 of its values occur, as for keys over a small
    // alphabet): then the dense code of the top byte times k2 plus the dense
    // code of the second byte scaled to k2 levels (k2 = min(n2, 256 / n1)),
    // which keeps the order and fills far more of the 256 bins (used when it
    // reaches at least 128 of them).  Lane j < 16
    // holds bitmap word j and the number of set bits before it in its byte, so
    // a code is two shuffles and a popcount.
    const uint32_t wj = lane < 16 ? wpres[lane] : 0u, cj = __popc(wj);
    uint32_t incj = cj;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incj, o);
        if ((lane & 7u) >= (uint32_t)o) incj += t;
    }
    const uint32_t exj = incj - cj;
    const uint32_t n1 = __shfl_sync(kFull, incj, 7), n2 = __shfl_sync(kFull, incj, 15);
    uint32_t k2 = n1 >= 1 && n1 <= 64 ? min(n2, (uint32_t)kLsWarpBins / n1) : 1u;
    const bool dense = n1 <= 64 && n1 * k2 >= 128;  // at least half the bins reachable
    if (!dense) k2 = 1;
    const uint32_t bl = 32 - __clz(hi - lo);  // hi > lo: the window holds the top varying bit
    const uint32_t sh = bl > (uint32_t)kLsWarpBinBits ? bl - kLsWarpBinBits : 0u;
    // every lane of the warp calls this (shuffles)
    auto digit = [&](uint32_t x) -> uint32_t {
        const uint32_t b1 = x >> 24, b2 = (x >> 16) & 255u;
        const uint32_t c1 = __shfl_sync(kFull, exj, b1 >> 5) +
                            __popc(__shfl_sync(kFull, wj, b1 >> 5) & ((1u << (b1 & 31u)) - 1u));
        const uint32_t c2 = __shfl_sync(kFull, exj, 8u + (b2 >> 5)) +
                            __popc(__shfl_sync(kFull, wj, 8u + (b2 >> 5)) & ((1u << (b2 & 31u)) - 1u));
        return dense ? c1 * k2 + (k2 == n2 ? c2 : c2 * k2 / n2) : (x - lo) >> sh;
    };
    for (uint32_t i = lane; i < (uint32_t)kLsWarpBins; i += 32) wh[i] = 0;
    __syncwarp();
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {  // warp-uniform: digit() shuffles
        if (32 * i >= r) break;
        const uint32_t p = p0 + lane + 32 * i;
        wx[i] = digit(p < pe ? wx[i] : lo);
        if (p < pe) atomicAdd(&wh[wx[i]], 1u);
    }
    __syncwarp();
    {  // exclusive scan, 8 bins per lane
        uint32_t c[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            c[i] = wh[lane * 8 + i];
            sum += c[i];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, inc, o);
            if (lane >= (uint32_t)o) inc += t;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            wh[lane * 8 + i] = run;
            run += c[i];
        }
    }
    __syncwarp();
#pragma unroll
    for (uint32_t i = 0; i < 4; ++i) {
        const uint32_t p = p0 + lane + 32 * i;
        if (p < pe) v.T[p0 + atomicAdd(&wh[wx[i]], 1u)] = (uint16_t)we[i];
    }
    __syncwarp();
    for (uint32_t p = p0 + lane; p < pe; p += 32) v.A[p] = v.T[p];
    __syncwarp();
    // wh[d] is now the end of bin d: each lane reads its 8 bins and lists
    // the long ones; the short ones go into two dense lists in wh (2 .. 4
    // pairs from the front, 5 .. 32 from the back)
    uint32_t st[8], sz[8], nsmall = 0, nrank = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t d = lane * 8 + i;
        st[i] = d ? wh[d - 1] : 0u;
        sz[i] = wh[d] - st[i];
        if (sz[i] > kLsRank) push_range(next, next_count, p0 + st[i], sz[i], fail);
        nsmall += (sz[i] >= 2 && sz[i] <= kLsSmall) ? 1u : 0u;
        nrank += (sz[i] > kLsSmall && sz[i] <= kLsRank) ? 1u : 0u;
    }
    uint32_t inc_s = nsmall, inc_r = nrank;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, inc_s, o), u = __shfl_up_sync(kFull, inc_r, o);
        if (lane >= (uint32_t)o) {
            inc_s += t;
            inc_r += u;
        }
    }
    const uint32_t tot_s = __shfl_sync(kFull, inc_s, 31), tot_r = __shfl_sync(kFull, inc_r, 31);
    __syncwarp();
    uint32_t as = inc_s - nsmall, ar = inc_r - nrank;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (sz[i] >= 2 && sz[i] <= kLsSmall) wh[as++] = (p0 + st[i]) | (sz[i] << 16);
        else if (sz[i] > kLsSmall && sz[i] <= kLsRank) wh[kLsWarpBins - 1 - ar++] = (p0 + st[i]) | (sz[i] << 16);
    }
    __syncwarp();
    for (uint32_t k = lane; k < tot_s; k += 32) small_sort(v, W, wh[k] & 0xFFFFu, wh[k] >> 16);
    __syncwarp();
    for (uint32_t k = 0; k < tot_r; ++k) {
        const uint32_t r = wh[kLsWarpBins - 1 - k];
        warp_rank_sort(v, W, r & 0xFFFFu, r >> 16);
    }
}

// Key of element e against splitter s (entry-major, K words): -1, 0, 1.
template <int KW>
__device__ __forceinline__ int cmp_key_spl(const LsView<KW>& v, uint32_t e, const uint32_t* s) {
#pragma unroll
    for (int w = KW - 1; w >= 0; --w) {
        const uint32_t x = v.key(e, w);
        if (x != s[w]) return x < s[w] ? -1 : 1;
    }
    return 0;
}

// Bucket b holds only one key value when its range is [v, v + 1).
__device__ __forceinline__ bool constant_range(const uint32_t* spl, uint32_t K, uint32_t nb, uint32_t b) {
    if (b == 0 || b + 1 >= nb) return false;
    const uint32_t* lo = spl + (size_t)(b - 1) * K;
    const uint32_t* hi = spl + (size_t)b * K;
    uint32_t carry = 1;
    for (uint32_t w = 0; w < K; ++w) {
        const uint64_t sum = (uint64_t)lo[w] + carry;
        if ((uint32_t)sum != hi[w]) return false;
        carry = (uint32_t)(sum >> 32);
    }
    return carry == 0;
}

// Checks positions [i0, i1) of constant bucket b (whose pairs start at s0):
// every key equals the splitter value v = spl[b - 1], row ids ascend.  Adds
// the pair hashes.  Block-strided over threads tid, step `step`.
__device__ __forceinline__ void check_constant(const LocalSortArgs& a, uint32_t b, uint64_t s0, uint64_t i0,
                                               uint64_t i1, uint32_t tid, uint32_t step, uint64_t* hash,
                                               uint32_t* bad) {
    const uint32_t* vkey = a.spl + (size_t)(b - 1) * a.K;
    for (uint64_t i = i0 + tid; i < i1; i += step) {
        const uint32_t r = a.rid[i];
        uint64_t h = pair_hash_start(r);
        bool ok = true;
        for (uint32_t w = 0; w < a.K; ++w) {
            const uint32_t x = a.ck[(uint64_t)w * a.ld + i];
            ok &= x == vkey[w];
            h = pair_hash_word(h, x);
        }
        if (i > s0 && a.rid[i - 1] >= r) ok = false;
        *hash += pair_hash_end(h);
        *bad += ok ? 0u : 1u;
    }
}

// Exclusive scan in place of hist[0, bins) (bins a power of two, 256 ..
// kLsBins) by the block; warp w scans the w-th 32nd of the bins with its
// lanes on consecutive bins (no bank conflicts), then the warps' totals are
// scanned and added.
template <int G = kLsThreads>
__device__ __forceinline__ void bins_exclusive_scan(uint32_t* hist, uint32_t bins, uint32_t* wsum,
                                                    LsGroup<G> grp = LsGroup<G>{0}) {
    constexpr uint32_t kWarps = LsGroup<G>::kWarps;
    const uint32_t lane = threadIdx.x & 31, warp = grp.tid() >> 5;
    const uint32_t seg = bins / kWarps, c0 = warp * seg;
    uint32_t run = 0;
    for (uint32_t k = 0; k < seg; k += 32) {
        const bool in = k + lane < seg;
        const uint32_t x = in ? hist[c0 + k + lane] : 0u;
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, inc, o);
            if (lane >= (uint32_t)o) inc += t;
        }
        if (in) hist[c0 + k + lane] = run + inc - x;
        run += __shfl_sync(kFull, inc, 31);
    }
    if (lane == 0) wsum[warp] = run;
    grp.sync();
    if (warp == 0) {
        const uint32_t x = lane < kWarps ? wsum[lane] : 0u;
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, inc, o);
            if (lane >= (uint32_t)o) inc += t;
        }
        if (lane < kWarps) wsum[lane] = inc - x;
    }
    grp.sync();
    const uint32_t add = wsum[warp];
    for (uint32_t k = lane; k < seg; k += 32) hist[c0 + k] += add;
    grp.sync();
}

// Shared state of the block-level splits.
struct LsBlockState {
    uint32_t* list;    // warp list (ranges of kLsRank + 1 .. kLsBlockRange - 1 pairs)
    uint32_t* count;
    uint32_t* stack;   // block stack (ranges of kLsBlockRange pairs or more)
    uint32_t* scount;
    uint32_t* orw;     // [KC]
    uint32_t* mm;      // [2]: window minimum, maximum
    uint32_t* wsum;    // [kLsWarps + 1]
    uint64_t* wsum64;  // [kLsWarps + 1]
    uint16_t* bytes;   // [3][256]: dense codes (digit terms, < kLsBins) of the window's top three bytes
    uint32_t* pres;    // [3][8]: which values each of those bytes takes (bitmaps)
    uint32_t* nbytes;  // [3]: values in use of each byte
};

// Step 1 on range A[p0, p0 + r) by a group of G threads (the whole block,
// or a quarter of it for ranges short enough for its quarter of the bins,
// hist[0, 2^(F+1))).  ident (whole block only): the range is the whole bucket
// in load order (A not yet written; element = position), and st.orw already
// holds the OR of every key word's difference to element p0.  Ends with every
// bin of the range listed or finished, and a barrier of the group.
template <int KW, int G = kLsThreads>
__device__ void block_split(const LsView<KW>& v, uint32_t p0, uint32_t r, bool ident, uint32_t* hist,
                            const LsBlockState& st, uint32_t* bad, LsGroup<G> grp = LsGroup<G>{0}) {
    constexpr uint32_t KC = KW + 1;
    constexpr uint32_t kWarps = LsGroup<G>::kWarps;
    const uint32_t tid = grp.tid(), lane = tid & 31;
    const uint32_t pe = p0 + r;
    // a quarter of the block holds its range's positions, then window values,
    // then digits in registers (its ranges are shorter than 4 G)
    constexpr bool kQuarter = G < kLsThreads;
    constexpr uint32_t kQItems = 4;
    static_assert(kLsGroupRange <= kQItems * (kLsThreads / 4), "quarter ranges fit the registers");
    uint32_t qe[kQItems], qx[kQItems];
    if (!ident) {  // OR of every composite word's difference to the range's first element
        if (tid < KC) st.orw[tid] = 0;
        grp.sync();
        const uint32_t e0 = v.A[p0];
        uint32_t o[KC];
#pragma unroll
        for (uint32_t w = 0; w < KC; ++w) o[w] = 0;
        for (uint32_t p = p0 + tid; p < pe; p += G) {
            const uint32_t e = v.A[p];
#pragma unroll
            for (uint32_t w = 0; w < KC; ++w) o[w] |= v.cw(e, w) ^ v.cw(e0, w);
        }
#pragma unroll
        for (uint32_t w = 0; w < KC; ++w) {
            const uint32_t x = __reduce_or_sync(kFull, o[w]);
            if (lane == 0 && x) atomicOr(&st.orw[w], x);
        }
        grp.sync();
    }
    const int P = top_bit_of<KC>(st.orw);
    if (P < 0) {  // one key in a bucket of equal keys (ident): already in order
        for (uint32_t p = p0 + tid; p < pe; p += G) v.A[p] = (uint16_t)p;
        grp.sync();
        return;
    }
    const LsWin W((uint32_t)(P >= 31 ? P - 31 : 0), KC);
    uint32_t F = 32 - __clz(r - 1);  // 2^F >= r
    F = F < 8 ? 8u : (F > (uint32_t)kLsBinBits ? (uint32_t)kLsBinBits : F);
    // bins of the digit: the power of two at or above the range's length
    // (the scan and the bin lists cost in proportion to the bins, more than
    // the extra short bins that fewer bins leave cost to sort)
    const uint32_t dbins = 1u << F;
    for (uint32_t d = tid; d < dbins; d += G) hist[d] = 0;
    if (tid < 24) st.pres[tid] = 0;
    if (tid == 0) {
        st.mm[0] = 0xFFFFFFFFu;
        st.mm[1] = 0;
    }
    grp.sync();  // mm initialised, bins and byte bitmaps zeroed
    {  // window range, and which values the window's top three bytes take: a
       // value's bit is set once (a plain read first), so keys over a small
       // alphabet, whose bytes take few values, do not queue on a few words
        uint32_t lo = 0xFFFFFFFFu, hi = 0;
        volatile uint32_t* pr = st.pres;
        auto visit = [&](uint32_t x) {
            lo = min(lo, x);
            hi = max(hi, x);
            const uint32_t w1 = x >> 29, m1 = 1u << ((x >> 24) & 31u);
            const uint32_t w2 = 8u + ((x >> 21) & 7u), m2 = 1u << ((x >> 16) & 31u);
            const uint32_t w3 = 16u + ((x >> 13) & 7u), m3 = 1u << ((x >> 8) & 31u);
            if (!(pr[w1] & m1)) atomicOr(&st.pres[w1], m1);
            if (!(pr[w2] & m2)) atomicOr(&st.pres[w2], m2);
            if (!(pr[w3] & m3)) atomicOr(&st.pres[w3], m3);
        };
        if constexpr (kQuarter) {
#pragma unroll
            for (uint32_t i = 0; i < kQItems; ++i) {
                const uint32_t p = p0 + tid + i * G;
                if (p < pe) {
                    qe[i] = v.A[p];
                    qx[i] = W(v, qe[i]);
                    visit(qx[i]);
                }
            }
        } else {
            for (uint32_t p = p0 + tid; p < pe; p += G) visit(W(v, ident ? p : v.A[p]));
        }
        lo = __reduce_min_sync(kFull, lo);
        hi = __reduce_max_sync(kFull, hi);
        if (lane == 0) {
            atomicMin(&st.mm[0], lo);
            atomicMax(&st.mm[1], hi);
        }
    }
    grp.sync();
    if (tid < 96) {  // dense codes of the values each byte takes (warp j: byte j; lane l: values 8l .. 8l + 7)
        const uint32_t j = tid >> 5;
        const uint32_t bits = (st.pres[8 * j + (lane >> 2)] >> (8 * (lane & 3u))) & 255u;
        const uint32_t c = __popc(bits);
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, inc, o);
            if (lane >= (uint32_t)o) inc += t;
        }
        const uint32_t run = inc - c;
#pragma unroll
        for (uint32_t i = 0; i < 8; ++i)
            st.bytes[256 * j + 8 * lane + i] = (uint16_t)(run + __popc(bits & ((1u << i) - 1u)));
        if (lane == 31) st.nbytes[j] = inc;
    }
    grp.sync();
    // The digit: the window's top bits after subtracting its minimum (2^F
    // bins), unless the top byte is sparse (at most 128 of its values occur,
    // as for keys over a small alphabet whose codes use few bit patterns):
    // then the mixed-radix number of the dense codes of the window's top
    // bytes -- all values of the first, of the second as far as the bins
    // allows (scaled down to k2 levels otherwise), of the third within what is
    // left (k3 levels) -- which keeps the order of the windows and spreads the
    // pairs over far more of the bins, if that gives 256 bins or more.
    const uint32_t n1 = st.nbytes[0], n2 = st.nbytes[1], n3 = st.nbytes[2];
    uint32_t k2 = 1, k3 = 1;
    bool dense = false;
    if (n1 <= 128) {
        k2 = min(n2, dbins / n1);
        k3 = k2 == n2 ? min(n3, dbins / (n1 * n2)) : 1u;
        dense = n1 * k2 * k3 >= 256;
    }
    uint32_t bins = 1u << F;
    if (dense) {
        bins = (n1 * k2 * k3 + 31) & ~31u;  // whole segments of the bin scan; the extra bins stay empty
        // codes -> digit terms: c1 k2 k3, scaled c2 times k3, scaled c3
        for (uint32_t i = tid; i < 768; i += G) {
            const uint32_t j = i >> 8, c = st.bytes[i];
            st.bytes[i] = (uint16_t)(j == 0 ? c * k2 * k3
                                            : (j == 1 ? (k2 == n2 ? c : c * k2 / n2) * k3 : (k3 == n3 ? c : c * k3 / n3)));
        }
        grp.sync();
    }
    const uint32_t wmin = st.mm[0];
    const uint32_t bl = 32 - __clz(st.mm[1] - wmin);
    const uint32_t sh = bl > F ? bl - F : 0u;
    const uint16_t* c1 = st.bytes;
    const uint16_t* c2 = st.bytes + 256;
    const uint16_t* c3 = st.bytes + 512;
    auto digit = [&](uint32_t x) -> uint32_t {
        return dense ? c1[x >> 24] + c2[(x >> 16) & 255u] + c3[(x >> 8) & 255u] : (x - wmin) >> sh;
    };
    if (ident) {  // the digits wait in T for the scatter (T is free until then)
        for (uint32_t p = tid; p < r; p += G) {
            const uint32_t d = digit(W(v, p));
            v.T[p] = (uint16_t)d;
            atomicAdd(&hist[d], 1u);
        }
    } else {
        if constexpr (kQuarter) {
#pragma unroll
            for (uint32_t i = 0; i < kQItems; ++i)
                if (p0 + tid + i * G < pe) {
                    qx[i] = digit(qx[i]);
                    atomicAdd(&hist[qx[i]], 1u);
                }
        } else {
            for (uint32_t p = p0 + tid; p < pe; p += G) atomicAdd(&hist[digit(W(v, v.A[p]))], 1u);
        }
    }
    grp.sync();
    // One pass over the bins, each thread on a chunk of c consecutive ones
    // (bins is a multiple of 32, so every chunk is whole): the bins' starts
    // and how many short bins of each kind come before the chunk, in one
    // group scan of three packed counters.  hist[d] becomes start | size << 16
    // (both < 2^15 <= cap), so the scatter's increments leave the size intact.
    const uint32_t c = bins <= G ? 1u : (bins <= 2 * G ? 2u : (bins <= 4 * G ? 4u : 8u));
    const uint32_t d0 = tid * c;
    const bool mine = d0 < bins;
    uint32_t as, a8, ar, ns_tot, n8_tot, nr_tot;
    {
        uint32_t cnt[8];
        uint32_t tot = 0, ns = 0, n8 = 0, nr = 0;
        load_chunk(hist + d0, mine ? c : 0u, cnt);
#pragma unroll
        for (uint32_t i = 0; i < 8; ++i) {
            tot += cnt[i];
            ns += (cnt[i] >= 2 && cnt[i] <= kLsSmall) ? 1u : 0u;
            n8 += (cnt[i] > kLsSmall && cnt[i] <= kLsSeg) ? 1u : 0u;
            nr += (cnt[i] > kLsSeg && cnt[i] <= kLsRank) ? 1u : 0u;
        }
        // four 16-bit fields: every count and sum is at most r <= cap < 2^16
        uint64_t all;
        const uint64_t ex = group_exclusive_sum64<G>(
            (uint64_t)tot | (uint64_t)ns << 16 | (uint64_t)n8 << 32 | (uint64_t)nr << 48, st.wsum64, &all, grp);
        uint32_t start = (uint32_t)ex & 0xFFFFu;
        as = (uint32_t)(ex >> 16) & 0xFFFFu;
        a8 = (uint32_t)(ex >> 32) & 0xFFFFu;
        ar = (uint32_t)(ex >> 48);
        ns_tot = (uint32_t)(all >> 16) & 0xFFFFu;
        n8_tot = (uint32_t)(all >> 32) & 0xFFFFu;
        nr_tot = (uint32_t)(all >> 48);
        if (mine) {
            uint32_t o[8];
#pragma unroll
            for (uint32_t i = 0; i < 8; ++i) {
                o[i] = start | cnt[i] << 16;
                start += cnt[i];
            }
            store_chunk(hist + d0, c, o);
        }
    }
    grp.sync();
    if (ident) {
        for (uint32_t p = tid; p < r; p += G) v.A[atomicAdd(&hist[v.T[p]], 1u) & 0xFFFFu] = (uint16_t)p;
    } else {
        if constexpr (kQuarter) {
#pragma unroll
            for (uint32_t i = 0; i < kQItems; ++i)
                if (p0 + tid + i * G < pe) v.T[p0 + (atomicAdd(&hist[qx[i]], 1u) & 0xFFFFu)] = (uint16_t)qe[i];
        } else {
            for (uint32_t p = p0 + tid; p < pe; p += G) {
                const uint32_t e = v.A[p];
                v.T[p0 + (atomicAdd(&hist[digit(W(v, e))], 1u) & 0xFFFFu)] = (uint16_t)e;
            }
        }
        grp.sync();
        for (uint32_t p = p0 + tid; p < pe; p += G) v.A[p] = v.T[p];
    }
    grp.sync();
    // hist[d] is now (end of bin d) | size << 16 (relative to p0).  Long bins
    // are listed for the block or the warps; the short ones densely in
    // T[p0 ..] as (start, length) pairs: 2 .. 4 pairs from the front (one
    // thread each), then 9 .. 32 (one warp each), and 5 .. 8 from the back
    // (eight lanes each).  A listed bin has two pairs or more, so the lists
    // fit the range's r entries of T.
    uint32_t hc[8];
    load_chunk(hist + d0, mine ? c : 0u, hc);
#pragma unroll
    for (uint32_t i = 0; i < 8; ++i) {
        if (!mine || i >= c) break;
        const uint32_t h = hc[i], sz = h >> 16, b0 = (h & 0xFFFFu) - sz;
        if (sz >= kLsBlockRange) {
            const uint32_t slot = atomicAdd(st.scount, 1u);
            if (slot < (uint32_t)kLsBlockStack) st.stack[slot] = (p0 + b0) | (sz << 16);
            else atomicAdd(bad, 1u);  // cannot happen (disjoint ranges of kLsBlockRange pairs or more)
        } else if (sz > kLsRank) {
            push_range(st.list, st.count, p0 + b0, sz, bad);
        } else if (sz >= 2 && sz <= kLsSmall) {
            v.T[p0 + 2 * as] = (uint16_t)(p0 + b0);
            v.T[p0 + 2 * as + 1] = (uint16_t)sz;
            ++as;
        } else if (sz > kLsSeg) {
            v.T[p0 + 2 * (ns_tot + ar)] = (uint16_t)(p0 + b0);
            v.T[p0 + 2 * (ns_tot + ar) + 1] = (uint16_t)sz;
            ++ar;
        } else if (sz > kLsSmall) {
            v.T[pe - 2 - 2 * a8] = (uint16_t)(p0 + b0);
            v.T[pe - 1 - 2 * a8] = (uint16_t)sz;
            ++a8;
        }
    }
    grp.sync();
    // the first threads take the odd small bins, the last warps the odd
    // longer ones
    const uint32_t rw = kWarps - 1 - (tid >> 5);
    for (uint32_t k = tid; k < ns_tot; k += G) small_sort(v, W, v.T[p0 + 2 * k], v.T[p0 + 2 * k + 1]);
    for (uint32_t k0 = 4 * rw; k0 < n8_tot; k0 += 4 * kWarps) {  // uniform in the warp
        const uint32_t k = k0 + (lane >> 3);
        seg8_rank_sort(v, W, k < n8_tot ? v.T[pe - 2 - 2 * k] : 0u, k < n8_tot ? v.T[pe - 1 - 2 * k] : 0u);
    }
    for (uint32_t k = rw; k < nr_tot; k += kWarps)
        warp_rank_sort(v, W, v.T[p0 + 2 * (ns_tot + k)], v.T[p0 + 2 * (ns_tot + k) + 1]);
    grp.sync();
}


// ---------------------------------------------------------------- narrow buckets
// A bucket whose splitter range [lo, hi] spans less than 2^32 keys (both
// splitters known, hi - lo < 2^32) is sorted by r = key - lo alone, a 32-bit
// value (the low word of the difference: the higher ones are zero), in pairs
// (r, position); the keys are rebuilt as lo + r when the bucket is written
// back.  The pairs sit in RS (r, by position) and A (position); R and T are
// scratch.  Sort key of slot p: (RS[p] << 16) | A[p], distinct.
struct LnView {
    uint32_t* RS;  // [cap] r by slot
    uint32_t* R;   // [cap] scratch (r by element at load)
    uint16_t* A;   // [cap]
    uint16_t* T;   // [cap] scratch
    __device__ __forceinline__ uint64_t k(uint32_t p) const { return ((uint64_t)RS[p] << 16) | A[p]; }
};

// Stable insertion sort of slots [p, p + len) (one thread).
__device__ __forceinline__ void ln_insertion_sort(const LnView& v, uint32_t p, uint32_t len) {
    for (uint32_t j = p + 1; j < p + len; ++j) {
        const uint32_t r = v.RS[j];
        const uint16_t x = v.A[j];
        const uint64_t kx = ((uint64_t)r << 16) | x;
        uint32_t i = j;
        while (i > p && v.k(i - 1) > kx) {
            v.RS[i] = v.RS[i - 1];
            v.A[i] = v.A[i - 1];
            --i;
        }
        v.RS[i] = r;
        v.A[i] = x;
    }
}

// One warp sorts slots [p, p + len) (len <= 32) by rank.
__device__ __forceinline__ void ln_rank_sort(const LnView& v, uint32_t p, uint32_t len) {
    const uint32_t lane = threadIdx.x & 31;
    const bool in = lane < len;
    const uint64_t kx = in ? v.k(p + lane) : ~0ull;
    uint32_t rank = 0;
    for (uint32_t j = 0; j < len; ++j) rank += __shfl_sync(kFull, kx, j) < kx ? 1u : 0u;
    __syncwarp();
    if (in) {
        v.RS[p + rank] = (uint32_t)(kx >> 16);
        v.A[p + rank] = (uint16_t)kx;
    }
    __syncwarp();
}

// Digit of slot p's key in a split of a range whose key window starts at bit
// `base` of the 48-bit key: ((window - lo) >> sh).
__device__ __forceinline__ uint32_t ln_window(const LnView& v, uint32_t p, uint32_t base) {
    return (uint32_t)(v.k(p) >> base);
}

// One warp splits slots [p0, p0 + r) (r > kLsRank) into 256 bins of its window.
__device__ void ln_warp_split(const LnView& v, uint32_t p0, uint32_t r, uint32_t* wh, uint32_t* next,
                              uint32_t* next_count, uint32_t* fail) {
    const uint32_t lane = threadIdx.x & 31, pe = p0 + r;
    const uint64_t k0 = v.k(p0);
    uint64_t o = 0;
    for (uint32_t p = p0 + lane; p < pe; p += 32) o |= v.k(p) ^ k0;
    o = (uint64_t)__reduce_or_sync(kFull, (uint32_t)o) | ((uint64_t)__reduce_or_sync(kFull, (uint32_t)(o >> 32)) << 32);
    if (o == 0) {  // distinct keys always differ somewhere
        if (lane == 0) atomicAdd(fail, 1u);
        return;
    }
    const uint32_t P = 63 - __clzll(o), base = P >= 31 ? P - 31 : 0u;
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    for (uint32_t p = p0 + lane; p < pe; p += 32) {
        const uint32_t x = ln_window(v, p, base);
        lo = min(lo, x);
        hi = max(hi, x);
    }
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    const uint32_t bl = 32 - __clz(hi - lo);
    const uint32_t sh = bl > (uint32_t)kLsWarpBinBits ? bl - kLsWarpBinBits : 0u;
    for (uint32_t i = lane; i < (uint32_t)kLsWarpBins; i += 32) wh[i] = 0;
    __syncwarp();
    for (uint32_t p = p0 + lane; p < pe; p += 32) atomicAdd(&wh[(ln_window(v, p, base) - lo) >> sh], 1u);
    __syncwarp();
    {
        uint32_t c[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            c[i] = wh[lane * 8 + i];
            sum += c[i];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int q = 1; q < 32; q <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, inc, q);
            if (lane >= (uint32_t)q) inc += t;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            wh[lane * 8 + i] = run;
            run += c[i];
        }
    }
    __syncwarp();
    for (uint32_t p = p0 + lane; p < pe; p += 32) {
        const uint32_t q = p0 + atomicAdd(&wh[(ln_window(v, p, base) - lo) >> sh], 1u);
        v.R[q] = v.RS[p];
        v.T[q] = v.A[p];
    }
    __syncwarp();
    for (uint32_t p = p0 + lane; p < pe; p += 32) {
        v.RS[p] = v.R[p];
        v.A[p] = v.T[p];
    }
    __syncwarp();
    uint32_t st[8], sz[8], nsmall = 0, nrank = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t d = lane * 8 + i;
        st[i] = d ? wh[d - 1] : 0u;
        sz[i] = wh[d] - st[i];
        if (sz[i] > kLsRank) push_range(next, next_count, p0 + st[i], sz[i], fail);
        nsmall += (sz[i] >= 2 && sz[i] <= kLsSmall) ? 1u : 0u;
        nrank += (sz[i] > kLsSmall && sz[i] <= kLsRank) ? 1u : 0u;
    }
    uint32_t inc_s = nsmall, inc_r = nrank;
#pragma unroll
    for (int q = 1; q < 32; q <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, inc_s, q), u = __shfl_up_sync(kFull, inc_r, q);
        if (lane >= (uint32_t)q) {
            inc_s += t;
            inc_r += u;
        }
    }
    const uint32_t tot_s = __shfl_sync(kFull, inc_s, 31), tot_r = __shfl_sync(kFull, inc_r, 31);
    __syncwarp();
    uint32_t as = inc_s - nsmall, ar = inc_r - nrank;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (sz[i] >= 2 && sz[i] <= kLsSmall) wh[as++] = (p0 + st[i]) | (sz[i] << 16);
        else if (sz[i] > kLsSmall && sz[i] <= kLsRank) wh[kLsWarpBins - 1 - ar++] = (p0 + st[i]) | (sz[i] << 16);
    }
    __syncwarp();
    for (uint32_t q = lane; q < tot_s; q += 32) ln_insertion_sort(v, wh[q] & 0xFFFFu, wh[q] >> 16);
    __syncwarp();
    for (uint32_t q = 0; q < tot_r; ++q) {
        const uint32_t e = wh[kLsWarpBins - 1 - q];
        ln_rank_sort(v, e & 0xFFFFu, e >> 16);
    }
}

// The whole block lists the bins [0, bins) of a split whose slots start at p0
// (hist[d] = end of bin d relative to p0, the range ends at pe) and finishes
// the short ones: 2 .. 4 slots by one thread, 5 .. 32 by one warp; longer bins
// go to the warp list (the narrow path splits every long bin by warps).
__device__ void ln_finish_bins(const LnView& v, const uint32_t* hist, uint32_t bins, uint32_t p0, uint32_t pe,
                               const LsBlockState& st, uint32_t* bad) {
    const uint32_t tid = threadIdx.x;
    uint32_t nsmall = 0, nrank = 0;
    for (uint32_t d = tid; d < bins; d += kLsThreads) {
        const uint32_t b0 = d ? hist[d - 1] : 0u, sz = hist[d] - b0;
        if (sz > kLsRank) push_range(st.list, st.count, p0 + b0, sz, bad);
        nsmall += (sz >= 2 && sz <= kLsSmall) ? 1u : 0u;
        nrank += (sz > kLsSmall && sz <= kLsRank) ? 1u : 0u;
    }
    uint32_t ns_tot, nr_tot;
    uint32_t as = block_exclusive_sum(nsmall, st.wsum, &ns_tot);
    uint32_t ar = block_exclusive_sum(nrank, st.wsum, &nr_tot);
    for (uint32_t d = tid; d < bins; d += kLsThreads) {
        const uint32_t b0 = d ? hist[d - 1] : 0u, sz = hist[d] - b0;
        if (sz >= 2 && sz <= kLsSmall) {
            v.T[p0 + 2 * as] = (uint16_t)(p0 + b0);
            v.T[p0 + 2 * as + 1] = (uint16_t)sz;
            ++as;
        } else if (sz > kLsSmall && sz <= kLsRank) {
            v.T[pe - 2 - 2 * ar] = (uint16_t)(p0 + b0);
            v.T[pe - 1 - 2 * ar] = (uint16_t)sz;
            ++ar;
        }
    }
    __syncthreads();
    for (uint32_t q = tid; q < ns_tot; q += kLsThreads) ln_insertion_sort(v, v.T[p0 + 2 * q], v.T[p0 + 2 * q + 1]);
    for (uint32_t q = tid >> 5; q < nr_tot; q += kLsWarps) ln_rank_sort(v, v.T[pe - 2 - 2 * q], v.T[pe - 1 - 2 * q]);
    __syncthreads();
}

// Is bucket b narrow (0 < b < nb - 1 and spl[b] - spl[b - 1] <= 2^32)?
// *D = spl[b] - spl[b - 1] - 1, the largest r.
__device__ __forceinline__ bool narrow_range(const uint32_t* spl, uint32_t K, uint32_t nb, uint32_t b, uint32_t* D) {
    if (b == 0 || b + 1 >= nb || K < 2) return false;
    const uint32_t* lo = spl + (size_t)(b - 1) * K;
    const uint32_t* hi = spl + (size_t)b * K;
    uint32_t borrow = 0, w0 = 0, w1 = 0;
    bool upper_zero = true;
    for (uint32_t w = 0; w < K; ++w) {
        const uint64_t d = (uint64_t)hi[w] - lo[w] - borrow;
        borrow = (uint32_t)(d >> 63);
        if (w == 0) w0 = (uint32_t)d;
        else if (w == 1) w1 = (uint32_t)d;
        else upper_zero &= (uint32_t)d == 0u;
    }
    if (!upper_zero || !(w1 == 0 || (w1 == 1 && w0 == 0))) return false;
    *D = w0 - 1u;  // hi - lo >= 1 (strictly increasing splitters); 2^32 gives 0xFFFFFFFF
    return true;
}

// Sorts narrow bucket b (m pairs at s0, 2 <= m <= cap) and writes it back,
// checking every key's range (lo <= key <= hi), the order of the output and
// the row-id order of equal keys, and adding the pair hashes.
template <int KW>
__device__ void sort_narrow_bucket(const LocalSortArgs& a, const LnView& v, uint32_t b, uint64_t s0, uint32_t m,
                                   uint32_t D, uint32_t* hist, const LsBlockState& st, uint32_t* list2,
                                   uint32_t* count2, uint32_t* grab, uint32_t* sbad, uint64_t* hash, uint32_t* bad) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t* lo = a.spl + (size_t)(b - 1) * KW;
    uint32_t lw[KW];
#pragma unroll
    for (int w = 0; w < KW; ++w) lw[w] = lo[w];
    uint32_t F = 33 - __clz(m - 1);  // about two bins per pair
    F = F < 8 ? 8u : (F > (uint32_t)kLsBinBits ? (uint32_t)kLsBinBits : F);
    const uint32_t bins = 1u << F;
    const uint32_t bl = 32 - __clz(D);
    const uint32_t sh = bl > F ? bl - F : 0u;
    for (uint32_t d = tid; d < bins; d += kLsThreads) hist[d] = 0;
    if (tid == 0) {
        st.count[0] = 0;
        *count2 = 0;
    }
    __syncthreads();
    // load: r = key - lo (its upper words must be zero and r <= D), count digits
    for (uint32_t t0 = tid; t0 < m; t0 += 4 * kLsThreads) {
        uint32_t x[4][KW];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t t = t0 + u * kLsThreads;
#pragma unroll
            for (int w = 0; w < KW; ++w) x[u][w] = t < m ? a.ck[(uint64_t)w * a.ld + s0 + t] : lw[w];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t t = t0 + u * kLsThreads;
            if (t >= m) continue;
            uint32_t borrow = 0, r = 0;
            bool ok = true;
#pragma unroll
            for (int w = 0; w < KW; ++w) {
                const uint64_t d = (uint64_t)x[u][w] - lw[w] - borrow;
                borrow = (uint32_t)(d >> 63);
                if (w == 0) r = (uint32_t)d;
                else ok &= (uint32_t)d == 0u;
            }
            ok &= borrow == 0 && r <= D;
            *bad += ok ? 0u : 1u;
            if (!ok) r = D;  // keeps the bin index in range; the bucket already fails its check
            v.R[t] = r;
            atomicAdd(&hist[r >> sh], 1u);
        }
    }
    __syncthreads();
    bins_exclusive_scan(hist, bins, st.wsum);
    for (uint32_t t = tid; t < m; t += kLsThreads) {
        const uint32_t r = v.R[t];
        const uint32_t q = atomicAdd(&hist[r >> sh], 1u);
        v.RS[q] = r;
        v.A[q] = (uint16_t)t;
    }
    __syncthreads();
    ln_finish_bins(v, hist, bins, 0, m, st, sbad);
    {
        bool cur = false;  // false: st.list is current, true: list2
        for (;;) {  // rounds of warp splits of the long bins
            uint32_t* cl = cur ? list2 : st.list;
            uint32_t* cc = cur ? count2 : st.count;
            uint32_t* nl = cur ? st.list : list2;
            uint32_t* nc = cur ? st.count : count2;
            const uint32_t nr = min(*cc, (uint32_t)kLsList);
            if (nr == 0) break;
            __syncthreads();
            if (tid == 0) {
                *nc = 0;
                *grab = 0;
            }
            __syncthreads();
            for (;;) {
                uint32_t e = 0;
                if (lane == 0) e = atomicAdd(grab, 1u);
                e = __shfl_sync(kFull, e, 0);
                if (e >= nr) break;
                const uint32_t r = cl[e];
                ln_warp_split(v, r & 0xFFFFu, r >> 16, hist + warp * kLsWarpBins, nl, nc, sbad);
            }
            __syncthreads();
            cur = !cur;
        }
    }
    __syncthreads();
    // write back: keys lo + r, row ids gathered into registers first (in place)
    uint32_t rr[kLsPerThread];
    const uint32_t jmax = (m + kLsThreads - 1) / kLsThreads;
#pragma unroll
    for (int j = 0; j < kLsPerThread; ++j) {
        const uint32_t t = tid + (uint32_t)j * kLsThreads;
        rr[j] = (uint32_t)j < jmax && t < m ? a.rid[s0 + v.A[t]] : 0u;
    }
    if (a.inject & CK_LEARNED_INJECT_RID_SWAP) {  // test only: exchange the row ids of positions 0 and 1
        const uint32_t other = __shfl_xor_sync(kFull, rr[0], 1);
        if (warp == 0 && lane < 2) rr[0] = other;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kLsPerThread; ++j) {
        const uint32_t t = tid + (uint32_t)j * kLsThreads;
        const bool in = (uint32_t)j < jmax && t < m;
        const uint32_t r = in ? v.RS[t] : 0u;
        // order: slots ascend; equal keys keep row-id order (the neighbour
        // slot t - 1 is the previous lane, except for lane 0)
        const uint32_t r_prev = __shfl_up_sync(kFull, r, 1), rid_prev = __shfl_up_sync(kFull, rr[j], 1);
        if (in) {
            uint32_t carry = r;
            uint64_t h = pair_hash_start(rr[j]);
#pragma unroll
            for (int w = 0; w < KW; ++w) {
                const uint64_t sum = (uint64_t)lw[w] + carry;
                const uint32_t word = (uint32_t)sum;
                carry = (uint32_t)(sum >> 32);
                a.ck[(uint64_t)w * a.ld + s0 + t] = word;
                h = pair_hash_word(h, word);
            }
            *hash += pair_hash_end(h);
            a.rid[s0 + t] = rr[j];
            if (t > 0) {
                if (v.k(t - 1) >= v.k(t)) ++*bad;
                if (lane > 0 && r_prev == r && rid_prev >= rr[j]) ++*bad;
            }
        }
    }
    __syncthreads();
    for (uint32_t t = tid & ~31u; t < m; t += kLsThreads)  // lane-0 slots: previous slot in another warp
        if (lane == 0 && t > 0 && v.RS[t - 1] == v.RS[t] && a.rid[s0 + t - 1] >= a.rid[s0 + t]) ++*bad;
}

// Starts words [i0, i1) of a 32-bit array on their way into L2 (a hint that
// is never waited for: only the 16-byte-aligned interior is named).
__device__ __forceinline__ void prefetch_l2(const uint32_t* base, uint64_t i0, uint64_t i1) {
    const uint64_t b0 = ((uint64_t)(uintptr_t)(base + i0) + 15) & ~15ull;
    const uint64_t b1 = (uint64_t)(uintptr_t)(base + i1) & ~15ull;
    if (b1 > b0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b0), "r"((uint32_t)(b1 - b0)) : "memory");
}

template <int KW>
__global__ void __launch_bounds__(kLsThreads, 1) local_sort_kernel(const LocalSortArgs a) {
    extern __shared__ __align__(16) unsigned char ls_raw[];
    __shared__ uint32_t s_list[2][kLsList];
    __shared__ uint32_t s_or[kMaxLearnedWords + 1];
    __shared__ uint32_t s_mm[2], s_bucket, s_next, s_cnt[2], s_grab, s_bcnt, s_bad;
    __shared__ uint64_t s_rng[2], s_nrng[2];  // start, end of this bucket and of the next one
    __shared__ uint32_t s_bstack[kLsBlockStack];
    __shared__ uint16_t s_bytes[768];
    __shared__ uint32_t s_pres[24], s_nbytes[3];
    // the four quarter-block groups' own split state
    __shared__ uint32_t s_gor[4][kMaxLearnedWords + 1], s_gmm[4][2], s_gwsum[4][kLsThreads / 4 / 32 + 1];
    __shared__ uint16_t s_gbytes[4][768];
    __shared__ uint32_t s_gpres[4][24], s_gnbytes[4][3];
    __shared__ __align__(16) uint32_t s_wpres[kLsWarps][16];  // warp splits: bitmaps of the window's top two bytes
    __shared__ uint32_t s_scan[kLsWarps + 1];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr uint32_t K = KW, KC = KW + 1;
    const uint32_t cap = a.cap;
    LearnedMisc* misc = a.misc;
    if (*(volatile uint32_t*)&misc->gate) return;
    if (tid == 0) s_bad = 0;  // failures found inside the splits (shared: they are counted by atomics)
    uint32_t* hist = reinterpret_cast<uint32_t*>(ls_raw);
    LsView<KW> v;
    v.keys = hist + kLsBins;
    v.A = reinterpret_cast<uint16_t*>(v.keys + (size_t)K * cap);
    v.T = v.A + cap;
    v.cap = cap;
    const uint32_t nb = min(misc->nsplit + 1, a.max_buckets);
    LsBlockState bst;
    bst.list = s_list[0];
    bst.count = &s_cnt[0];
    bst.stack = s_bstack;
    bst.scount = &s_bcnt;
    bst.orw = s_or;
    bst.mm = s_mm;
    bst.wsum = s_scan;
    // the 64-bit scans of the block splits borrow the warp splits' bitmaps (the
    // two never run at the same time): the block's, then each quarter's
    static_assert(sizeof(s_wpres) >= 8 * (kLsWarps + 1 + 4 * (kLsThreads / 4 / 32 + 1)), "scan storage");
    uint64_t* scan64 = reinterpret_cast<uint64_t*>(&s_wpres[0][0]);
    bst.wsum64 = scan64;
    bst.bytes = s_bytes;
    bst.pres = s_pres;
    bst.nbytes = s_nbytes;
    LsBlockState gst = bst;  // this thread's quarter-block group (ranges shorter than kLsGroupRange)
    {
        const uint32_t g = tid / (kLsThreads / 4);
        gst.orw = s_gor[g];
        gst.mm = s_gmm[g];
        gst.wsum = s_gwsum[g];
        gst.wsum64 = scan64 + (kLsWarps + 1) + g * (kLsThreads / 4 / 32 + 1);
        gst.bytes = s_gbytes[g];
        gst.pres = s_gpres[g];
        gst.nbytes = s_gnbytes[g];
    }
    uint64_t my_hash = 0;
    uint32_t my_bad = 0;
    constexpr uint32_t kNone = 0xFFFFFFFEu;  // no bucket taken ahead
    if (tid == 0) s_next = kNone;
    for (;;) {
        // Thread 0 takes the bucket taken ahead in the round before (or a new
        // one), then takes the following bucket now and starts its rows on
        // their way into L2, so that its load finds them there.
        if (tid == 0) {
            uint32_t b = s_next;
            if (*(volatile uint32_t*)&misc->fail) {
                b = 0xFFFFFFFFu;
            } else if (b == kNone) {
                b = atomicAdd(&misc->queue, 1u);
                if (b < nb) {
                    s_nrng[0] = a.start[b];
                    s_nrng[1] = a.start[b + 1];
                }
            }
            s_bucket = b;
            s_next = kNone;
            if (b < nb) {
                s_rng[0] = s_nrng[0];
                s_rng[1] = s_nrng[1];
                const uint32_t nx = atomicAdd(&misc->queue, 1u);
                s_next = nx;  // >= nb: the next round ends the loop
                if (nx < nb) {
                    const uint64_t n0 = a.start[nx], n1 = a.start[nx + 1];
                    s_nrng[0] = n0;
                    s_nrng[1] = n1;
                    if (n1 - n0 <= cap) {
                        for (uint32_t w = 0; w < K; ++w) prefetch_l2(a.ck + (uint64_t)w * a.ld, n0, n1);
                        prefetch_l2(a.rid, n0, n1);
                    }
                }
            }
        }
        __syncthreads();
        const uint32_t b = s_bucket;
        if (b >= nb) break;
        const uint64_t s0 = s_rng[0];
        const uint32_t m = (uint32_t)(s_rng[1] - s0);
        if (m == 0) {
            __syncthreads();
            continue;
        }
        if (tid == 0) atomicMax(&misc->counts[2], m);
        if (constant_range(a.spl, K, nb, b)) {
            if (m <= kConstInline) {
                check_constant(a, b, s0, s0, s0 + m, tid, kLsThreads, &my_hash, &my_bad);
            } else if (tid == 0) {
                const uint32_t slot = atomicAdd(&misc->nconst, 1u);
                if (slot < a.max_const) {
                    a.const_list[3 * slot] = (uint32_t)s0;
                    a.const_list[3 * slot + 1] = m;
                    a.const_list[3 * slot + 2] = b;
                } else {
                    ++my_bad;  // list full: the plain sort takes over
                }
            }
            if (tid == 0) atomicAdd(&misc->counts[1], 1u);
            __syncthreads();
            continue;
        }
        if (m > cap) {  // more than a block holds: the plain sort takes over
            if (tid == 0) {
                atomicAdd(&misc->counts[3], 1u);
                ++my_bad;
            }
            __syncthreads();
            continue;
        }
        uint32_t D;
        if (KW >= 2 && m >= 2 && narrow_range(a.spl, K, nb, b, &D)) {
            LnView ln;
            ln.R = v.keys;
            ln.RS = v.keys + cap;
            ln.A = v.A;
            ln.T = v.T;
            sort_narrow_bucket<KW>(a, ln, b, s0, m, D, hist, bst, s_list[1], &s_cnt[1], &s_grab, &s_bad, &my_hash,
                                   &my_bad);
            if (tid == 0) atomicAdd(&misc->counts[0], 1u);
            __syncthreads();
            continue;
        }

        // load the keys (four rows per thread in flight); OR of every key's
        // difference to the first
        if (tid < KC) s_or[tid] = 0;
        if (tid == 0) {
            s_cnt[0] = 0;
            s_cnt[1] = 0;
            s_bcnt = 0;
        }
        {
            uint32_t first[KW], orw[KW];
#pragma unroll
            for (uint32_t w = 0; w < K; ++w) {
                first[w] = a.ck[(uint64_t)w * a.ld + s0];
                orw[w] = 0;
            }
            for (uint32_t t0 = tid; t0 < m; t0 += 4 * kLsThreads) {
                uint32_t x[4][KW];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t t = t0 + u * kLsThreads;
#pragma unroll
                    for (uint32_t w = 0; w < K; ++w) x[u][w] = t < m ? a.ck[(uint64_t)w * a.ld + s0 + t] : first[w];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t t = t0 + u * kLsThreads;
#pragma unroll
                    for (uint32_t w = 0; w < K; ++w) {
                        if (t < m) v.keys[w * cap + t] = x[u][w];
                        orw[w] |= x[u][w] ^ first[w];
                    }
                }
            }
            __syncthreads();  // s_or zeroed
#pragma unroll
            for (uint32_t w = 0; w < K; ++w) {
                const uint32_t o = __reduce_or_sync(kFull, orw[w]);
                if (lane == 0 && o) atomicOr(&s_or[w + 1], o);
            }
        }
        __syncthreads();
        // step 1 on the bucket, then on every long range, then the warp rounds
        block_split<KW>(v, 0, m, true, hist, bst, &s_bad);
        for (;;) {
            // up to four ranges shorter than kLsGroupRange from the top of the
            // stack, each split by a quarter of the block on a quarter of the
            // bins (a split is bound by its chain of barriers, so four at a
            // time take little longer than one); else the top range, by the block
            const uint32_t nbk = s_bcnt;
            if (nbk == 0) break;
            uint32_t k = 0;
            while (k < 4 && k < nbk && (s_bstack[nbk - 1 - k] >> 16) < kLsGroupRange) ++k;
            const uint32_t g = tid / (kLsThreads / 4);
            const uint32_t r = s_bstack[nbk - 1 - (g < k ? g : 0u)];
            __syncthreads();  // every thread has read the stack
            if (tid == 0) s_bcnt = nbk - (k ? k : 1u);
            __syncthreads();  // the pops precede any push of the splits below
            if (k == 0)
                block_split<KW>(v, r & 0xFFFFu, r >> 16, false, hist, bst, &s_bad);
            else if (g < k)
                block_split<KW, kLsThreads / 4>(v, r & 0xFFFFu, r >> 16, false, hist + g * (kLsBins / 4), gst, &s_bad,
                                                LsGroup<kLsThreads / 4>{g});
            __syncthreads();
        }
        {
            uint32_t cur = 0;
            for (;;) {  // rounds of warp splits until no long range is left
                const uint32_t nr = min(s_cnt[cur], (uint32_t)kLsList);
                if (nr == 0) break;
                __syncthreads();  // every thread has read the count
                if (tid == 0) {
                    s_cnt[cur ^ 1] = 0;
                    s_grab = 0;
                }
                __syncthreads();
                for (;;) {
                    uint32_t e = 0;
                    if (lane == 0) e = atomicAdd(&s_grab, 1u);
                    e = __shfl_sync(kFull, e, 0);
                    if (e >= nr) break;
                    const uint32_t r = s_list[cur][e];
                    warp_split_range<KW>(v, r & 0xFFFFu, r >> 16, hist + warp * kLsWarpBins, s_wpres[warp],
                                         s_list[cur ^ 1], &s_cnt[cur ^ 1], &s_bad);
                }
                __syncthreads();
                cur ^= 1;
            }
        }
        __syncthreads();
        // the keys lie in the bucket's range
        if (tid == 0) {
            if (b > 0 && cmp_key_spl(v, v.A[0], a.spl + (size_t)(b - 1) * K) < 0) ++my_bad;
            if (b + 1 < nb && cmp_key_spl(v, v.A[m - 1], a.spl + (size_t)b * K) >= 0) ++my_bad;
        }
        // row ids gathered into registers (the bucket is rewritten in place,
        // so every read precedes the barrier below); each warp's last lane
        // leaves its row ids in shared memory for the next warp's first lane
        // (s_wpres is free after the warp rounds: 32 warps x 16 rows)
        uint32_t rr[kLsPerThread];
        const uint32_t jmax = (m + kLsThreads - 1) / kLsThreads;
#pragma unroll
        for (int j = 0; j < kLsPerThread; ++j) {
            const uint32_t t = tid + (uint32_t)j * kLsThreads;
            rr[j] = (uint32_t)j < jmax && t < m ? a.rid[s0 + v.A[t]] : 0u;
        }
        if (a.inject & CK_LEARNED_INJECT_RID_SWAP) {  // test only: exchange the row ids of positions 0 and 1
            const uint32_t other = __shfl_xor_sync(kFull, rr[0], 1);
            if (warp == 0 && lane < 2 && m >= 2) rr[0] = other;
        }
        static_assert(kLsPerThread <= 16, "one row id per warp and round in s_wpres");
        if (lane == 31)
#pragma unroll
            for (int j = 0; j < kLsPerThread; ++j) s_wpres[warp][j] = rr[j];
        __syncthreads();
        // one pass: each pair is checked against the pair before it (adjacent
        // keys ascend; equal keys by position and by row id) -- whose key,
        // position and row id come from the neighbouring lane, or for a
        // warp's first lane from shared memory -- and written back in order
        // with the hash of every output pair
#pragma unroll
        for (int j = 0; j < kLsPerThread; ++j) {
            if ((uint32_t)j >= jmax) break;  // uniform: every lane of the block has the same jmax
            const uint32_t t = tid + (uint32_t)j * kLsThreads;
            const bool in = t < m;
            const uint32_t f = in ? v.A[t] : 0u;
            uint32_t x[KW];
#pragma unroll
            for (int w = 0; w < KW; ++w) x[w] = in ? v.key(f, w) : 0u;
            uint32_t e = __shfl_up_sync(kFull, f, 1), rp = __shfl_up_sync(kFull, rr[j], 1);
            uint32_t y[KW];
#pragma unroll
            for (int w = 0; w < KW; ++w) y[w] = __shfl_up_sync(kFull, x[w], 1);
            if (lane == 0 && t >= 1 && in) {
                e = v.A[t - 1];
#pragma unroll
                for (int w = 0; w < KW; ++w) y[w] = v.key(e, w);
                rp = warp ? s_wpres[warp - 1][j] : s_wpres[kLsWarps - 1][j - 1];
            }
            if (t >= 1 && in) {
                int c = 0;
#pragma unroll
                for (int w = KW - 1; w >= 0; --w)
                    if (c == 0) c = y[w] < x[w] ? -1 : (y[w] > x[w] ? 1 : 0);
                if (c > 0 || (c == 0 && (e >= f || rp >= rr[j]))) ++my_bad;
            }
            if (in) {
                a.rid[s0 + t] = rr[j];
                uint64_t h = pair_hash_start(rr[j]);
#pragma unroll
                for (int w = 0; w < KW; ++w) {
                    a.ck[(uint64_t)w * a.ld + s0 + t] = x[w];
                    h = pair_hash_word(h, x[w]);
                }
                my_hash += pair_hash_end(h);
            }
        }
        if (tid == 0) atomicAdd(&misc->counts[0], 1u);
        __syncthreads();
    }
    // block totals
    __syncthreads();
    if (tid == 0) my_bad += s_bad;
    my_bad = __reduce_add_sync(kFull, my_bad);
    for (int o = 16; o > 0; o >>= 1) my_hash += __shfl_xor_sync(kFull, my_hash, o);
    if (lane == 0) {
        if (my_bad) atomicAdd(&misc->fail, my_bad);
        if (my_hash) atomicAdd(&misc->hash_out, (unsigned long long)my_hash);
    }
}

// The large constant buckets listed by the local sort, checked in chunks of
// kConstChunk pairs by all blocks.
__global__ void __launch_bounds__(256) const_check_kernel(const LocalSortArgs a) {
    __shared__ uint32_t s_pre[1025];
    __shared__ uint32_t s_chunk;
    LearnedMisc* misc = a.misc;
    if (*(volatile uint32_t*)&misc->gate) return;
    const uint32_t nc = min(misc->nconst, min(a.max_const, 1024u));
    if (nc == 0) return;
    if (threadIdx.x == 0) {  // chunk prefix over the list (short)
        uint32_t run = 0;
        for (uint32_t i = 0; i < nc; ++i) {
            s_pre[i] = run;
            run += (a.const_list[3 * i + 1] + kConstChunk - 1) / kConstChunk;
        }
        s_pre[nc] = run;
    }
    __syncthreads();
    const uint32_t total = s_pre[nc];
    uint64_t my_hash = 0;
    uint32_t my_bad = 0;
    for (;;) {
        if (threadIdx.x == 0) s_chunk = atomicAdd(&misc->const_queue, 1u);
        __syncthreads();
        const uint32_t c = s_chunk;
        __syncthreads();
        if (c >= total) break;
        uint32_t lo = 0, hi = nc - 1;  // last entry with s_pre <= c
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (s_pre[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        const uint64_t s0 = a.const_list[3 * lo];
        const uint32_t m = a.const_list[3 * lo + 1], b = a.const_list[3 * lo + 2];
        const uint64_t i0 = s0 + (uint64_t)(c - s_pre[lo]) * kConstChunk;
        const uint64_t i1 = min(s0 + m, i0 + kConstChunk);
        check_constant(a, b, s0, i0, i1, threadIdx.x, blockDim.x, &my_hash, &my_bad);
    }
    my_bad = __reduce_add_sync(kFull, my_bad);
    for (int o = 16; o > 0; o >>= 1) my_hash += __shfl_xor_sync(kFull, my_hash, o);
    if ((threadIdx.x & 31) == 0) {
        if (my_bad) atomicAdd(&misc->fail, my_bad);
        if (my_hash) atomicAdd(&misc->hash_out, (unsigned long long)my_hash);
    }
    if (threadIdx.x == 0 && misc->nconst > 1024u) atomicAdd(&misc->fail, 1u);  // not all listed: fall back
}

template <int KW>
static cudaError_t launch_local_kw(const LocalSortArgs& a, size_t smem, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(local_sort_kernel<KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    local_sort_kernel<KW><<<num_sms(), kLsThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_local_sort(const LocalSortArgs& a, cudaStream_t s) {
    const size_t smem = local_sort_smem(a.cap, a.K);
    if (a.cap > kLsMaxCap || a.cap > 65535 || smem + kLsStaticSmem > kSmemLimit) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (a.K) {
        case 1: e = launch_local_kw<1>(a, smem, s); break;
        case 2: e = launch_local_kw<2>(a, smem, s); break;
        case 3: e = launch_local_kw<3>(a, smem, s); break;
        case 4: e = launch_local_kw<4>(a, smem, s); break;
        case 5: e = launch_local_kw<5>(a, smem, s); break;
        case 6: e = launch_local_kw<6>(a, smem, s); break;
        case 7: e = launch_local_kw<7>(a, smem, s); break;
        case 8: e = launch_local_kw<8>(a, smem, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const_check_kernel<<<num_sms() * 2, 256, 0, s>>>(a);
    count_launch(2);
    return cudaGetLastError();
}

}  // namespace ck

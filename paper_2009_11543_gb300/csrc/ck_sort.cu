// ck_sort.cu -- stable LSD radix sort of (compressed key, row id) pairs.
//
// The paper sorts with a parallel comparison sort (Sec. 5.2, Appendix A);
// here the sort is a GPU onesweep radix sort (Adinets and Merrill, "Onesweep:
// a faster least significant digit radix sort for GPUs", 2022), written for
// word-major multi-word keys:
//
//   upsweep  one read of the keys -> the digit histogram of every pass
//   scan     per pass, exclusive scan of the histogram -> digit bucket bases
//   pass     per digit, one kernel: each block takes the next tile (dynamic
//            tile id), counts its digits and publishes the counts, ranks the
//            digits stably (warp ballots + per-warp counters), obtains the
//            counts of all earlier tiles by decoupled look-back, and scatters
//            every key word and the row id through shared memory so that each
//            digit run leaves as contiguous stores.
//
// Look-back words pack a 2-bit state (1 = tile aggregate, 2 = inclusive
// prefix) over a 30-bit count, hence n <= 2^30 - 1.  Every wait on a
// predecessor is bounded by spin_limit polls; when it runs out the block
// records CK_ETIMEOUT, assumes zero for the missing counts (which keeps every
// store in bounds), and carries on so that later tiles never wait forever.
#include "ck_internal.cuh"

namespace ck {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;
// Two shapes of the pass block over the same 4096-pair tile: 256 threads with
// 16 pairs each (more independent work per thread; 64 registers and a
// two-slot staging ring, so four blocks fit on an SM), or 512 threads with 8
// pairs each (three blocks), which is faster only for small passes of one key
// word that stay in L2.
constexpr int kTile = kPassTile;  // pairs per tile
constexpr int kPassThreadsWide = 512, kPassThreadsDeep = 256;
constexpr uint32_t kDeepMinArrays = 3;           // deep shape from this many arrays on,
constexpr uint64_t kWideMaxPairs = 1ull << 22;   // or above this many pairs
constexpr int kRing = 2;                         // staging buffers per block
constexpr int kPassBlocksPerSM = 3;              // resident blocks of the 512-thread shape
constexpr int kPassDeepBlocksPerSM = 4;          // of the 256-thread shape
constexpr int kUpThreads = 256;

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

// Digit of pass p (bits [shift, shift + bits) of the right-aligned key).
__device__ __forceinline__ uint32_t digit_of(const uint32_t* ck, uint64_t ld, uint64_t r, uint32_t shift,
                                             uint32_t bits) {
    const uint32_t w = shift >> 5, sh = shift & 31;
    uint32_t d = ck[(uint64_t)w * ld + r] >> sh;
    if (sh + bits > 32) d |= ck[(uint64_t)(w + 1) * ld + r] << (32 - sh);
    return d & ((1u << bits) - 1u);
}

// ------------------------------------------------------------------ upsweep
template <int RB>
__global__ void __launch_bounds__(kUpThreads) upsweep_kernel(const uint32_t* __restrict__ ck, uint64_t n, uint64_t ld,
                                                             uint32_t nbits, uint32_t p0, uint32_t np,
                                                             uint32_t* __restrict__ hist) {
    constexpr int BINS = 1 << RB;
    extern __shared__ uint32_t sh[];
    for (uint32_t i = threadIdx.x; i < np * BINS; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        for (uint32_t p = 0; p < np; ++p) {
            const uint32_t shift = (p0 + p) * RB;
            const uint32_t bits = min((uint32_t)RB, nbits - shift);
            atomicAdd(&sh[p * BINS + digit_of(ck, ld, r, shift, bits)], 1u);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < np * BINS; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[(uint64_t)p0 * BINS + i], sh[i]);
}

// The same with the key's KW words held in registers: every digit is cut from
// them (word indices are compile-time constants), so a key is read once.
template <int RB, int KW>
__global__ void __launch_bounds__(kUpThreads) upsweep_kw_kernel(const uint32_t* __restrict__ ck, uint64_t n,
                                                                uint64_t ld, uint32_t nbits, uint32_t p0,
                                                                uint32_t np, uint32_t* __restrict__ hist) {
    constexpr int BINS = 1 << RB, DIGITS = (32 * KW + RB - 1) / RB;
    extern __shared__ uint32_t sh[];
    for (uint32_t i = threadIdx.x; i < np * BINS; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        uint32_t w[KW];
#pragma unroll
        for (int k = 0; k < KW; ++k) w[k] = ck[(uint64_t)k * ld + r];
#pragma unroll
        for (int q = 0; q < DIGITS; ++q) {
            const uint32_t shift = (uint32_t)q * RB, wi = shift >> 5, s = shift & 31;
            if (q < (int)p0 || q >= (int)(p0 + np) || shift >= nbits) continue;
            uint32_t d = w[wi] >> s;
            if (s + RB > 32 && wi + 1 < KW) d |= w[wi + 1] << (32 - s);
            const uint32_t bits = nbits - shift < (uint32_t)RB ? nbits - shift : (uint32_t)RB;
            atomicAdd(&sh[(q - p0) * BINS + (d & ((1u << bits) - 1u))], 1u);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < np * BINS; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[(uint64_t)p0 * BINS + i], sh[i]);
}

template <int RB>
static void launch_upsweep(const uint32_t* ck, uint64_t n, uint64_t ld, uint32_t K, uint32_t nbits, uint32_t p0,
                           uint32_t np, uint32_t* hist, int grid, cudaStream_t s) {
    const size_t smem = sizeof(uint32_t) * np * (1u << RB);
    switch (K) {
        case 1: upsweep_kw_kernel<RB, 1><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist); break;
        case 2: upsweep_kw_kernel<RB, 2><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist); break;
        case 3: upsweep_kw_kernel<RB, 3><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist); break;
        case 4: upsweep_kw_kernel<RB, 4><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist); break;
        case 5: upsweep_kw_kernel<RB, 5><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist); break;
        case 6: upsweep_kw_kernel<RB, 6><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist); break;
        case 7: upsweep_kw_kernel<RB, 7><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist); break;
        case 8: upsweep_kw_kernel<RB, 8><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist); break;
        default: upsweep_kernel<RB><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist); break;
    }
}

template <int RB>
__global__ void __launch_bounds__(256) scan_kernel(uint32_t* hist) {
    __shared__ uint32_t scratch[256 / 32 + 1];
    block_exclusive_scan<256>(hist + (uint64_t)blockIdx.x * (1u << RB), 1 << RB, scratch);
}

__global__ void iota_kernel(uint32_t* out, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)i;
}

// ------------------------------------------------------------------ pass
// Shared memory of one pass block: a ring of kRing staging buffers (one array
// of the tile each), per-warp digit counters, per-slot source position,
// per-digit tile counts and destinations, and the ring's mbarriers.
template <int RB, int THREADS>
struct PassSmem {
    static constexpr int BINS = 1 << RB, WARPS = THREADS / 32;
    uint32_t stage[kRing][kTile];
    uint16_t whist[WARPS][BINS];  // counts <= kTile fit 16 bits
    uint16_t src_pos[kTile];
    uint32_t tile_total[BINS];
    uint32_t tile_excl[BINS];
    int32_t dest_base[BINS];
    uint32_t scratch[WARPS + 2];
    int16_t use[kMaxPassArrays];  // staging sequence number of each array, -1 if not staged
    alignas(8) uint64_t bar[kRing];
};

template <int RB, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == 256 ? kPassDeepBlocksPerSM : kPassBlocksPerSM)
    onesweep_pass_kernel(const PassArgs a, const __grid_constant__ PassArrays arr) {
    constexpr int kPassThreads = THREADS;
    constexpr int BINS = 1 << RB, WARPS = THREADS / 32, ITEMS = kTile / THREADS, WITEMS = 32 * ITEMS;
    static_assert(ITEMS * THREADS == kTile, "tile size of the pass kernel");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PassSmem<RB, THREADS>& S = *reinterpret_cast<PassSmem<RB, THREADS>*>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t n = a.n;
    const uint32_t sh = a.sh;
    const bool straddle = a.straddle != 0;
    const uint32_t M = a.narr;
    if (tid == 0) {
        S.scratch[WARPS + 1] = atomicAdd(a.tile_counter, 1u);
        int16_t u = 0;
        for (uint32_t m = 0; m < M; ++m) S.use[m] = arr.src[m] ? u++ : (int16_t)-1;
        for (int b = 0; b < kRing; ++b) mbar_init(&S.bar[b], 1);
        fence_mbar_init();
    }
    for (int i = tid; i < WARPS * BINS; i += kPassThreads) (&S.whist[0][0])[i] = 0;
    for (int i = tid; i < BINS; i += kPassThreads) S.tile_total[i] = 0;
    __syncthreads();
    const uint32_t tile = S.scratch[WARPS + 1];
    const uint64_t tile_base = (uint64_t)tile * kTile;
    const uint32_t count = (uint32_t)min((uint64_t)kTile, n - tile_base);
    const bool bulk = a.bulk && count == (uint32_t)kTile;

    // array m lives in ring slot use[m] % kRing; its k-th use is phase k of that slot's barrier
    auto buf_of = [&](uint32_t m) -> uint32_t* { return S.stage[S.use[m] % kRing]; };
    auto issue = [&](uint32_t m) {  // thread 0 only, bulk tiles only
        if (arr.src[m])
            bulk_load(buf_of(m), arr.src[m] + tile_base, kTile * sizeof(uint32_t), &S.bar[S.use[m] % kRing]);
    };
    auto stage_plain = [&](uint32_t m) {  // all threads; the caller synchronises
        if (arr.src[m]) {
            uint32_t* b = buf_of(m);
            for (uint32_t e = tid; e < count; e += kPassThreads) b[e] = arr.src[m][tile_base + e];
        }
    };
    auto wait_array = [&](uint32_t m) {
        if (!arr.src[m]) return;
        if (!mbar_wait(&S.bar[S.use[m] % kRing], (uint32_t)(S.use[m] / kRing) & 1u, a.spin_limit))
            report(a.status, CK_ETIMEOUT, (uint64_t)a.pass | ((uint64_t)tile << 16) | (1ull << 47));
    };
    // the staged arrays whose use < kRing can all start now
    const uint32_t staged_total = [&] {
        uint32_t c = 0;
        for (uint32_t m = 0; m < M; ++m) c += arr.src[m] ? 1u : 0u;
        return c;
    }();

    if (bulk) {
        if (tid == 0)
            for (uint32_t m = 0; m < M; ++m)
                if (arr.src[m] && S.use[m] < kRing) issue(m);
        wait_array(0);
        if (straddle) wait_array(1);
    } else {
        stage_plain(0);
        if (straddle) stage_plain(1);
        __syncthreads();
    }
    const uint32_t* dig0 = buf_of(0);
    const uint32_t* dig1 = straddle ? buf_of(1) : dig0;

    // 1. digits of this warp's items, warp-striped: item j of lane l is e = warp*WITEMS + 32j + l
    const uint32_t dmask = (1u << a.bits) - 1u;
    uint32_t dr[ITEMS];  // digit in bits 0..15, rank within the warp in bits 16..31
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t e = warp * WITEMS + 32 * j + lane;
        uint32_t d = 0;
        if (e < count) {
            d = dig0[e] >> sh;
            if (straddle) d |= dig1[e] << (32 - sh);
            d &= dmask;
        }
        dr[j] = d;
        if (e < count) atomicAdd(&S.tile_total[d], 1u);
    }
    __syncthreads();

    // 2. the tile's digit counts are published before the ranking, so later
    //    tiles' look-backs need not wait for it
    const bool stall = (a.inject & CK_INJECT_STALL_FIRST_TILE) && a.pass == 0 && tile == 0;
    if (!stall)
        for (int b = tid; b < BINS; b += kPassThreads)
            st_relaxed(&a.lookback[(uint64_t)tile * BINS + b], (tile == 0 ? kFlagPrefix : kFlagAgg) | S.tile_total[b]);

    // 3. stable rank within the warp: lanes with equal digits found by RB ballots
    uint16_t* my = S.whist[warp];
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const bool valid = warp * WITEMS + 32 * j + lane < count;
        const uint32_t d = dr[j];
        uint32_t peers = __ballot_sync(kFull, valid);
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const bool bit = (d >> b) & 1u;
            const uint32_t bal = __ballot_sync(kFull, bit);
            peers &= bit ? bal : ~bal;
        }
        const uint32_t base = valid ? my[d] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0) my[d] = (uint16_t)(base + __popc(peers));
        __syncwarp();
        dr[j] = d | ((base + __popc(peers & lt)) << 16);  // < WITEMS, fits 16 bits
    }
    __syncthreads();

    // 4. per digit: exclusive prefix over warps
    for (int b = tid; b < BINS; b += kPassThreads) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) {
            const uint32_t t = S.whist[w][b];
            S.whist[w][b] = (uint16_t)sum;
            sum += t;
        }
        S.tile_excl[b] = sum;
    }
    __syncthreads();
    block_exclusive_scan<kPassThreads>(S.tile_excl, BINS, S.scratch);

    // 5. decoupled look-back: counts of every digit in all earlier tiles.  The
    //    thread of digit b reads the words of the kLookDepth tiles before the
    //    current position at once (the warp's threads read consecutive digits,
    //    so every word load is one line per warp), adds them up to the nearest
    //    tile holding an inclusive prefix, and repeats further back while none
    //    does; it waits (bounded) at a tile that has published nothing yet.
    //    Tiles before tile 0 read as prefix 0.
    for (int b = tid; b < BINS; b += kPassThreads) {
        constexpr int kLookDepth = 8;
        uint32_t excl = 0;
        if (tile > 0) {
            int64_t next = (int64_t)tile - 1;  // newest tile not yet added
            uint32_t polls = 0;
            while (next >= 0) {
                uint32_t v[kLookDepth];
#pragma unroll
                for (int j = 0; j < kLookDepth; ++j)
                    v[j] = next - j >= 0 ? ld_relaxed(&a.lookback[(uint64_t)(next - j) * BINS + b]) : kFlagPrefix;
                bool done = false;
#pragma unroll
                for (int j = 0; j < kLookDepth; ++j) {
                    const uint32_t flag = v[j] & ~kValMask;
                    if (flag == 0) break;  // tile next - j has not published: wait for it
                    excl += v[j] & kValMask;
                    --next;
                    if (flag == kFlagPrefix) {
                        done = true;
                        break;
                    }
                }
                if (done || next < 0) break;
                if ((v[0] & ~kValMask) == 0) {  // no progress: the newest word is not published yet
                    if (++polls > a.spin_limit) {
                        report(a.status, CK_ETIMEOUT, (uint64_t)a.pass | ((uint64_t)tile << 16));
                        break;
                    }
                    __nanosleep(64);
                }
            }
            st_relaxed(&a.lookback[(uint64_t)tile * BINS + b], kFlagPrefix | ((excl + S.tile_total[b]) & kValMask));
        }
        S.dest_base[b] = (int32_t)(a.bucket_base[b] + excl) - (int32_t)S.tile_excl[b];
    }

    // 6. local slot of every item in digit order: record where it comes from
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t e = warp * WITEMS + 32 * j + lane;
        const uint32_t d = dr[j] & 0xFFFFu;
        if (e < count) S.src_pos[(dr[j] >> 16) + S.tile_excl[d] + my[d]] = (uint16_t)e;
    }
    __syncthreads();
    // this thread's slots tid + i*THREADS: source position and global destination
    // (the digit is re-read from the staged digit word(s), not refilled before this)
    uint32_t srcp[ITEMS], dst[ITEMS];
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const uint32_t s = tid + i * kPassThreads;
        srcp[i] = 0;
        dst[i] = 0;
        if (s < count) {
            const uint32_t e = S.src_pos[s];
            uint32_t d = dig0[e] >> sh;
            if (straddle) d |= dig1[e] << (32 - sh);
            srcp[i] = e;
            dst[i] = (uint32_t)(S.dest_base[d & dmask] + (int32_t)s);  // < 2^30
        }
    }
    __syncthreads();  // every thread has read the digit words; their slots may be refilled

    // 7. every array in staging order: wait for it, scatter it, refill its ring slot
    for (uint32_t m = 0; m < M; ++m) {
        const bool digit_array = m == 0 || (straddle && m == 1);
        if (bulk) {
            if (!digit_array) wait_array(m);
        } else if (!digit_array) {
            stage_plain(m);
            __syncthreads();
        }
        uint32_t* out = arr.dst[m];
        if (out) {
            const bool iota = arr.src[m] == nullptr;
            const uint32_t* buf = iota ? nullptr : buf_of(m);
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t s = tid + i * kPassThreads;
                if (s < count) out[dst[i]] = iota ? (uint32_t)(tile_base + srcp[i]) : buf[srcp[i]];
            }
        }
        if (bulk && arr.src[m] && (uint32_t)S.use[m] + kRing < staged_total) {
            __syncthreads();  // ring slot of array m is free again
            if (tid == 0) {
                fence_proxy_async_smem();
                for (uint32_t q = m + 1; q < M; ++q)
                    if (arr.src[q] && S.use[q] == S.use[m] + kRing) issue(q);
            }
        } else if (!bulk) {
            __syncthreads();
        }
    }
}

// Launches one pass; `arrays` lists the arrays in staging order.
template <int RB, int THREADS>
static cudaError_t launch_pass_shape(const PassArgs& a, const PassArrays& arrays, uint32_t tiles, cudaStream_t s) {
    constexpr size_t smem = sizeof(PassSmem<RB, THREADS>);
    static_assert(sizeof(PassSmem<RB, THREADS>) <= 227 * 1024, "pass block exceeds shared memory");
    cudaError_t e = cudaFuncSetAttribute(onesweep_pass_kernel<RB, THREADS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    onesweep_pass_kernel<RB, THREADS><<<tiles, THREADS, smem, s>>>(a, arrays);
    count_launch();
    return cudaGetLastError();
}

template <int RB>
static cudaError_t launch_pass(const PassArgs& a, const PassArrays& arrays, uint32_t tiles, cudaStream_t s) {
    return a.narr >= kDeepMinArrays || a.n > kWideMaxPairs
               ? launch_pass_shape<RB, kPassThreadsDeep>(a, arrays, tiles, s)
               : launch_pass_shape<RB, kPassThreadsWide>(a, arrays, tiles, s);
}

cudaError_t launch_onesweep_pass(uint32_t rb, const PassArgs& a, const PassArrays& arrays, uint32_t tiles,
                                 cudaStream_t s) {
    switch (rb) {
        case 4: return launch_pass<4>(a, arrays, tiles, s);
        case 5: return launch_pass<5>(a, arrays, tiles, s);
        case 6: return launch_pass<6>(a, arrays, tiles, s);
        case 7: return launch_pass<7>(a, arrays, tiles, s);
        case 8: return launch_pass<8>(a, arrays, tiles, s);
        case 9: return launch_pass<9>(a, arrays, tiles, s);
        case 10: return launch_pass<10>(a, arrays, tiles, s);
        case 11: return launch_pass<11>(a, arrays, tiles, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_bucket_scan(uint32_t* hist, uint32_t sets, uint32_t rb, cudaStream_t s) {
    switch (rb) {
        case 4: scan_kernel<4><<<sets, 256, 0, s>>>(hist); break;
        case 5: scan_kernel<5><<<sets, 256, 0, s>>>(hist); break;
        case 6: scan_kernel<6><<<sets, 256, 0, s>>>(hist); break;
        case 7: scan_kernel<7><<<sets, 256, 0, s>>>(hist); break;
        case 8: scan_kernel<8><<<sets, 256, 0, s>>>(hist); break;
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool make_sort_plan(uint64_t n, uint32_t K, uint32_t nbits, uint32_t digit_bits, SortPlan* p, uint64_t ld) {
    if (digit_bits == 0) digit_bits = 8;
    p->ld = ld ? ld : CK_LD(n);
    if (p->ld < n) return false;
    if (digit_bits < 4 || digit_bits > 11) return false;
    p->digit_bits = digit_bits;
    p->passes = (nbits + digit_bits - 1) / digit_bits;
    p->tile = kTile;
    p->tiles = (uint32_t)((n + kTile - 1) / kTile);
    p->K = K;
    const size_t bins = (size_t)1 << digit_bits;
    size_t off = 0;
    p->off_hist = off;
    off = align256(off + sizeof(uint32_t) * bins * p->passes);
    p->off_counter = off;
    off = align256(off + sizeof(uint32_t) * p->passes);
    p->off_lookback = off;
    off = align256(off + sizeof(uint32_t) * bins * (size_t)p->tiles * p->passes);
    p->off_alt_ck = off;
    off = align256(off + sizeof(uint32_t) * (size_t)K * p->ld);
    p->off_alt_rid = off;
    off = align256(off + sizeof(uint32_t) * n);
    p->total = off;
    return true;
}

// All pass histograms of compressed keys, in chunks that fit 64 KB of shared memory.
template <int RB>
static cudaError_t upsweep_all(const uint32_t* ck_in, uint64_t n, uint64_t ld, uint32_t K, uint32_t nbits,
                               uint32_t passes, uint32_t* hist, cudaStream_t s) {
    constexpr int BINS = 1 << RB;
    cudaError_t e = cudaSuccess;
    const uint32_t chunk = (uint32_t)(65536 / (sizeof(uint32_t) * BINS));
    const int up_grid = num_sms() * 8;  // 8 blocks of 256 threads per SM
    if (passes * BINS * sizeof(uint32_t) > 48 * 1024) {  // chunks above the default shared-memory limit
        e = cudaFuncSetAttribute(upsweep_kernel<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
        if (e != cudaSuccess) return e;
        if (K <= 8) {
            const void* fn[8] = {(const void*)upsweep_kw_kernel<RB, 1>, (const void*)upsweep_kw_kernel<RB, 2>,
                                 (const void*)upsweep_kw_kernel<RB, 3>, (const void*)upsweep_kw_kernel<RB, 4>,
                                 (const void*)upsweep_kw_kernel<RB, 5>, (const void*)upsweep_kw_kernel<RB, 6>,
                                 (const void*)upsweep_kw_kernel<RB, 7>, (const void*)upsweep_kw_kernel<RB, 8>};
            e = cudaFuncSetAttribute(fn[K - 1], cudaFuncAttributeMaxDynamicSharedMemorySize, 65536);
            if (e != cudaSuccess) return e;
        }
    }
    for (uint32_t p0 = 0; p0 < passes; p0 += chunk) {
        const uint32_t np = min(chunk, passes - p0);
        launch_upsweep<RB>(ck_in, n, ld, K, nbits, p0, np, hist, up_grid, s);
        count_launch();
    }
    return cudaGetLastError();
}

template <int RB>
static cudaError_t run_sort_rb(const SortPlan& p, const uint32_t* ck_in, const uint32_t* rid_in, uint32_t* ck_out,
                               uint32_t* rid_out, uint64_t n, uint32_t nbits, uint32_t spin_limit, uint32_t inject,
                               uint32_t flags, cudaEvent_t* ev, unsigned char* ws, cudaStream_t s,
                               const uint32_t* hist_in) {
    constexpr int BINS = 1 << RB;
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + p.off_hist);
    uint32_t* counters = reinterpret_cast<uint32_t*>(ws + p.off_counter);
    uint32_t* lookback = reinterpret_cast<uint32_t*>(ws + p.off_lookback);
    uint32_t* alt_ck = reinterpret_cast<uint32_t*>(ws + p.off_alt_ck);
    uint32_t* alt_rid = reinterpret_cast<uint32_t*>(ws + p.off_alt_rid);
    const uint64_t ld = p.ld;
    cudaError_t e = cudaMemsetAsync(ws, 0, p.off_alt_ck, s);
    if (e != cudaSuccess) return e;

    if (hist_in) {  // counted during extraction (ck_extract_hist)
        e = cudaMemcpyAsync(hist, hist_in, sizeof(uint32_t) * BINS * p.passes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    } else {
        e = upsweep_all<RB>(ck_in, n, ld, p.K, nbits, p.passes, hist, s);
        if (e != cudaSuccess) return e;
    }
    scan_kernel<RB><<<p.passes, 256, 0, s>>>(hist);
    count_launch();

    const bool perm_only = (flags & CK_SORT_PERM_ONLY) != 0;
    const bool inplace = (ck_in == ck_out) || (rid_in != nullptr && rid_in == rid_out);
    auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    const uint32_t bulk = al16(ck_in) && al16(ck_out) && al16(rid_out) && (rid_in == nullptr || al16(rid_in)) ? 1u : 0u;
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    const uint32_t* cur_ck = ck_in;
    const uint32_t* cur_rid = rid_in;
    static thread_local PassArrays arrays;
    for (uint32_t q = 0; q < p.passes; ++q) {
        const bool to_out = inplace ? (q % 2 == 1) : ((p.passes - 1 - q) % 2 == 0);
        uint32_t* out_ck = to_out ? ck_out : alt_ck;
        uint32_t* out_rid = to_out ? rid_out : alt_rid;
        const uint32_t shift = q * RB, wlo = shift >> 5, sh = shift & 31;
        const uint32_t bits = min((uint32_t)RB, nbits - shift);
        const bool straddle = sh + bits > 32;
        // first key word still needed after this pass (all of them unless only
        // the permutation is wanted)
        const uint32_t keep = perm_only ? (q + 1 < p.passes ? ((q + 1) * RB) >> 5 : p.K) : 0u;
        uint32_t m = 0;
        auto add_word = [&](uint32_t w) {
            arrays.src[m] = cur_ck + (uint64_t)w * ld;
            arrays.dst[m] = w >= keep ? out_ck + (uint64_t)w * ld : nullptr;
            ++m;
        };
        add_word(wlo);
        if (straddle) add_word(wlo + 1);
        for (uint32_t w = keep; w < p.K; ++w)
            if (w != wlo && !(straddle && w == wlo + 1)) add_word(w);
        arrays.src[m] = cur_rid;
        arrays.dst[m] = out_rid;
        ++m;
        PassArgs a;
        a.n = n;
        a.narr = m;
        a.sh = sh;
        a.bits = bits;
        a.straddle = straddle ? 1u : 0u;
        a.pass = q;
        a.bulk = bulk;
        a.bucket_base = hist + (size_t)q * BINS;
        a.lookback = lookback + (size_t)q * BINS * p.tiles;
        a.tile_counter = counters + q;
        a.spin_limit = spin_limit;
        a.inject = inject;
        a.status = status_ptr();
        e = launch_pass<RB>(a, arrays, p.tiles, s);
        if (e != cudaSuccess) return e;
        if (ev && (e = cudaEventRecord(ev[q + 1], s)) != cudaSuccess) return e;
        cur_ck = out_ck;
        cur_rid = out_rid;
    }
    if (!perm_only && cur_ck != ck_out) {
        e = cudaMemcpy2DAsync(ck_out, sizeof(uint32_t) * ld, cur_ck, sizeof(uint32_t) * ld, sizeof(uint32_t) * n, p.K,
                              cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    if (cur_rid != rid_out) {
        e = cudaMemcpyAsync(rid_out, cur_rid, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t run_sort(const SortPlan& p, const uint32_t* ck_in, const uint32_t* rid_in, uint32_t* ck_out,
                     uint32_t* rid_out, uint64_t n, uint32_t nbits, uint32_t spin_limit, uint32_t inject,
                     uint32_t flags, cudaEvent_t* ev, unsigned char* ws, cudaStream_t s, const uint32_t* hist_in) {
    if (p.passes == 0) {  // nothing to order: outputs are the inputs
        cudaError_t e = cudaSuccess;
        if (ck_out != ck_in)
            e = cudaMemcpy2DAsync(ck_out, sizeof(uint32_t) * p.ld, ck_in, sizeof(uint32_t) * p.ld, sizeof(uint32_t) * n,
                                  p.K, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        if (rid_in == nullptr) {
            iota_kernel<<<num_sms() * 4, 256, 0, s>>>(rid_out, n);
            count_launch();
        } else if (rid_out != rid_in) {
            e = cudaMemcpyAsync(rid_out, rid_in, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
        }
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    switch (p.digit_bits) {
        case 4: return run_sort_rb<4>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in);
        case 5: return run_sort_rb<5>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in);
        case 6: return run_sort_rb<6>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in);
        case 7: return run_sort_rb<7>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in);
        case 8: return run_sort_rb<8>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in);
        case 9: return run_sort_rb<9>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in);
        case 10: return run_sort_rb<10>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in);
        case 11: return run_sort_rb<11>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_upsweep_all(const uint32_t* ck, uint64_t n, uint64_t ld, uint32_t K, uint32_t nbits, uint32_t rb,
                               uint32_t* hist, cudaStream_t s) {
    const uint32_t passes = (nbits + rb - 1) / rb;
    if (passes == 0) return cudaSuccess;
    switch (rb) {
        case 4: return upsweep_all<4>(ck, n, ld, K, nbits, passes, hist, s);
        case 5: return upsweep_all<5>(ck, n, ld, K, nbits, passes, hist, s);
        case 6: return upsweep_all<6>(ck, n, ld, K, nbits, passes, hist, s);
        case 7: return upsweep_all<7>(ck, n, ld, K, nbits, passes, hist, s);
        case 8: return upsweep_all<8>(ck, n, ld, K, nbits, passes, hist, s);
        case 9: return upsweep_all<9>(ck, n, ld, K, nbits, passes, hist, s);
        case 10: return upsweep_all<10>(ck, n, ld, K, nbits, passes, hist, s);
        case 11: return upsweep_all<11>(ck, n, ld, K, nbits, passes, hist, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ck

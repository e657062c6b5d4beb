// ck_pass.cu -- one onesweep pass of the radix sort (ck_sort.cu runs them):
// each block takes the next tile (dynamic tile id), counts its digits and
// publishes the counts, ranks the digits stably (warp ballots + per-warp
// counters), obtains the counts of all earlier tiles by decoupled look-back,
// and scatters every key word and the row id through shared memory so that
// each digit run leaves as contiguous stores.
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
// Shapes of the pass block.  The default 4096-pair tile has two: 256 threads
// with 16 pairs each (more independent work per thread; 64 registers and a
// two-slot staging ring, so four blocks fit on an SM), or 512 threads with 8
// pairs each (three blocks), which is faster only for small passes of one key
// word that stay in L2.  The tile size is a tuning knob of the sort
// (ck_sort_opts.tile): 2048-pair tiles take 256 threads with 8 pairs (six
// blocks per SM), 8192-pair tiles 512 threads with 16 pairs (two blocks).
// Smaller tiles mean more look-back words and more blocks in flight, larger
// ones fewer tiles and longer contiguous runs per digit.
constexpr int kPassThreadsWide = 512, kPassThreadsDeep = 256;
constexpr uint32_t kDeepMinArrays = 3;           // deep shape from this many arrays on,
constexpr uint64_t kWideMaxPairs = 1ull << 22;   // or above this many pairs
constexpr int kRing = 2;                         // staging buffers per block

// resident blocks per SM of a (threads, tile) shape
__host__ __device__ constexpr int pass_blocks_per_sm(int threads, int tile) {
    return tile == 2048 ? 6 : tile == 8192 ? 2 : threads == 256 ? 4 : 3;
}

// ------------------------------------------------------------------ pass
// Shared memory of one pass block: a ring of kRing staging buffers (one array
// of the tile each), per-warp digit counters, per-slot source position,
// per-digit tile counts and destinations, and the ring's mbarriers.
template <int RB, int THREADS, int TILE>
struct PassSmem {
    static constexpr int BINS = 1 << RB, WARPS = THREADS / 32;
    uint32_t stage[kRing][TILE];
    uint16_t whist[WARPS][BINS];  // counts <= TILE fit 16 bits
    uint16_t src_pos[TILE];
    uint32_t tile_total[BINS];
    uint32_t tile_excl[BINS];
    int32_t dest_base[BINS];
    uint32_t scratch[WARPS + 2];
    int16_t use[kMaxPassArrays];  // staging sequence number of each array, -1 if not staged
    alignas(8) uint64_t bar[kRing];
};

// PERSIST: a fixed grid whose blocks take tiles until none is left, staging
// with plain loads (the shape of a gated sort that usually does not run: when
// the gate is shut, a few hundred blocks return at once instead of one block
// per tile).  Without PERSIST every block takes one tile.
template <int RB, int THREADS, bool PERSIST, int TILE>
__global__ void __launch_bounds__(THREADS, pass_blocks_per_sm(THREADS, TILE))
    onesweep_pass_kernel(const PassArgs a, const __grid_constant__ PassArrays arr) {
    constexpr int kPassThreads = THREADS, kTile = TILE;
    constexpr int BINS = 1 << RB, WARPS = THREADS / 32, ITEMS = kTile / THREADS, WITEMS = 32 * ITEMS;
    static_assert(ITEMS * THREADS == kTile, "tile size of the pass kernel");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    PassSmem<RB, THREADS, TILE>& S = *reinterpret_cast<PassSmem<RB, THREADS, TILE>*>(smem_raw);

    if (a.gate && *(volatile const uint32_t*)a.gate != a.gate_run) return;  // decided on the device
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t n = a.n;
    const uint32_t sh = a.sh;
    const bool straddle = a.straddle != 0;
    const uint32_t M = a.narr;
    if (tid == 0) {
        int16_t u = 0;
        for (uint32_t m = 0; m < M; ++m) S.use[m] = arr.src[m] ? u++ : (int16_t)-1;
        for (int b = 0; b < kRing; ++b) mbar_init(&S.bar[b], 1);
        fence_mbar_init();
    }
  for (;;) {
    if (tid == 0) S.scratch[WARPS + 1] = atomicAdd(a.tile_counter, 1u);
    for (int i = tid; i < WARPS * BINS; i += kPassThreads) (&S.whist[0][0])[i] = 0;
    for (int i = tid; i < BINS; i += kPassThreads) S.tile_total[i] = 0;
    __syncthreads();
    const uint32_t tile = S.scratch[WARPS + 1];
    if (PERSIST && tile >= a.tiles) break;
    const uint64_t tile_base = (uint64_t)tile * kTile;
    const uint32_t count = (uint32_t)min((uint64_t)kTile, n - tile_base);
    const bool bulk = !PERSIST && a.bulk && count == (uint32_t)kTile;

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
    if (!PERSIST) break;
    __syncthreads();  // the tile's shared state is free for the next tile
  }
}

// Launches one pass; `arrays` lists the arrays in staging order.  A pass
// gated to run only on the device's say-so (a fallback) takes the persistent
// shape (default tile only).
template <int RB, int THREADS, int TILE>
static cudaError_t launch_pass_shape(const PassArgs& a_in, const PassArrays& arrays, uint32_t tiles, cudaStream_t s) {
    constexpr size_t smem = sizeof(PassSmem<RB, THREADS, TILE>);
    static_assert(sizeof(PassSmem<RB, THREADS, TILE>) <= 227 * 1024, "pass block exceeds shared memory");
    PassArgs a = a_in;
    a.tiles = tiles;
    const bool persist = a.gate != nullptr && a.gate_run != 0;
    if (persist && TILE != kPassTile) return cudaErrorInvalidValue;
    const void* fn = persist ? (const void*)onesweep_pass_kernel<RB, THREADS, true, kPassTile>
                             : (const void*)onesweep_pass_kernel<RB, THREADS, false, TILE>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (persist) {
        const uint32_t per_sm = pass_blocks_per_sm(THREADS, kPassTile);
        const uint32_t grid = (uint32_t)min((uint64_t)tiles, (uint64_t)num_sms() * per_sm);
        onesweep_pass_kernel<RB, THREADS, true, kPassTile><<<grid, THREADS, smem, s>>>(a, arrays);
    } else {
        onesweep_pass_kernel<RB, THREADS, false, TILE><<<tiles, THREADS, smem, s>>>(a, arrays);
    }
    count_launch();
    return cudaGetLastError();
}

template <int RB>
static cudaError_t launch_pass(const PassArgs& a, const PassArrays& arrays, uint32_t tile, uint32_t tiles,
                               cudaStream_t s) {
    switch (tile) {
        case 2048: return launch_pass_shape<RB, kPassThreadsDeep, 2048>(a, arrays, tiles, s);
        case 8192: return launch_pass_shape<RB, kPassThreadsWide, 8192>(a, arrays, tiles, s);
        case kPassTile:
            return a.narr >= kDeepMinArrays || a.n > kWideMaxPairs
                       ? launch_pass_shape<RB, kPassThreadsDeep, kPassTile>(a, arrays, tiles, s)
                       : launch_pass_shape<RB, kPassThreadsWide, kPassTile>(a, arrays, tiles, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_onesweep_pass(uint32_t rb, const PassArgs& a, const PassArrays& arrays, uint32_t tiles,
                                 cudaStream_t s, uint32_t tile) {
    switch (rb) {
        case 4: return launch_pass<4>(a, arrays, tile, tiles, s);
        case 5: return launch_pass<5>(a, arrays, tile, tiles, s);
        case 6: return launch_pass<6>(a, arrays, tile, tiles, s);
        case 7: return launch_pass<7>(a, arrays, tile, tiles, s);
        case 8: return launch_pass<8>(a, arrays, tile, tiles, s);
        case 9: return launch_pass<9>(a, arrays, tile, tiles, s);
        case 10: return launch_pass<10>(a, arrays, tile, tiles, s);
        case 11: return launch_pass<11>(a, arrays, tile, tiles, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ck

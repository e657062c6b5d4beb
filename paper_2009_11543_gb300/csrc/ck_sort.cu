// ck_sort.cu -- stable LSD radix sort of (compressed key, row id) pairs.
//
// The paper sorts with a parallel comparison sort (Sec. 5.2, Appendix A);
// here the sort is a GPU onesweep radix sort (Adinets and Merrill, "Onesweep:
// a faster least significant digit radix sort for GPUs", 2022), written for
// word-major multi-word keys:
//
//   upsweep  one read of the keys -> the digit histogram of every pass
//   scan     per pass, exclusive scan of the histogram -> digit bucket bases
//   pass     per digit, one onesweep kernel (ck_pass.cu).
#include "ck_internal.cuh"

namespace ck {

constexpr int kUpThreads = 256;

// Digit of pass p (bits [shift, shift + bits) of the right-aligned key).
__device__ __forceinline__ uint32_t digit_of(const uint32_t* ck, uint64_t ld, uint64_t r, uint32_t shift,
                                             uint32_t bits) {
    const uint32_t w = shift >> 5, sh = shift & 31;
    uint32_t d = ck[(uint64_t)w * ld + r] >> sh;
    if (sh + bits > 32) d |= ck[(uint64_t)(w + 1) * ld + r] << (32 - sh);
    return d & ((1u << bits) - 1u);
}

// ------------------------------------------------------------------ upsweep
// A gated kernel (gate != NULL) returns at once unless *gate != 0.
__device__ __forceinline__ bool gated_off(const uint32_t* gate) {
    return gate != nullptr && *(volatile const uint32_t*)gate == 0;
}

template <int RB>
__global__ void __launch_bounds__(kUpThreads) upsweep_kernel(const uint32_t* __restrict__ ck, uint64_t n, uint64_t ld,
                                                             uint32_t nbits, uint32_t p0, uint32_t np,
                                                             uint32_t* __restrict__ hist, const uint32_t* gate) {
    constexpr int BINS = 1 << RB;
    extern __shared__ uint32_t sh[];
    if (gated_off(gate)) return;
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
                                                                uint32_t np, uint32_t* __restrict__ hist,
                                                                const uint32_t* gate) {
    constexpr int BINS = 1 << RB, DIGITS = (32 * KW + RB - 1) / RB;
    extern __shared__ uint32_t sh[];
    if (gated_off(gate)) return;
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
                           uint32_t np, uint32_t* hist, int grid, cudaStream_t s, const uint32_t* g) {
    const size_t smem = sizeof(uint32_t) * np * (1u << RB);
    switch (K) {
        case 1: upsweep_kw_kernel<RB, 1><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist, g); break;
        case 2: upsweep_kw_kernel<RB, 2><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist, g); break;
        case 3: upsweep_kw_kernel<RB, 3><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist, g); break;
        case 4: upsweep_kw_kernel<RB, 4><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist, g); break;
        case 5: upsweep_kw_kernel<RB, 5><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist, g); break;
        case 6: upsweep_kw_kernel<RB, 6><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist, g); break;
        case 7: upsweep_kw_kernel<RB, 7><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist, g); break;
        case 8: upsweep_kw_kernel<RB, 8><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist, g); break;
        default: upsweep_kernel<RB><<<grid, kUpThreads, smem, s>>>(ck, n, ld, nbits, p0, np, hist, g); break;
    }
}

template <int RB>
__global__ void __launch_bounds__(256) scan_kernel(uint32_t* hist, const uint32_t* gate) {
    __shared__ uint32_t scratch[256 / 32 + 1];
    if (gated_off(gate)) return;
    block_exclusive_scan<256>(hist + (uint64_t)blockIdx.x * (1u << RB), 1 << RB, scratch);
}

// Zeroes words [0, count) unless gated off (the gated sort's workspace clear).
__global__ void gated_zero_kernel(uint32_t* p, uint64_t count, const uint32_t* gate) {
    if (gated_off(gate)) return;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = 0;
}

__global__ void iota_kernel(uint32_t* out, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)i;
}

cudaError_t launch_bucket_scan(uint32_t* hist, uint32_t sets, uint32_t rb, cudaStream_t s) {
    switch (rb) {
        case 4: scan_kernel<4><<<sets, 256, 0, s>>>(hist, nullptr); break;
        case 5: scan_kernel<5><<<sets, 256, 0, s>>>(hist, nullptr); break;
        case 6: scan_kernel<6><<<sets, 256, 0, s>>>(hist, nullptr); break;
        case 7: scan_kernel<7><<<sets, 256, 0, s>>>(hist, nullptr); break;
        case 8: scan_kernel<8><<<sets, 256, 0, s>>>(hist, nullptr); break;
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool make_sort_plan(uint64_t n, uint32_t K, uint32_t nbits, uint32_t digit_bits, SortPlan* p, uint64_t ld,
                    uint32_t tile) {
    if (digit_bits == 0) digit_bits = 8;
    if (tile == 0) tile = kPassTile;
    if (tile != 2048 && tile != kPassTile && tile != 8192) return false;
    p->ld = ld ? ld : CK_LD(n);
    if (p->ld < n) return false;
    if (digit_bits < 4 || digit_bits > 11) return false;
    p->digit_bits = digit_bits;
    p->passes = (nbits + digit_bits - 1) / digit_bits;
    p->tile = tile;
    p->tiles = (uint32_t)((n + tile - 1) / tile);
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
                               uint32_t passes, uint32_t* hist, cudaStream_t s, const uint32_t* gate = nullptr) {
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
        launch_upsweep<RB>(ck_in, n, ld, K, nbits, p0, np, hist, up_grid, s, gate);
        count_launch();
    }
    return cudaGetLastError();
}

template <int RB>
static cudaError_t run_sort_rb(const SortPlan& p, const uint32_t* ck_in, const uint32_t* rid_in, uint32_t* ck_out,
                               uint32_t* rid_out, uint64_t n, uint32_t nbits, uint32_t spin_limit, uint32_t inject,
                               uint32_t flags, cudaEvent_t* ev, unsigned char* ws, cudaStream_t s,
                               const uint32_t* hist_in, const uint32_t* gate) {
    constexpr int BINS = 1 << RB;
    uint32_t* hist = reinterpret_cast<uint32_t*>(ws + p.off_hist);
    uint32_t* counters = reinterpret_cast<uint32_t*>(ws + p.off_counter);
    uint32_t* lookback = reinterpret_cast<uint32_t*>(ws + p.off_lookback);
    uint32_t* alt_ck = reinterpret_cast<uint32_t*>(ws + p.off_alt_ck);
    uint32_t* alt_rid = reinterpret_cast<uint32_t*>(ws + p.off_alt_rid);
    const uint64_t ld = p.ld;
    cudaError_t e = cudaSuccess;
    if (gate) {
        gated_zero_kernel<<<num_sms() * 4, 256, 0, s>>>(reinterpret_cast<uint32_t*>(ws), p.off_alt_ck / 4, gate);
        count_launch();
    } else {
        e = cudaMemsetAsync(ws, 0, p.off_alt_ck, s);
        if (e != cudaSuccess) return e;
    }

    if (hist_in) {  // counted during extraction (ck_extract_hist)
        e = cudaMemcpyAsync(hist, hist_in, sizeof(uint32_t) * BINS * p.passes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    } else {
        e = upsweep_all<RB>(ck_in, n, ld, p.K, nbits, p.passes, hist, s, gate);
        if (e != cudaSuccess) return e;
    }
    scan_kernel<RB><<<p.passes, 256, 0, s>>>(hist, gate);
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
        a.gate = gate;
        a.gate_run = 1;
        e = launch_onesweep_pass(RB, a, arrays, p.tiles, s, p.tile);
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
                     uint32_t flags, cudaEvent_t* ev, unsigned char* ws, cudaStream_t s, const uint32_t* hist_in,
                     const uint32_t* gate) {
    if (gate && (p.passes == 0 || hist_in || ck_in == ck_out || (rid_in != nullptr && rid_in == rid_out)))
        return cudaErrorInvalidValue;
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
        case 4: return run_sort_rb<4>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in, gate);
        case 5: return run_sort_rb<5>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in, gate);
        case 6: return run_sort_rb<6>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in, gate);
        case 7: return run_sort_rb<7>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in, gate);
        case 8: return run_sort_rb<8>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in, gate);
        case 9: return run_sort_rb<9>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in, gate);
        case 10: return run_sort_rb<10>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in, gate);
        case 11: return run_sort_rb<11>(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin_limit, inject, flags, ev, ws, s, hist_in, gate);
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

// ck_btree.cu -- bottom-up bulk load of the index tree (Sec. 5.3) from the
// sorted (compressed key, row id) pairs, with the D-bitmap recompute of
// Sec. 4.3 (rebuild step 1) fused into the leaf pass.
//
// D-offset (Sec. 5.3): D-offset[q] = position of the (q+1)-st set bit of the
// D-bitmap used for extraction.  The full-key D-bit of two keys is
// D-offset[D-bit of their compressed keys], where the compressed D-bit counts
// from the most significant of the nbits compressed bits.
//
// Inner levels do not depend on each other: with f entries per node, entry e
// of level l covers the sorted keys [e * f^l, (e+1) * f^l), so the highest key
// under it is sorted index min((e+1) * f^l, n) - 1.  One launch therefore
// writes every inner entry of every level.
#include "ck_internal.cuh"

namespace ck {

// D-offset table in shared memory, built from the bitmap by each block.
__device__ void build_doffset(const uint64_t* mask, uint32_t key_bits, uint16_t* doff) {
    for (uint32_t p = threadIdx.x; p < key_bits; p += blockDim.x) {
        const uint64_t w = mask[p >> 6];
        const uint32_t in_word = p & 63;
        if ((w >> (63 - in_word)) & 1ull) {
            uint32_t q = 0;
            for (uint32_t i = 0; i < (p >> 6); ++i) q += __popcll(mask[i]);
            if (in_word) q += __popcll(w >> (64 - in_word));
            doff[q] = (uint16_t)p;
        }
    }
}

// Compressed D-bit of sorted rows i and j (q = 0 is the most significant of the
// nbits compressed bits); -1 if equal, -2 if a bit above nbits differs.
__device__ __forceinline__ int32_t ck_dbit(const uint32_t* ck, uint64_t ld, uint32_t K, uint32_t nbits, uint64_t i,
                                           uint64_t j) {
    for (int k = (int)K - 1; k >= 0; --k) {
        const uint32_t x = ck[(uint64_t)k * ld + i] ^ ck[(uint64_t)k * ld + j];
        if (x) {
            const uint32_t v = 32u * k + 31u - __clz(x);
            return v < nbits ? (int32_t)(nbits - 1 - v) : -2;
        }
    }
    return -1;
}

__global__ void __launch_bounds__(256) leaf_kernel(const __grid_constant__ BtreeArgs a, uint32_t* __restrict__ leaf_rid,
                                                   uint16_t* __restrict__ leaf_dbit, uint32_t* __restrict__ leaf_high,
                                                   uint64_t nodes0, uint64_t* __restrict__ refined,
                                                   unsigned long long* status) {
    __shared__ uint16_t doff[kMaxKeyBits];
    __shared__ uint32_t rmask[kMaxKeyWords];
    build_doffset(a.dmask, a.key_bits, doff);
    const uint32_t nw32 = (a.key_bits + 31) / 32;
    for (uint32_t i = threadIdx.x; i < nw32; i += blockDim.x) rmask[i] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t n = a.n;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
        const uint64_t i = i0 + lane;
        int32_t p = -1;
        if (i < n) {
            if (leaf_rid) leaf_rid[i] = a.rid[i];  // NULL: the sort wrote the tree's row ids
            if (i > 0) {
                const int32_t q = ck_dbit(a.ck, a.ld, a.K, a.nbits, i - 1, i);
                if (q >= 0) p = doff[q];
                else if (q == -2) report(status, CK_EINVAL, i);
            }
            leaf_dbit[i] = p >= 0 ? (uint16_t)p : (uint16_t)CK_NO_DBIT;
            if (i < nodes0) leaf_high[i] = (uint32_t)(min((i + 1) * (uint64_t)a.f, n) - 1);
        }
        if (refined) {
            const uint32_t peers = __match_any_sync(kFull, p);
            if (p >= 0 && (__ffs(peers) - 1) == (int)lane) atomicOr(&rmask[p >> 5], 0x80000000u >> (p & 31));
        }
    }
    if (!refined) return;
    __syncthreads();
    for (uint32_t q = threadIdx.x; 2 * q < nw32; q += blockDim.x) {
        const uint64_t hi = rmask[2 * q], lo = (2 * q + 1 < nw32) ? rmask[2 * q + 1] : 0u;
        const uint64_t v = (hi << 32) | lo;
        if (v) atomicOr(reinterpret_cast<unsigned long long*>(refined + q), (unsigned long long)v);
    }
}

// The same for keys of KW words: a thread loads its row's words once, takes
// the previous row's from the neighbouring lane (lane 0 loads them), and
// finds the D-bit from registers, so a run of equal high words costs no
// dependent loads.
template <int KW>
__global__ void __launch_bounds__(256) leaf_kw_kernel(const __grid_constant__ BtreeArgs a, uint32_t* __restrict__ leaf_rid,
                                                      uint16_t* __restrict__ leaf_dbit,
                                                      uint32_t* __restrict__ leaf_high, uint64_t nodes0,
                                                      uint64_t* __restrict__ refined, unsigned long long* status) {
    __shared__ uint16_t doff[kMaxKeyBits];
    __shared__ uint32_t rmask[kMaxKeyWords];
    build_doffset(a.dmask, a.key_bits, doff);
    const uint32_t nw32 = (a.key_bits + 31) / 32;
    for (uint32_t i = threadIdx.x; i < nw32; i += blockDim.x) rmask[i] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t n = a.n;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n; i0 += stride) {
        const uint64_t i = i0 + lane;
        uint32_t w[KW], pw[KW];
#pragma unroll
        for (int k = 0; k < KW; ++k) w[k] = i < n ? a.ck[(uint64_t)k * a.ld + i] : 0u;
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            pw[k] = __shfl_up_sync(kFull, w[k], 1);
            if (lane == 0) pw[k] = i > 0 && i < n ? a.ck[(uint64_t)k * a.ld + i - 1] : 0u;
        }
        int32_t p = -1;
        if (i < n) {
            if (leaf_rid) leaf_rid[i] = a.rid[i];  // NULL: the sort wrote the tree's row ids
            if (i > 0) {
                int32_t q = -1;  // compressed D-bit; -2: a bit above nbits differs
#pragma unroll
                for (int k = KW - 1; k >= 0; --k) {
                    const uint32_t x = w[k] ^ pw[k];
                    if (q == -1 && x) {
                        const uint32_t v = 32u * k + 31u - __clz(x);
                        q = v < a.nbits ? (int32_t)(a.nbits - 1 - v) : -2;
                    }
                }
                if (q >= 0) p = doff[q];
                else if (q == -2) report(status, CK_EINVAL, i);
            }
            leaf_dbit[i] = p >= 0 ? (uint16_t)p : (uint16_t)CK_NO_DBIT;
            if (i < nodes0) leaf_high[i] = (uint32_t)(min((i + 1) * (uint64_t)a.f, n) - 1);
        }
        if (refined) {
            const uint32_t peers = __match_any_sync(kFull, p);
            if (p >= 0 && (__ffs(peers) - 1) == (int)lane) atomicOr(&rmask[p >> 5], 0x80000000u >> (p & 31));
        }
    }
    if (!refined) return;
    __syncthreads();
    for (uint32_t q = threadIdx.x; 2 * q < nw32; q += blockDim.x) {
        const uint64_t hi = rmask[2 * q], lo = (2 * q + 1 < nw32) ? rmask[2 * q + 1] : 0u;
        const uint64_t v = (hi << 32) | lo;
        if (v) atomicOr(reinterpret_cast<unsigned long long*>(refined + q), (unsigned long long)v);
    }
}

using InnerShape = InnerLevels;

__global__ void __launch_bounds__(256) inner_kernel(const __grid_constant__ BtreeArgs a,
                                                    const __grid_constant__ InnerShape sh, uint32_t* __restrict__ child,
                                                    uint32_t* __restrict__ high, uint32_t* __restrict__ high_rid,
                                                    uint32_t* __restrict__ high_ck, uint16_t* __restrict__ dbit,
                                                    unsigned long long* status) {
    __shared__ uint16_t doff[kMaxKeyBits];
    build_doffset(a.dmask, a.key_bits, doff);
    __syncthreads();
    const uint64_t n = a.n;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < sh.inner_entries; g += stride) {
        uint32_t l = 1;
        while (l + 1 < sh.levels && g >= sh.offset[l + 1]) ++l;
        const uint64_t e = g - sh.offset[l];
        uint64_t span = 1;  // f^l, capped at n (a capped span only occurs when the level has one entry)
        for (uint32_t t = 0; t < l; ++t) span = min(span * a.f, n);
        const uint64_t hi = min((e + 1) * span, n) - 1;
        child[g] = (uint32_t)e;
        high[g] = (uint32_t)hi;
        high_rid[g] = a.rid[hi];
        for (uint32_t k = 0; k < a.K; ++k) high_ck[g * a.K + k] = a.ck[(uint64_t)k * a.ld + hi];
        int32_t p = -1;
        if (e > 0) {
            const int32_t q = ck_dbit(a.ck, a.ld, a.K, a.nbits, e * span - 1, hi);
            if (q >= 0) p = doff[q];
            else if (q == -2) report(status, CK_EINVAL, hi);
        }
        dbit[g] = p >= 0 ? (uint16_t)p : (uint16_t)CK_NO_DBIT;
    }
}

cudaError_t launch_btree(const BtreeArgs& a, const ck_btree_shape& shape, ck_btree* t, uint64_t* refined,
                         cudaStream_t s) {
    if (refined) {
        cudaError_t e = cudaMemsetAsync(refined, 0, sizeof(uint64_t) * ((a.key_bits + 63) / 64), s);
        if (e != cudaSuccess) return e;
    }
    if (a.n == 0) return cudaSuccess;
    const uint64_t cap = (uint64_t)num_sms() * 8;
    uint64_t grid = (a.n + 255) / 256;
    const unsigned g = (unsigned)(grid < cap ? grid : cap);
    // row ids sorted straight into the tree's leaf array need no copy
    uint32_t* lr = t->leaf_rid == a.rid ? nullptr : t->leaf_rid;
    uint16_t* ld = t->leaf_dbit;
    uint32_t* lh = t->leaf_high;
    const uint64_t n0 = shape.level_nodes[0];
    unsigned long long* st = status_ptr();
    switch (a.K) {
        case 1: leaf_kw_kernel<1><<<g, 256, 0, s>>>(a, lr, ld, lh, n0, refined, st); break;
        case 2: leaf_kw_kernel<2><<<g, 256, 0, s>>>(a, lr, ld, lh, n0, refined, st); break;
        case 3: leaf_kw_kernel<3><<<g, 256, 0, s>>>(a, lr, ld, lh, n0, refined, st); break;
        case 4: leaf_kw_kernel<4><<<g, 256, 0, s>>>(a, lr, ld, lh, n0, refined, st); break;
        case 5: leaf_kw_kernel<5><<<g, 256, 0, s>>>(a, lr, ld, lh, n0, refined, st); break;
        case 6: leaf_kw_kernel<6><<<g, 256, 0, s>>>(a, lr, ld, lh, n0, refined, st); break;
        case 7: leaf_kw_kernel<7><<<g, 256, 0, s>>>(a, lr, ld, lh, n0, refined, st); break;
        case 8: leaf_kw_kernel<8><<<g, 256, 0, s>>>(a, lr, ld, lh, n0, refined, st); break;
        default: leaf_kernel<<<g, 256, 0, s>>>(a, lr, ld, lh, n0, refined, st); break;
    }
    count_launch();
    if (shape.inner_entries > 0) {
        InnerShape sh;
        sh.levels = shape.levels;
        sh.inner_entries = shape.inner_entries;
        for (uint32_t l = 0; l < CK_MAX_LEVELS; ++l) sh.offset[l] = shape.inner_offset[l];
        grid = (shape.inner_entries + 255) / 256;
        inner_kernel<<<(unsigned)(grid < cap ? grid : cap), 256, 0, s>>>(a, sh, t->inner_child, t->inner_high,
                                                                        t->inner_high_rid, t->inner_high_ck,
                                                                        t->inner_dbit, status_ptr());
        count_launch();
    }
    return cudaGetLastError();
}

}  // namespace ck

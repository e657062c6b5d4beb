// ck_insert.cu -- DS-metadata under a batch of inserts (Sec. 4.3, "Search and
// Update Operations", Insert).
//
// The paper inserts a key K between its neighbours A and B and sets
// max(D-bit(A, K), D-bit(K, B)) in the D-bitmap (the smaller one is D-bit(A, B)
// by Lemma 1 and already set), and ORs K xor the reference key into the
// variant bitmap.  For a whole batch the result does not depend on the order
// of the inserts: it adds the D-bits of every adjacent pair of the merged
// sorted order (old keys and batch) that involves a batch key.  So the batch
// is sorted once (by its own varying bits, Theorem 2), and every batch key j
// finds its place among the old keys by binary search; its neighbours in the
// merged order are the larger of (old key before its place, batch key j - 1)
// and the smaller of (old key at its place, batch key j + 1).  Equal keys have
// no D-bit, so the way ties are ordered does not matter.
#include "ck_internal.cuh"

namespace ck {

namespace {

constexpr int kInsertThreads = 256;

__device__ __forceinline__ void mark(uint32_t* sm, int32_t p) {  // one shared atomic per distinct position per warp
    const uint32_t peers = __match_any_sync(kFull, p);
    if (p >= 0 && (__ffs(peers) - 1) == (int)(threadIdx.x & 31)) atomicOr(&sm[p >> 5], 0x80000000u >> (p & 31));
}

__device__ __forceinline__ void merge(const uint32_t* sm, uint32_t nwords32, uint64_t* out) {
    for (uint32_t q = threadIdx.x; 2 * q < nwords32; q += blockDim.x) {
        const uint64_t hi = sm[2 * q], lo = (2 * q + 1 < nwords32) ? sm[2 * q + 1] : 0u;
        const uint64_t v = (hi << 32) | lo;
        if (v) atomicOr(reinterpret_cast<unsigned long long*>(out + q), (unsigned long long)v);
    }
}

// One thread per batch key in sorted position j (grid-stride, warp-uniform
// trip count for the warp-wide marking).
template <int VEC, int QW>
__global__ void __launch_bounds__(kInsertThreads) insert_kernel(const __grid_constant__ KeyDesc old_k, uint64_t n,
                                                               const uint32_t* __restrict__ order,
                                                               const __grid_constant__ KeyDesc new_k, uint64_t m,
                                                               const uint32_t* __restrict__ border, uint64_t ref_row,
                                                               uint64_t* __restrict__ dmask,
                                                               uint64_t* __restrict__ vmask,
                                                               unsigned long long* status) {
    __shared__ uint32_t sd[kMaxKeyWords], sv[kMaxKeyWords];
    for (uint32_t i = threadIdx.x; i < old_k.nwords; i += blockDim.x) {
        sd[i] = 0;
        sv[i] = 0;
    }
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, nchunks = (old_k.nwords + 3) / 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t j0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); j0 < m; j0 += stride) {
        const uint64_t j = j0 + lane;
        int32_t pl = -1, pr = -1;
        if (j < m) {
            const uint32_t rb = border[j];
            const KeyRef key{&new_k, rb < m ? rb : 0};
            if (rb >= m) report(status, CK_EINVAL, j);
            const QueryView<VEC, QW> K(new_k, key.r);  // the new key, in registers when it is short
            // place among the old keys: the first sorted position whose key is >= K
            uint64_t lo = 0, hi = n;
            while (lo < hi) {
                const uint64_t mid = (lo + hi) >> 1;
                const uint32_t r = order[mid];
                if (r >= n) {  // a corrupt order entry: recorded, searched past
                    report(status, CK_EINVAL, mid);
                    lo = mid + 1;
                    continue;
                }
                int32_t dd;
                if (K.cmp(old_k, r, &dd) < 0) lo = mid + 1;
                else hi = mid;
            }
            // neighbours in the merged order
            bool has_a = false, has_b = false;
            KeyRef a{&old_k, 0}, b{&old_k, 0};
            if (lo > 0 && order[lo - 1] < n) {
                a = KeyRef{&old_k, order[lo - 1]};
                has_a = true;
            }
            if (j > 0 && border[j - 1] < m) {
                const KeyRef prev{&new_k, border[j - 1]};
                if (!has_a || cmp_keys<VEC>(prev, a) > 0) a = prev;
                has_a = true;
            }
            if (lo < n && order[lo] < n) {
                b = KeyRef{&old_k, order[lo]};
                has_b = true;
            }
            if (j + 1 < m && border[j + 1] < m) {
                const KeyRef next{&new_k, border[j + 1]};
                if (!has_b || cmp_keys<VEC>(next, b) < 0) b = next;
                has_b = true;
            }
            if (has_a) K.cmp(*a.k, a.r, &pl);  // the D-bit of the two keys (-1 if equal)
            if (has_b) K.cmp(*b.k, b.r, &pr);
        }
        mark(sd, pl);
        mark(sd, pr);
        // variant bitmap: K xor the reference key
        for (uint32_t c = 0; c < nchunks; ++c) {
            uint32_t w[4] = {0, 0, 0, 0}, ref[4];
            load_chunk<VEC>(old_k, ref_row, c, ref);
            if (j < m && border[j] < m) load_chunk<VEC>(new_k, border[j], c, w);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t x = __reduce_or_sync(kFull, j < m ? (w[i] ^ ref[i]) : 0u);
                if (lane == 0 && x && 4 * c + i < old_k.nwords) atomicOr(&sv[4 * c + i], x);
            }
        }
    }
    __syncthreads();
    merge(sd, old_k.nwords, dmask);
    merge(sv, old_k.nwords, vmask);
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct InsertPlan {
    uint32_t K;  // words of the batch's sort key (upper bound for the workspace)
    size_t off_ck, off_ck_sorted, off_rid, off_sort_ws, total;
};

bool make_insert_plan(uint64_t m, uint32_t key_bytes, InsertPlan* p) {
    const uint32_t nwords = (key_bytes + 3) / 4;
    p->K = nwords;
    size_t off = 0;
    p->off_ck = off;
    off = a256(off + 4ull * nwords * CK_LD(m));
    p->off_ck_sorted = off;
    off = a256(off + 4ull * nwords * CK_LD(m));
    p->off_rid = off;
    off = a256(off + 4ull * m);
    p->off_sort_ws = off;
    const size_t sws = ck_sort_workspace_bytes(m, nwords, 32 * nwords, nullptr);
    if (sws == 0 && m > 1) return false;
    off = a256(off + sws);
    p->total = off;
    return true;
}

}  // namespace
}  // namespace ck

using namespace ck;

extern "C" {

size_t ck_insert_workspace_bytes(uint64_t m, uint32_t key_bytes) {
    InsertPlan p;
    if (key_bytes == 0 || key_bytes > CK_MAX_KEY_BYTES || m > CK_MAX_ROWS || !make_insert_plan(m, key_bytes, &p))
        return 0;
    return p.total;
}

ck_status ck_insert_batch(const ck_column* keys, const uint32_t* order, const ck_column* batch, uint64_t ref_row,
                          uint64_t* dmask, uint64_t* vmask, void* ws_v, size_t ws_bytes, ck_stream stream) {
    KeyDesc ok, nk;
    int vo = 1, vn = 1;
    if (!make_key_desc(keys, &ok, &vo) || !make_key_desc(batch, &nk, &vn)) return CK_EINVAL;
    if (keys->key_bytes != batch->key_bytes || keys->kind != batch->kind) return CK_EINVAL;
    if (!dmask || !vmask) return CK_EINVAL;
    const uint64_t n = keys->n, m = batch->n;
    if (m == 0) return CK_OK;
    if (n == 0 || !order || ref_row >= n) return CK_EINVAL;
    InsertPlan P;
    if (!make_insert_plan(m, keys->key_bytes, &P)) return CK_EINVAL;
    if (!ws_v || ws_bytes < P.total || (reinterpret_cast<uintptr_t>(ws_v) & 255)) return CK_ENOMEM;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(ws_v);
    auto at = [&](size_t off) { return reinterpret_cast<uint32_t*>(ws + off); };
    uint32_t* border = at(P.off_rid);

    // 1. the batch's sorted order by its full keys: any superset of the
    //    batch's D-bitmap orders it (Theorem 2), and the all-ones bitmap is
    //    known here without reading the device, so the call never waits for
    //    the GPU (a batch is small: the extra passes cost little)
    const uint32_t key_bits = 8u * keys->key_bytes, mw = (key_bits + 63) / 64;
    static thread_local uint64_t full_mask[(8 * CK_MAX_KEY_BYTES + 63) / 64];
    for (uint32_t w = 0; w < mw; ++w)
        full_mask[w] = (w + 1 < mw || key_bits % 64 == 0) ? ~0ull : ~0ull << (64 - key_bits % 64);
    ck_status st = ck_extract(batch, full_mask, P.K, at(P.off_ck), stream);
    if (st != CK_OK) return st;
    st = ck_sort(at(P.off_ck), nullptr, at(P.off_ck_sorted), border, m, P.K, key_bits, nullptr, ws + P.off_sort_ws,
                 ws_bytes - P.off_sort_ws, stream);
    if (st != CK_OK) return st;

    // 2. every batch key's neighbours in the merged order: D-bits and variant bits
    unsigned long long* status = status_ptr();
    if (!status) return CK_ECUDA;
    const int vec = vo < vn ? vo : vn;
    const uint64_t want = (m + kInsertThreads - 1) / kInsertThreads, cap = (uint64_t)num_sms() * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    const uint32_t nw = nk.nwords;
    const int qw = nw <= 2 ? 2 : nw <= 4 ? 4 : nw <= 8 ? 8 : 0;  // the new key's words kept in registers
#define CK_INSERT_LAUNCH(V, Q) \
    insert_kernel<V, Q><<<grid, kInsertThreads, 0, s>>>(ok, n, order, nk, m, border, ref_row, dmask, vmask, status)
#define CK_INSERT_QW(V)                          \
    switch (qw) {                                \
        case 2: CK_INSERT_LAUNCH(V, 2); break;   \
        case 4: CK_INSERT_LAUNCH(V, 4); break;   \
        case 8: CK_INSERT_LAUNCH(V, 8); break;   \
        default: CK_INSERT_LAUNCH(V, 0); break;  \
    }
    switch (vec) {
        case 16: CK_INSERT_QW(16) break;
        case 8: CK_INSERT_QW(8) break;
        case 4: CK_INSERT_QW(4) break;
        default: CK_INSERT_QW(1) break;
    }
#undef CK_INSERT_QW
#undef CK_INSERT_LAUNCH
    count_launch();
    return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

}  // extern "C"

// ck_learned.cu -- the learned-partition sort (not in the paper): a tiny fp32
// CDF model, trained on the GPU on a sample of the compressed keys, places
// every key in one of about B = 2^bucket_bits key-range buckets; two radix
// passes on the bucket id partition the pairs stably, and each bucket is then
// sorted in shared memory.  The result is the same permutation as the plain
// radix sort:
//
//  * the buckets are ranges between monotone splitters (the B-quantiles of the
//    sorted sample moved to the nearer end of their run of equal keys, with
//    heavy keys isolated in buckets of their own), so a stable partition by
//    bucket followed by a stable sort inside each bucket is a stable sort of
//    the whole column;
//  * the model proposes each key's bucket as floor(y(x) * B) in O(1); a short
//    walk against the splitters makes the assignment exact (a far-off guess
//    falls back to binary search), so a poor model costs time, not
//    correctness.  Without the model every key needs a binary search;
//  * a bucket is sorted by the 32-bit window at its first varying bit, and
//    ties are settled below the window; a non-constant bucket too large for a
//    block is sorted by the plain radix sort on its segment;
//  * a verification pass checks every adjacent output pair; if it fails, the
//    plain radix sort recomputes the result from the untouched input (status
//    CK_EVERIFY).
//
// The model: y(x) = b2 + sum_j w2_j relu(w1_j x + b1_j), 16 hidden units, on
// x = the top 24 bits of the compressed key / 2^24, fitted by full-batch Adam
// to the empirical CDF (rank + 0.5) / S of the sorted sample.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ck_internal.cuh"

namespace ck {

constexpr int kHidden = CK_MLP_HIDDEN;
constexpr int kParams = CK_MLP_PARAMS;  // [w1(16), b1(16), w2(16), b2]
constexpr int kRed = kParams + 1;       // gradient + loss
constexpr int kTrainThreads = 256;
constexpr int kMaxLearnedWords = 8;
constexpr uint64_t kMaxTrainPoints = 65536;  // training uses a stride subsample of the sorted sample

__device__ __forceinline__ float mlp_eval(const float* p, float x) {
    float y = p[3 * kHidden];
#pragma unroll
    for (int j = 0; j < kHidden; ++j) {
        const float z = fmaf(p[j], x, p[kHidden + j]);
        y = fmaf(p[2 * kHidden + j], fmaxf(z, 0.0f), y);
    }
    return y;
}

// Adds the gradient of (y(x) - t)^2 * scale to g[0..48] and returns the squared residual.
__device__ __forceinline__ float mlp_accumulate(const float* p, float x, float t, float scale, float* g) {
    float z[kHidden];
    float y = p[3 * kHidden];
#pragma unroll
    for (int j = 0; j < kHidden; ++j) {
        z[j] = fmaf(p[j], x, p[kHidden + j]);
        y = fmaf(p[2 * kHidden + j], fmaxf(z[j], 0.0f), y);
    }
    const float r = y - t;
    const float dy = 2.0f * r * scale;
    g[3 * kHidden] += dy;
#pragma unroll
    for (int j = 0; j < kHidden; ++j) {
        if (z[j] > 0.0f) {
            g[2 * kHidden + j] += dy * z[j];
            const float dz = dy * p[2 * kHidden + j];
            g[j] += dz * x;
            g[kHidden + j] += dz;
        }
    }
    return r * r;
}

// Top 24 bits of an nbits-bit compressed key (word-major, leading dimension
// ld) as a float in [0, 1); exact in fp32.
__device__ __forceinline__ float key_feature(const uint32_t* ck, uint64_t ld, uint64_t i, uint32_t K,
                                             uint32_t nbits) {
    uint32_t top;
    if (nbits >= 24) {
        const uint32_t lo = nbits - 24, w = lo >> 5, s = lo & 31;
        uint64_t v = ck[(uint64_t)w * ld + i];
        if (w + 1 < K) v |= (uint64_t)ck[(uint64_t)(w + 1) * ld + i] << 32;
        top = (uint32_t)(v >> s) & 0xFFFFFFu;
    } else {
        top = (ck[i] << (24 - nbits)) & 0xFFFFFFu;
    }
    return (float)top * (1.0f / 16777216.0f);
}

// Deterministic block reduction of kRed per-thread values: warp butterflies,
// then the warps' results summed in warp order.  Result in out[0..kRed).
__device__ void block_reduce_red(float (&v)[kRed], float* sm /*[warps][kRed]*/, float* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < kRed; ++k) {
        float x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (lane == 0) sm[warp * kRed + k] = x;
    }
    __syncthreads();
    if (threadIdx.x < kRed) {
        float s = 0.0f;
        for (int w = 0; w < warps; ++w) s += sm[w * kRed + threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// ------------------------------------------------------------ sample, features
__global__ void sample_kernel(const uint32_t* __restrict__ ck, uint64_t ld, uint32_t K, uint64_t div, uint64_t S,
                              uint32_t* __restrict__ out, uint64_t ld_s) {
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < S; j += (uint64_t)gridDim.x * blockDim.x)
        for (uint32_t w = 0; w < K; ++w) out[(uint64_t)w * ld_s + j] = ck[(uint64_t)w * ld + j * div];
}

__global__ void features_kernel(const uint32_t* __restrict__ ck, uint64_t ld, uint64_t S, uint32_t K, uint32_t nbits,
                                float* __restrict__ xs) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += (uint64_t)gridDim.x * blockDim.x)
        xs[i] = key_feature(ck, ld, i, K, nbits);
}

// Initial parameters: the linear spline through the sample CDF at 16 knots
// (sample quantiles j / 16).  Hidden unit j is relu(x - k_j); its output weight
// is the change of slope at k_j.  One warp.
__global__ void mlp_init_kernel(const float* __restrict__ xs, uint64_t S, float* __restrict__ params) {
    __shared__ float k[kHidden + 1], y[kHidden + 1];
    const int j = threadIdx.x;
    if (j <= kHidden) {
        const uint64_t idx = j < kHidden ? (uint64_t)j * S / kHidden : S - 1;
        k[j] = xs[idx];
        y[j] = j < kHidden ? ((float)idx + 0.5f) / (float)S : 1.0f;
    }
    __syncwarp();
    if (j < kHidden) {
        auto slope = [&](int q) {
            const float dx = k[q + 1] - k[q];
            return dx > 1e-7f ? (y[q + 1] - y[q]) / dx : 0.0f;
        };
        const float sj = slope(j), sp = j > 0 ? slope(j - 1) : 0.0f;
        params[j] = 1.0f;
        params[kHidden + j] = -k[j];
        params[2 * kHidden + j] = sj - sp;
    }
    if (j == 0) params[3 * kHidden] = y[0];
}

// ------------------------------------------------------------ fwd + bwd
// Loss and gradient of the model over S samples (targets (i + 0.5) / S when
// t == NULL), one launch: per-block partials in partial[block][kRed].
__global__ void __launch_bounds__(kTrainThreads) mlp_grad_kernel(const float* __restrict__ params,
                                                                  const float* __restrict__ xs,
                                                                  const float* __restrict__ ts, uint64_t S,
                                                                  float* __restrict__ partial) {
    __shared__ float p[kParams];
    __shared__ float red[(kTrainThreads / 32) * kRed];
    __shared__ float out[kRed];
    if (threadIdx.x < kParams) p[threadIdx.x] = params[threadIdx.x];
    __syncthreads();
    float g[kRed];
#pragma unroll
    for (int q = 0; q < kRed; ++q) g[q] = 0.0f;
    const float scale = 1.0f / (float)S;
    const uint64_t i0 = S * blockIdx.x / gridDim.x, i1 = S * (blockIdx.x + 1) / gridDim.x;
    for (uint64_t i = i0 + threadIdx.x; i < i1; i += kTrainThreads) {
        const float t = ts ? ts[i] : ((float)i + 0.5f) * scale;
        g[kParams] += mlp_accumulate(p, xs[i], t, scale, g);
    }
    block_reduce_red(g, red, out);
    if (threadIdx.x < kRed) partial[(uint64_t)blockIdx.x * kRed + threadIdx.x] = out[threadIdx.x];
}

// Fixed-order sum of the per-block partials: grad[0..48], loss = sum r^2 / S.
__global__ void mlp_grad_sum_kernel(const float* __restrict__ partial, uint32_t blocks, uint64_t S,
                                    float* __restrict__ grad, float* __restrict__ loss) {
    const int k = threadIdx.x;
    if (k >= kRed) return;
    float s = 0.0f;
    for (uint32_t b = 0; b < blocks; ++b) s += partial[(uint64_t)b * kRed + k];
    if (k < kParams) grad[k] = s;
    else if (loss) *loss = s / (float)S;
}

// ------------------------------------------------------------ training
struct TrainArgs {
    const float* xs;      // features of the sorted sample, [S]
    uint64_t S;           // sample size (targets (i + 0.5) / S)
    uint64_t T, stride;   // training points: sample indices 0, stride, ..., (T - 1) * stride
    float* params;        // in: initial parameters, out: trained
    float* partial;       // [2][gridDim][kRed]
    unsigned* barrier;    // zeroed
    float* loss;          // out: loss of the last epoch
    uint32_t epochs;
    float lr;
    uint32_t spin_limit;
    unsigned long long* status;
};

__device__ __forceinline__ uint32_t ld_acquire(const unsigned* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// All blocks of the (cooperatively launched, hence co-resident) grid arrive;
// the wait is bounded and reports CK_ETIMEOUT instead of hanging.
__device__ void grid_barrier(unsigned* ctr, unsigned target, uint32_t limit, unsigned long long* status) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        uint32_t polls = 0;
        while (ld_acquire(ctr) < target) {
            if (++polls > limit) {
                report(status, CK_ETIMEOUT, (1ull << 46) | target);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
}

// Full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8).  Every block keeps the
// parameters and the moments in shared memory and applies the same update to
// the same fixed-order gradient sum, so all copies stay identical.
__global__ void __launch_bounds__(kTrainThreads) mlp_train_kernel(const TrainArgs a) {
    __shared__ float p[kParams], m1[kParams], m2[kParams];
    __shared__ float red[(kTrainThreads / 32) * kRed];
    __shared__ float out[kRed];
    const int tid = threadIdx.x;
    if (tid < kParams) {
        p[tid] = a.params[tid];
        m1[tid] = 0.0f;
        m2[tid] = 0.0f;
    }
    __syncthreads();
    const float scale = 1.0f / (float)a.T, tscale = 1.0f / (float)a.S;
    const uint64_t i0 = a.T * blockIdx.x / gridDim.x, i1 = a.T * (blockIdx.x + 1) / gridDim.x;
    float b1t = 1.0f, b2t = 1.0f, last_loss = 0.0f;
    for (uint32_t ep = 0; ep < a.epochs; ++ep) {
        float g[kRed];
#pragma unroll
        for (int q = 0; q < kRed; ++q) g[q] = 0.0f;
        for (uint64_t i = i0 + tid; i < i1; i += kTrainThreads) {
            const uint64_t si = i * a.stride;
            g[kParams] += mlp_accumulate(p, a.xs[si], ((float)si + 0.5f) * tscale, scale, g);
        }
        block_reduce_red(g, red, out);
        float* part = a.partial + (uint64_t)(ep & 1) * gridDim.x * kRed;
        if (tid < kRed) part[(uint64_t)blockIdx.x * kRed + tid] = out[tid];
        grid_barrier(a.barrier, (ep + 1) * gridDim.x, a.spin_limit, a.status);
        b1t *= 0.9f;
        b2t *= 0.999f;
        if (tid < kRed) {
            float s = 0.0f;
            for (uint32_t b = 0; b < gridDim.x; ++b) s += __ldcg(&part[(uint64_t)b * kRed + tid]);
            if (tid < kParams) {
                m1[tid] = 0.9f * m1[tid] + 0.1f * s;
                m2[tid] = 0.999f * m2[tid] + 0.001f * s * s;
                const float mh = m1[tid] / (1.0f - b1t), vh = m2[tid] / (1.0f - b2t);
                p[tid] -= a.lr * mh / (sqrtf(vh) + 1e-8f);
            } else {
                last_loss = s * scale;
            }
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        if (tid < kParams) a.params[tid] = p[tid];
        if (tid == kParams && a.loss) *a.loss = last_loss;
    }
}


// ------------------------------------------------------------ splitters
// Multi-word comparison of key a (K words, entry-major or registers) with b.
__device__ __forceinline__ int cmp_words(const uint32_t* a, const uint32_t* b, uint32_t K) {
    for (int w = (int)K - 1; w >= 0; --w)
        if (a[w] != b[w]) return a[w] < b[w] ? -1 : 1;
    return 0;
}

// Is the K-word key v the largest nbits-bit key (no v + 1)?
__device__ __forceinline__ bool is_max_key(const uint32_t* v, uint32_t K, uint32_t nbits) {
    for (uint32_t w = 0; w < K; ++w) {
        const uint32_t bits = min(32u, nbits > 32 * w ? nbits - 32 * w : 0u);
        const uint32_t full = bits == 32 ? 0xFFFFFFFFu : ((1u << bits) - 1u);
        if (v[w] != full) return false;
    }
    return true;
}

// Splitters from the sorted sample.  Quantile b (1 <= b < B) sits at sample
// position q_b = floor(b S / B) with value v.  The sample holds v at [i0, i1);
// moving the bucket boundary off the quantile to the nearer end of that run
// (splitter v puts the boundary at i0, v + 1 at i1) keeps every copy of v in
// one bucket and moves the boundary by at most half the run.  A value with at
// least `heavy` sample copies gets a bucket of its own, [v, v + 1) (splitters
// v and v + 1 at its first quantile); later quantiles inside the same run
// repeat the run's last splitter (empty buckets).  codes[b - 1]: bits 0-1 =
// choice with heavy buckets, bits 2-3 = choice without (1: v, 2: v + 1,
// 3: v and v + 1).
__global__ void quantile_kernel(const uint32_t* __restrict__ sample, uint64_t ld_s, uint64_t S, uint32_t K,
                                uint32_t B, uint32_t nbits, uint64_t heavy, uint8_t* __restrict__ codes) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x + 1; b < B; b += gridDim.x * blockDim.x) {
        uint64_t q = (uint64_t)b * S / B;
        if (q >= S) q = S - 1;
        uint32_t v[kMaxLearnedWords];
        for (uint32_t w = 0; w < K; ++w) v[w] = sample[(uint64_t)w * ld_s + q];
        auto cmp_at = [&](uint64_t i) {  // sample[i] vs v
            for (int w = (int)K - 1; w >= 0; --w) {
                const uint32_t x = sample[(uint64_t)w * ld_s + i];
                if (x != v[w]) return x < v[w] ? -1 : 1;
            }
            return 0;
        };
        uint64_t lo = 0, hi = q;  // i0: first position with sample >= v
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (cmp_at(mid) < 0) lo = mid + 1;
            else hi = mid;
        }
        const uint64_t i0 = lo;
        lo = q + 1;
        hi = S;  // i1: first position with sample > v
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (cmp_at(mid) <= 0) lo = mid + 1;
            else hi = mid;
        }
        const uint64_t i1 = lo;
        // the first quantile inside the run decides for all of them
        uint64_t bf = (i0 * B + S - 1) / S;  // smallest b' with floor(b' S / B) >= i0
        if (bf < 1) bf = 1;
        uint64_t qf = bf * S / B;
        if (qf >= S) qf = S - 1;
        const bool top = is_max_key(v, K, nbits);
        const bool up = !top && (i1 - qf) < (qf - i0);
        const bool is_heavy = !top && i1 - i0 >= heavy;
        const uint32_t single = up ? 2u : 1u;
        const uint32_t with_heavy = is_heavy ? (bf == b ? 3u : 2u) : single;
        codes[b - 1] = (uint8_t)(with_heavy | (single << 2));
    }
}

// Writes the splitters in order (one block): with heavy buckets when all of
// them fit max_buckets, else without.  nsplit[0] = number of splitters (the
// buckets are [spl[b - 1], spl[b]), b = 0 .. nsplit, open at both ends).
__global__ void __launch_bounds__(1024) emit_splitters_kernel(const uint32_t* __restrict__ sample, uint64_t ld_s,
                                                              uint64_t S, uint32_t K, uint32_t B,
                                                              uint32_t max_buckets,
                                                              const uint8_t* __restrict__ codes,
                                                              uint32_t* __restrict__ spl, uint32_t* nsplit) {
    __shared__ uint32_t part[1024];
    __shared__ uint32_t s_heavy;
    const uint32_t tid = threadIdx.x, nq = B - 1;
    const uint32_t per = (nq + 1023) / 1024, lo = tid * per, hi = min(nq, lo + per);
    if (tid == 0) s_heavy = 0;
    __syncthreads();
    uint32_t extra = 0;
    for (uint32_t c = lo; c < hi; ++c) extra += (codes[c] & 3u) == 3u ? 1u : 0u;
    if (extra) atomicAdd(&s_heavy, extra);
    __syncthreads();
    const uint32_t shift = nq + s_heavy + 1 <= max_buckets ? 0u : 2u;
    uint32_t cnt = 0;
    for (uint32_t c = lo; c < hi; ++c) cnt += ((codes[c] >> shift) & 3u) == 3u ? 2u : 1u;
    part[tid] = cnt;
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (int t = 0; t < 1024; ++t) {
            const uint32_t x = part[t];
            part[t] = run;
            run += x;
        }
        *nsplit = run;
    }
    __syncthreads();
    uint32_t at = part[tid];
    for (uint32_t c = lo; c < hi; ++c) {
        const uint32_t code = (codes[c] >> shift) & 3u;
        uint64_t q = (uint64_t)(c + 1) * S / B;
        if (q >= S) q = S - 1;
        if (code & 1u) {  // v
            for (uint32_t w = 0; w < K; ++w) spl[(uint64_t)at * K + w] = sample[(uint64_t)w * ld_s + q];
            ++at;
        }
        if (code & 2u) {  // v + 1
            uint32_t carry = 1;
            for (uint32_t w = 0; w < K; ++w) {
                const uint64_t sum = (uint64_t)sample[(uint64_t)w * ld_s + q] + carry;
                spl[(uint64_t)at * K + w] = (uint32_t)sum;
                carry = (uint32_t)(sum >> 32);
            }
            ++at;
        }
    }
}

// ------------------------------------------------------------ bucket ids
struct BucketArgs {
    const uint32_t* ck;
    uint64_t ld, n;
    uint32_t K, nbits, max_buckets, use_model;
    const uint32_t* nsplit;  // number of splitters (buckets - 1), on the device
    const uint32_t* spl;     // [nsplit * K], entry-major, non-decreasing
    const float* params;
    const float* loss;    // training loss (mean squared CDF error) of params
    uint32_t* bkt;        // [n]
    uint32_t* hist;       // [2][256] digit histograms of the bucket id (low byte, high bits)
    unsigned long long* steps;  // [0]: total search steps, [1]: max
};

// Compile-time-width helpers for the bucket kernel (key in registers; word
// indices are resolved by unrolled selects so the key never leaves registers).
template <int KW>
__device__ __forceinline__ int cmp_key(const uint32_t (&key)[KW], const uint32_t* s) {
#pragma unroll
    for (int w = KW - 1; w >= 0; --w)
        if (key[w] != s[w]) return key[w] < s[w] ? -1 : 1;
    return 0;
}

// The top 32 bits of an nbits-bit key, left-aligned (zero-filled below a
// shorter key).  Keys compare as their top32 values first.
template <int KW>
__device__ __forceinline__ uint32_t top32_regs(const uint32_t (&key)[KW], uint32_t nbits) {
    if (nbits < 32) return key[0] << (32 - nbits);
    const uint32_t lo = nbits - 32, w = lo >> 5, sh = lo & 31;
    uint32_t a = 0, b = 0;
#pragma unroll
    for (int j = 0; j < KW; ++j) {
        if ((uint32_t)j == w) a = key[j];
        if ((uint32_t)j == w + 1) b = key[j];
    }
    return sh ? __funnelshift_r(a, b, sh) : a;
}

__device__ __forceinline__ uint32_t top32_mem(const uint32_t* key, uint32_t K, uint32_t nbits) {
    if (nbits < 32) return key[0] << (32 - nbits);
    const uint32_t lo = nbits - 32, w = lo >> 5, sh = lo & 31;
    return sh ? __funnelshift_r(key[w], key[w + 1 < K ? w + 1 : w], sh) : key[w];
}

// Comparison of key x (top32 value t) with splitter m: the shared table of
// splitter top32 values decides unless they are equal, then the full
// splitter is read.
template <int KW, bool STAGED>
__device__ __forceinline__ int cmp_at(const uint32_t (&key)[KW], uint32_t t, const uint32_t* top,
                                      const uint32_t* spl, uint32_t m) {
    if (STAGED) {
        const uint32_t u = top[m];
        if (t != u) return t < u ? -1 : 1;
    }
    return cmp_key<KW>(key, spl + (uint64_t)m * KW);
}

// Number of splitters <= x within [lo, hi] (binary search).
template <int KW, bool STAGED>
__device__ __forceinline__ uint32_t search_range(const uint32_t (&key)[KW], uint32_t t, const uint32_t* top,
                                                 const uint32_t* spl, uint32_t lo, uint32_t hi, uint32_t* cmp) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        ++*cmp;
        if (cmp_at<KW, STAGED>(key, t, top, spl, mid) >= 0) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Exact bucket from a guess g in [lo, hi] (the key's bucket is known to lie
// there): check the guess's range, then gallop away from it (1, 2, 4, ...
// buckets) and finish with a binary search, so a guess that is e buckets off
// costs about 2 log2(e) + 2 comparisons.
template <int KW, bool STAGED>
__device__ __forceinline__ uint32_t search_from_guess(const uint32_t (&key)[KW], uint32_t t, const uint32_t* top,
                                                      const uint32_t* spl, uint32_t lo, uint32_t hi, uint32_t g,
                                                      uint32_t* cmp) {
    ++*cmp;
    if (g > lo && cmp_at<KW, STAGED>(key, t, top, spl, g - 1) < 0) {  // below: gallop down
        uint32_t h = g - 1, step = 1;
        while (true) {
            const uint32_t probe = h >= lo + step ? h - step : lo;
            ++*cmp;
            if (cmp_at<KW, STAGED>(key, t, top, spl, probe) >= 0)
                return search_range<KW, STAGED>(key, t, top, spl, probe + 1, h, cmp);
            if (probe == lo) return lo;
            h = probe;
            step <<= 1;
        }
    }
    ++*cmp;
    if (g < hi && cmp_at<KW, STAGED>(key, t, top, spl, g) >= 0) {  // above: gallop up
        uint32_t l = g + 1, step = 1;
        while (true) {
            const uint32_t probe = l + step - 1 < hi ? l + step - 1 : hi - 1;
            ++*cmp;
            if (cmp_at<KW, STAGED>(key, t, top, spl, probe) < 0)
                return search_range<KW, STAGED>(key, t, top, spl, l, probe, cmp);
            l = probe + 1;
            if (probe == hi - 1) return hi;
            step <<= 1;
        }
    }
    return g;
}

// Bucket id of every key (B = splitters + 1 buckets).  With STAGED, the top32
// value of every splitter sits in shared memory, with a table over its top
// kPrefixBits bits: pre[p] = first splitter whose top32 is >= p << (32 -
// kPrefixBits).  A key whose top32 has prefix p has its bucket in [pre[p],
// pre[p + 1]].  The model's guess, clamped into the range, starts a galloping
// search where that is expected to be cheaper than a binary search of the
// range: its error is about e = sqrt(loss) B buckets, so galloping costs about
// 2 log2(e + 1) + 2 comparisons against log2(range + 1).  Without STAGED the
// range is all buckets.
constexpr int kPrefixBits = 12;

template <int KW, bool STAGED>
__global__ void __launch_bounds__(1024) bucket_kernel(const BucketArgs a) {
    extern __shared__ uint32_t top[];
    uint32_t* pre = top + (a.max_buckets - 1);  // [2^kPrefixBits + 1] when staged
    __shared__ float p[kParams];
    __shared__ uint32_t hlo[256], hhi[256];
    __shared__ unsigned long long s_sum, s_max;
    const int tid = threadIdx.x;
    const uint32_t B = min(*a.nsplit + 1, a.max_buckets), nbits = a.nbits;
    const float err = a.use_model ? sqrtf(fmaxf(*a.loss, 0.0f)) * (float)B + 1.0f : 0.0f;
    const float model_min_range = 4.0f * err * err;  // use the model on ranges wider than this
    if (tid < kParams) p[tid] = a.params ? a.params[tid] : 0.0f;
    if (tid < 256) {
        hlo[tid] = 0;
        hhi[tid] = 0;
    }
    if (tid == 0) {
        s_sum = 0;
        s_max = 0;
    }
    if (STAGED) {
        for (uint32_t m = tid; m + 1 < B; m += blockDim.x) top[m] = top32_mem(a.spl + (uint64_t)m * KW, KW, nbits);
        __syncthreads();
        for (uint32_t q = tid; q <= (1u << kPrefixBits); q += blockDim.x) {
            uint32_t lo = 0, hi = B - 1;  // first m with top[m] >= q << (32 - kPrefixBits)
            const uint64_t bound = (uint64_t)q << (32 - kPrefixBits);
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if ((uint64_t)top[mid] >= bound) hi = mid;
                else lo = mid + 1;
            }
            pre[q] = lo;
        }
    }
    __syncthreads();
    unsigned long long my_sum = 0, my_max = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t next[KW];  // the following key's words, loaded while this key is searched
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + tid;
#pragma unroll
    for (int w = 0; w < KW; ++w) next[w] = i < a.n ? a.ck[(uint64_t)w * a.ld + i] : 0u;
    for (; i < a.n; i += stride) {
        uint32_t key[KW];
#pragma unroll
        for (int w = 0; w < KW; ++w) {
            key[w] = next[w];
            next[w] = i + stride < a.n ? a.ck[(uint64_t)w * a.ld + i + stride] : 0u;
        }
        const uint32_t t = top32_regs<KW>(key, nbits);
        uint32_t g, steps = 0, lo = 0, hi = B - 1;
        if (STAGED) {
            const uint32_t q = t >> (32 - kPrefixBits);
            lo = pre[q];
            hi = pre[q + 1];
        }
        if (a.use_model && (float)(hi - lo) + 1.0f > model_min_range) {
            const float x = (float)(t >> 8) * (1.0f / 16777216.0f);  // the top 24 bits, as in training
            const float y = mlp_eval(p, x) * (float)B;
            uint32_t guess = y <= 0.0f ? 0u : (y >= (float)(B - 1) ? B - 1 : (uint32_t)y);
            guess = guess < lo ? lo : (guess > hi ? hi : guess);
            g = search_from_guess<KW, STAGED>(key, t, top, a.spl, lo, hi, guess, &steps);
        } else {
            g = search_range<KW, STAGED>(key, t, top, a.spl, lo, hi, &steps);
        }
        a.bkt[i] = g;
        atomicAdd(&hlo[g & 255u], 1u);
        atomicAdd(&hhi[g >> 8], 1u);
        my_sum += steps;
        my_max = my_max > steps ? my_max : steps;
    }
    atomicAdd(&s_sum, my_sum);
    atomicMax(&s_max, my_max);
    __syncthreads();
    if (tid < 256) {
        if (hlo[tid]) atomicAdd(&a.hist[tid], hlo[tid]);
        if (hhi[tid]) atomicAdd(&a.hist[256 + tid], hhi[tid]);
    }
    if (tid == 0) {
        atomicAdd(&a.steps[0], s_sum);
        atomicMax(&a.steps[1], s_max);
    }
}

template <int KW>
static cudaError_t launch_bucket_kw(const BucketArgs& ba, bool staged, size_t smem, int sms, cudaStream_t s) {
    if (staged) {
        cudaError_t e = cudaFuncSetAttribute(bucket_kernel<KW, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        bucket_kernel<KW, true><<<sms, 1024, smem, s>>>(ba);
    } else {
        bucket_kernel<KW, false><<<sms, 1024, 0, s>>>(ba);
    }
    return cudaGetLastError();
}

static cudaError_t launch_bucket(const BucketArgs& ba, bool staged, size_t smem, int sms, cudaStream_t s) {
    switch (ba.K) {
        case 1: return launch_bucket_kw<1>(ba, staged, smem, sms, s);
        case 2: return launch_bucket_kw<2>(ba, staged, smem, sms, s);
        case 3: return launch_bucket_kw<3>(ba, staged, smem, sms, s);
        case 4: return launch_bucket_kw<4>(ba, staged, smem, sms, s);
        case 5: return launch_bucket_kw<5>(ba, staged, smem, sms, s);
        case 6: return launch_bucket_kw<6>(ba, staged, smem, sms, s);
        case 7: return launch_bucket_kw<7>(ba, staged, smem, sms, s);
        default: return launch_bucket_kw<8>(ba, staged, smem, sms, s);
    }
}

// ------------------------------------------------------------ bucket sorts
// start[b] = first position of bucket b in the partitioned keys: the first
// position whose key is >= spl[b - 1].  The partition is by key range, so
// that predicate is monotone in the position and a binary search finds it.
// start[0] = 0; buckets past the last splitter are empty (start = n).
__global__ void bucket_bounds_kernel(const uint32_t* __restrict__ ck, uint64_t ld, uint64_t n, uint32_t K,
                                     const uint32_t* __restrict__ spl, const uint32_t* nsplit, uint32_t max_buckets,
                                     uint32_t* __restrict__ start) {
    const uint32_t ns = min(*nsplit, max_buckets - 1);
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= max_buckets; b += gridDim.x * blockDim.x) {
        uint64_t pos = b == 0 ? 0 : n;
        if (b >= 1 && b <= ns) {
            const uint32_t* v = spl + (uint64_t)(b - 1) * K;
            uint64_t lo = 0, hi = n;
            while (lo < hi) {
                const uint64_t mid = (lo + hi) >> 1;
                int c = 0;
                for (int w = (int)K - 1; w >= 0 && c == 0; --w) {
                    const uint32_t x = ck[(uint64_t)w * ld + mid];
                    c = x < v[w] ? -1 : (x > v[w] ? 1 : 0);
                }
                if (c < 0) lo = mid + 1;
                else hi = mid;
            }
            pos = lo;
        }
        start[b] = (uint32_t)pos;
    }
}

// Bucket b holds only equal keys when its range is [v, v + 1).
__device__ bool constant_bucket(const uint32_t* spl, uint32_t K, uint32_t B, uint32_t b) {
    if (b == 0 || b + 1 >= B) return false;
    const uint32_t* lo = spl + (uint64_t)(b - 1) * K;
    const uint32_t* hi = spl + (uint64_t)b * K;
    uint32_t carry = 1;
    for (uint32_t w = 0; w < K; ++w) {  // hi == lo + 1 ?
        const uint64_t sum = (uint64_t)lo[w] + carry;
        if ((uint32_t)sum != hi[w]) return false;
        carry = (uint32_t)(sum >> 32);
    }
    return carry == 0;
}

struct LocalArgs {
    uint32_t* ck;          // partitioned, sorted in place; word-major, leading dimension ld
    uint32_t* rid;
    const uint32_t* start; // [B + 1]
    const uint32_t* spl;   // splitters
    const uint32_t* nsplit;  // their number, on the device (buckets = nsplit + 1)
    uint64_t ld;
    uint32_t K, B, cap;    // B: size of the bucket id space (buckets past nsplit are empty)
    uint32_t* next;        // bucket queue
    uint32_t* flags;       // [0] oversize buckets (also the length of `over`)
    uint32_t* counts;      // [0] buckets sorted, [1] constant buckets, [2] max bucket
    uint32_t* over;        // [2 * max_over] start/end of oversize buckets
    uint32_t max_over;
};

constexpr int kLocalThreads = 1024;
constexpr int kLocalWarps = kLocalThreads / 32;
constexpr uint32_t kShortRun = 16;  // runs of equal windows up to this length: insertion sort by one thread
constexpr uint32_t kBlockRun = 256; // runs from this length on are sorted by the whole block
constexpr int kRunList = 1024;      // shorter runs of one warp round (disjoint, so at most cap / 17)
constexpr int kBlockStack = 64;     // runs waiting for the block (disjoint, so at most cap / kBlockRun)

// Key i < key j (bucket-local indices into the word-major shared key array).
__device__ __forceinline__ bool key_less(const uint32_t* keys, uint32_t cap, uint32_t K, uint32_t i, uint32_t j) {
    for (int w = (int)K - 1; w >= 0; --w) {
        const uint32_t x = keys[(size_t)w * cap + i], y = keys[(size_t)w * cap + j];
        if (x != y) return x < y;
    }
    return false;
}

// Stable insertion sort of positions [p, p + len) of idx by key (one thread).
__device__ __forceinline__ void insertion_sort_run(uint16_t* idx, uint32_t p, uint32_t len, const uint32_t* keys,
                                                   uint32_t cap, uint32_t K) {
    for (uint32_t j = p + 1; j < p + len; ++j) {
        const uint16_t v = idx[j];
        uint32_t k = j;
        while (k > p && key_less(keys, cap, K, v, idx[k - 1])) {
            idx[k] = idx[k - 1];
            --k;
        }
        idx[k] = v;
    }
}

// Does any bit of [lo, lo + len) vary (mask over K words, bit 0 = word 0 bit 0)?
__device__ __forceinline__ bool bits_vary(const uint32_t* vary, uint32_t lo, uint32_t len, uint32_t K) {
    for (uint32_t w = lo >> 5; w < K && 32 * w < lo + len; ++w) {
        const uint32_t a = lo > 32 * w ? lo - 32 * w : 0u;
        const uint32_t e = lo + len - 32 * w;  // > a
        const uint32_t hi_mask = e >= 32 ? 0xFFFFFFFFu : ((1u << e) - 1u);
        if (vary[w] & hi_mask & (0xFFFFFFFFu << a)) return true;
    }
    return false;
}

// The sort window of a run: the 32 bits [base, base + 32) of the key that end
// at the run's top varying bit (all keys of the run agree above it).
struct Window {
    const uint32_t* lo;
    const uint32_t* hi;
    uint32_t sh, base;
    __device__ Window(const uint32_t* keys, uint32_t cap, uint32_t K, uint32_t top) {
        base = top >= 31 ? top - 31 : 0u;
        const uint32_t wl = base >> 5;
        sh = base & 31;
        lo = keys + (size_t)wl * cap;
        hi = keys + (size_t)(sh && wl + 1 < K ? wl + 1 : wl) * cap;
    }
    __device__ __forceinline__ uint32_t operator()(uint32_t i) const {
        return sh ? __funnelshift_r(lo[i], hi[i], sh) : lo[i];
    }
};

__device__ __forceinline__ int top_bit(const uint32_t* vary, uint32_t K) {
    for (int w = (int)K - 1; w >= 0; --w)
        if (vary[w]) return 32 * w + 31 - __clz(vary[w]);
    return -1;
}

// After a run is sorted by its window: items with equal windows (a sub-run)
// still differ below it.  The first position of every sub-run finds the
// sub-run's end by binary search (windows ascend) and sorts a short one at
// once; a longer one goes to the warp list, one of kBlockRun or more items
// to the block's stack (bstack == nullptr: the warp list).  Positions
// p0 + first, + step, ...
__device__ __forceinline__ void settle_sub_runs(uint16_t* idx, uint32_t p0, uint32_t pe, uint32_t first,
                                                uint32_t step, const Window& win, const uint32_t* keys, uint32_t cap,
                                                uint32_t K, uint32_t* list, uint32_t* count, uint32_t* bstack,
                                                uint32_t* bcount, uint32_t* overflow) {
    for (uint32_t p = p0 + first; p < pe; p += step) {
        const uint32_t wv = win(idx[p]);
        // (a sub-run's items all carry its window, so insertion sorts running
        // meanwhile in other threads do not change what is read here)
        if (p > p0 && win(idx[p - 1]) == wv) continue;      // not the first of its sub-run
        if (p + 1 >= pe || win(idx[p + 1]) != wv) continue;  // a single item
        uint32_t lo = p + 2, hi = pe;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (win(idx[mid]) == wv) lo = mid + 1;
            else hi = mid;
        }
        const uint32_t len = lo - p;
        if (len <= kShortRun) {
            insertion_sort_run(idx, p, len, keys, cap, K);
            continue;
        }
        const bool big = bstack && len >= kBlockRun;
        const uint32_t slot = atomicAdd(big ? bcount : count, 1u);
        if (slot < (big ? (uint32_t)kBlockStack : (uint32_t)kRunList)) (big ? bstack : list)[slot] = (len << 16) | p;
        else atomicAdd(overflow, 1u);  // cannot happen (disjoint runs); verification then fails
    }
}

// One warp sorts run [p0, p0 + r) by its window: LSD passes over the varying
// window digits, ranks by ballots against the warp's own 256 counters (which
// accumulate over the run's chunks, so a rank is the item's place among all
// earlier items of its digit), then its sub-runs are settled.
__device__ __forceinline__ void warp_sort_run(uint32_t p0, uint32_t r, const uint32_t* keys, uint32_t cap,
                                              uint32_t K, uint16_t* idx, uint16_t* alt, uint16_t* rnk, uint8_t* dig,
                                              uint16_t* wh, uint32_t* vary, uint32_t* list, uint32_t* count,
                                              uint32_t* overflow) {
    const uint32_t lane = threadIdx.x & 31, lt = (1u << lane) - 1u, pe = p0 + r;
    const uint32_t first = idx[p0];
    for (uint32_t w = 0; w < K; ++w) {
        const uint32_t* kw = keys + (size_t)w * cap;
        const uint32_t f = kw[first];
        uint32_t diff = 0;
        for (uint32_t p = p0 + lane; p < pe; p += 32) diff |= kw[idx[p]] ^ f;
        diff = __reduce_or_sync(kFull, diff);
        if (lane == 0) vary[w] = diff;
    }
    __syncwarp();
    const int top = top_bit(vary, K);
    if (top < 0) return;  // equal keys: already in order
    const Window win(keys, cap, K, (uint32_t)top);
    uint16_t* cur = idx;
    uint16_t* nxt = alt;
    for (uint32_t q = 0; q < 4; ++q) {
        if (!bits_vary(vary, win.base + 8 * q, 8, K)) continue;
        for (uint32_t i = lane; i < 256; i += 32) wh[i] = 0;
        __syncwarp();
        for (uint32_t c0 = p0; c0 < pe; c0 += 32) {
            const uint32_t p = c0 + lane;
            const bool valid = p < pe;
            const uint32_t d = valid ? (win(cur[p]) >> (8 * q)) & 0xFFu : 0u;
            uint32_t peers = __ballot_sync(kFull, valid);
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                const bool x = (d >> bit) & 1u;
                const uint32_t bal = __ballot_sync(kFull, x);
                peers &= x ? bal : ~bal;
            }
            const uint32_t cnt = valid ? wh[d] : 0u;
            __syncwarp();
            if (valid && (peers & lt) == 0) wh[d] = (uint16_t)(cnt + __popc(peers));
            __syncwarp();
            if (valid) {
                rnk[p] = (uint16_t)(cnt + __popc(peers & lt));
                dig[p] = (uint8_t)d;
            }
        }
        __syncwarp();
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            v[i] = wh[lane * 8 + i];
            sum += v[i];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, inc, o);
            if (lane >= (uint32_t)o) inc += t;
        }
        uint32_t ex = inc - sum;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            wh[lane * 8 + i] = (uint16_t)ex;
            ex += v[i];
        }
        __syncwarp();
        for (uint32_t p = p0 + lane; p < pe; p += 32) nxt[p0 + wh[dig[p]] + rnk[p]] = cur[p];
        __syncwarp();
        uint16_t* t = cur;
        cur = nxt;
        nxt = t;
    }
    if (cur != idx) {
        for (uint32_t p = p0 + lane; p < pe; p += 32) idx[p] = cur[p];
        __syncwarp();
    }
    if (win.base > 0 && bits_vary(vary, 0, win.base, K))
        settle_sub_runs(idx, p0, pe, lane, 32, win, keys, cap, K, list, count, nullptr, nullptr, overflow);
    __syncwarp();
}

// Shared state of a block sorting one bucket.
struct LocalShared {
    uint16_t whist[kLocalWarps][256];
    uint32_t dtot[256];
    uint32_t vary[kMaxLearnedWords];
    uint32_t wvary[kLocalWarps][kMaxLearnedWords];
    uint32_t lists[2][kRunList];
    uint32_t bstack[kBlockStack];
    uint32_t bucket, count[2], bcount, grab, run;
};

// The whole block sorts run [p0, p0 + r) of idx by its window: LSD passes
// over the varying window digits, each ranking the items of every warp's
// share (consecutive chunks of 32) by ballots against the warp's counters,
// then exclusive offsets digit-major, warp-minor over the warps that hold
// items, then the scatter.  Then its sub-runs are settled.
__device__ __forceinline__ void block_sort_run(uint32_t p0, uint32_t r, const uint32_t* keys, uint32_t cap,
                                               uint32_t K, uint16_t* idx, uint16_t* alt, uint16_t* rnk, uint8_t* dig,
                                               LocalShared& S, uint32_t* overflow) {
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, lt = (1u << lane) - 1u, pe = p0 + r;
    if (tid < K) S.vary[tid] = 0;
    __syncthreads();
    {
        const uint32_t first = idx[p0];
        for (uint32_t w = 0; w < K; ++w) {
            const uint32_t* kw = keys + (size_t)w * cap;
            const uint32_t f = kw[first];
            uint32_t diff = 0;
            for (uint32_t p = p0 + tid; p < pe; p += kLocalThreads) diff |= kw[idx[p]] ^ f;
            diff = __reduce_or_sync(kFull, diff);
            if (lane == 0 && diff) atomicOr(&S.vary[w], diff);
        }
    }
    __syncthreads();
    const int top = top_bit(S.vary, K);
    if (top < 0) return;  // equal keys: already in order (uniform: every thread returns)
    const Window win(keys, cap, K, (uint32_t)top);
    uint16_t* cur = idx;
    uint16_t* nxt = alt;
    const uint32_t per = ((r + kLocalWarps * 32 - 1) / (kLocalWarps * 32)) * 32;
    const uint32_t nw = (r + per - 1) / per;  // warps that hold items
    const uint32_t pbeg = p0 + warp * per, pend = min(pe, pbeg + per);
    for (uint32_t q = 0; q < 4; ++q) {
        if (!bits_vary(S.vary, win.base + 8 * q, 8, K)) continue;
        for (uint32_t d = tid; d < nw * 256; d += kLocalThreads) (&S.whist[0][0])[d] = 0;
        __syncthreads();
        for (uint32_t c0 = pbeg; c0 < pend; c0 += 32) {  // warp-uniform trip count
            const uint32_t p = c0 + lane;
            const bool valid = p < pend;
            const uint32_t d = valid ? (win(cur[p]) >> (8 * q)) & 0xFFu : 0u;
            uint32_t peers = __ballot_sync(kFull, valid);
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                const bool x = (d >> bit) & 1u;
                const uint32_t bal = __ballot_sync(kFull, x);
                peers &= x ? bal : ~bal;
            }
            const uint32_t cnt = valid ? S.whist[warp][d] : 0u;
            __syncwarp();
            if (valid && (peers & lt) == 0) S.whist[warp][d] = (uint16_t)(cnt + __popc(peers));
            __syncwarp();
            if (valid) {
                rnk[p] = (uint16_t)(cnt + __popc(peers & lt));
                dig[p] = (uint8_t)d;
            }
        }
        __syncthreads();
        // per digit: totals over warps, then exclusive offsets digit-major, warp-minor
        if (tid < 256) {
            uint32_t sum = 0;
            for (uint32_t ww = 0; ww < nw; ++ww) sum += S.whist[ww][tid];
            S.dtot[tid] = sum;
        }
        __syncthreads();
        if (tid < 32) {  // exclusive scan of 256 totals by one warp, 8 per lane
            uint32_t v[8], run_sum = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                v[i] = S.dtot[lane * 8 + i];
                run_sum += v[i];
            }
            uint32_t inc = run_sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, inc, o);
                if (lane >= (uint32_t)o) inc += t;
            }
            uint32_t ex = inc - run_sum;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                S.dtot[lane * 8 + i] = ex;
                ex += v[i];
            }
        }
        __syncthreads();
        if (tid < 256) {
            uint32_t off = S.dtot[tid];
            for (uint32_t ww = 0; ww < nw; ++ww) {
                const uint32_t c = S.whist[ww][tid];
                S.whist[ww][tid] = (uint16_t)off;
                off += c;
            }
        }
        __syncthreads();
        for (uint32_t p = pbeg + lane; p < pend; p += 32) nxt[p0 + S.whist[warp][dig[p]] + rnk[p]] = cur[p];
        __syncthreads();
        uint16_t* t = cur;
        cur = nxt;
        nxt = t;
    }
    if (cur != idx) {
        for (uint32_t p = p0 + tid; p < pe; p += kLocalThreads) idx[p] = cur[p];
        __syncthreads();
    }
    if (win.base > 0 && bits_vary(S.vary, 0, win.base, K))
        settle_sub_runs(idx, p0, pe, tid, kLocalThreads, win, keys, cap, K, S.lists[0], &S.count[0], S.bstack,
                        &S.bcount, overflow);
    __syncthreads();
}

// Persistent blocks take buckets from a queue.  A bucket of m <= cap pairs is
// loaded into shared memory and sorted by the 32-bit window that ends at its
// top varying bit (all its keys agree above it; the window separates almost
// all keys of a bucket, whose keys span a narrow key range): the whole block
// runs an LSD radix sort over the window's varying 8-bit digits, ranking a
// 16-bit index by warp ballots.  Items left with equal windows form sub-runs
// that differ only below the window: up to kShortRun items are sorted at once
// by a stable insertion sort of one thread; runs of kBlockRun or more items by
// the whole block in the same way, one after another; the others in rounds,
// one warp per sub-run, by their own windows, until none is left.  A run of
// equal keys is already in order (the partition is stable).  The keys then
// leave in sorted order and the row ids are gathered through the index.
// Constant buckets larger than cap are left as partitioned; other oversize
// buckets are listed for the plain radix sort.
__global__ void __launch_bounds__(kLocalThreads, 1) local_sort_kernel(const LocalArgs a) {
    extern __shared__ __align__(16) uint32_t lsm[];
    const uint32_t K = a.K, cap = a.cap;
    uint32_t* keys = lsm;                                                 // [K][cap]
    uint16_t* idx = reinterpret_cast<uint16_t*>(keys + (size_t)K * cap);  // [cap] current order
    uint16_t* alt = idx + cap;                                            // [cap]
    uint16_t* rnk = alt + cap;                                            // [cap] rank within the warp
    uint8_t* dig = reinterpret_cast<uint8_t*>(rnk + cap);                 // [cap]
    __shared__ LocalShared S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) {
            S.bucket = atomicAdd(a.next, 1u);
            S.count[0] = 0;
            S.count[1] = 0;
            S.bcount = 0;
        }
        __syncthreads();
        const uint32_t b = S.bucket;
        if (b >= a.B) break;
        const uint32_t s = a.start[b], m = a.start[b + 1] - s;
        if (tid == 0 && m > 0) atomicMax(&a.counts[2], m);
        if (m <= 1) {
            __syncthreads();
            continue;
        }
        if (m > cap) {
            if (tid == 0) {
                if (constant_bucket(a.spl, K, *a.nsplit + 1, b)) {
                    atomicAdd(&a.counts[1], 1u);
                } else {
                    const uint32_t slot = atomicAdd(&a.flags[0], 1u);
                    if (slot < a.max_over) {
                        a.over[2 * slot] = s;
                        a.over[2 * slot + 1] = s + m;
                    }
                }
            }
            __syncthreads();
            continue;
        }
        for (uint32_t w = 0; w < K; ++w)
            for (uint32_t t = tid; t < m; t += kLocalThreads)
                keys[(size_t)w * cap + t] = a.ck[(uint64_t)w * a.ld + s + t];
        for (uint32_t t = tid; t < m; t += kLocalThreads) idx[t] = (uint16_t)t;
        __syncthreads();
        if (m <= kShortRun) {
            if (tid == 0) insertion_sort_run(idx, 0, m, keys, cap, K);
        } else {
            if (tid == 0) {
                S.bstack[0] = m << 16;  // run = (length << 16) | first position; m <= cap < 2^16
                S.bcount = 1;
            }
            __syncthreads();
            for (;;) {  // runs for the whole block, one after another
                if (tid == 0) S.run = S.bcount > 0 ? S.bstack[--S.bcount] : 0xFFFFFFFFu;
                __syncthreads();
                const uint32_t run = S.run;
                if (run == 0xFFFFFFFFu) break;
                block_sort_run(run & 0xFFFFu, run >> 16, keys, cap, K, idx, alt, rnk, dig, S, &a.flags[1]);
                __syncthreads();
            }
            // rounds: one warp per shorter sub-run, appending the next round's runs
            uint32_t cur_list = 0;
            for (;;) {
                const uint32_t nruns = min(S.count[cur_list], (uint32_t)kRunList);
                if (nruns == 0) break;
                if (tid == 0) {
                    S.count[cur_list ^ 1] = 0;
                    S.grab = 0;
                }
                __syncthreads();
                for (;;) {
                    uint32_t e = 0;
                    if (lane == 0) e = atomicAdd(&S.grab, 1u);
                    e = __shfl_sync(kFull, e, 0);
                    if (e >= nruns) break;
                    const uint32_t run = S.lists[cur_list][e];
                    warp_sort_run(run & 0xFFFFu, run >> 16, keys, cap, K, idx, alt, rnk, dig, S.whist[warp],
                                  S.wvary[warp], S.lists[cur_list ^ 1], &S.count[cur_list ^ 1], &a.flags[1]);
                }
                __syncthreads();
                if (tid == 0) S.count[cur_list] = 0;
                cur_list ^= 1;
            }
        }
        __syncthreads();
        // write the bucket back in sorted order; row ids through the permutation
        for (uint32_t t = tid; t < m; t += kLocalThreads) {
            const uint32_t src = idx[t];
            for (uint32_t w = 0; w < K; ++w) a.ck[(uint64_t)w * a.ld + s + t] = keys[(size_t)w * cap + src];
        }
        __syncthreads();
        uint32_t* rtmp = keys;  // the keys are written out; their space holds the row ids
        for (uint32_t t = tid; t < m; t += kLocalThreads) rtmp[t] = a.rid[s + t];
        __syncthreads();
        for (uint32_t t = tid; t < m; t += kLocalThreads) a.rid[s + t] = rtmp[idx[t]];
        if (tid == 0) atomicAdd(&a.counts[0], 1u);
        __syncthreads();
    }
}

// Every adjacent output pair must be in (key, row id) order.
__global__ void verify_kernel(const uint32_t* __restrict__ ck, const uint32_t* __restrict__ rid, uint64_t ld,
                              uint64_t n, uint32_t K, uint32_t* __restrict__ flags) {
    uint32_t bad = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        int c = 0;
        for (int w = (int)K - 1; w >= 0 && c == 0; --w) {
            const uint32_t x = ck[(uint64_t)w * ld + i - 1], y = ck[(uint64_t)w * ld + i];
            c = x < y ? -1 : (x > y ? 1 : 0);
        }
        if (c > 0 || (c == 0 && rid[i - 1] >= rid[i])) ++bad;
    }
    if (bad) atomicAdd(&flags[1], bad);
}

// ------------------------------------------------------------ separators
// Model-proposed inner separators: for inner entry e of level l the canonical
// separator is the key of sorted rank hi = min((e + 1) f^l, n) - 1; the model
// proposes its top 24 compressed bits as the smallest 24-bit feature value x
// with y(x) >= (hi + 0.5) / n (bisection, 24 steps).  A proposal is a hit when
// it equals the canonical separator's top 24 bits; the tree always keeps the
// canonical key, so a miss is simply replaced.
__global__ void separators_kernel(const float* __restrict__ params, const __grid_constant__ InnerLevels lv, uint64_t n,
                                  uint32_t f, const uint32_t* __restrict__ high_ck, uint32_t K, uint32_t nbits,
                                  uint32_t* __restrict__ prop, uint32_t* __restrict__ hits) {
    __shared__ float p[kParams];
    if (threadIdx.x < kParams) p[threadIdx.x] = params[threadIdx.x];
    __syncthreads();
    uint32_t my_hits = 0;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < lv.inner_entries;
         g += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t l = 1;
        while (l + 1 < lv.levels && g >= lv.offset[l + 1]) ++l;
        const uint64_t e = g - lv.offset[l];
        uint64_t span = 1;
        for (uint32_t t = 0; t < l; ++t) span = min(span * f, n);
        const uint64_t hi = min((e + 1) * span, n) - 1;
        const float target = ((float)hi + 0.5f) / (float)n;
        uint32_t lo = 0, up = 1u << 24;
        while (lo < up) {
            const uint32_t mid = (lo + up) >> 1;
            if (mlp_eval(p, (float)mid * (1.0f / 16777216.0f)) >= target) up = mid;
            else lo = mid + 1;
        }
        const uint32_t proposal = lo > 0xFFFFFFu ? 0xFFFFFFu : lo;
        prop[g] = proposal;
        // canonical top 24 bits of the entry's compressed key (entry-major, K words)
        uint32_t canon;
        const uint32_t* c = high_ck + g * K;
        if (nbits >= 24) {
            const uint32_t lob = nbits - 24, w = lob >> 5, sh = lob & 31;
            uint64_t v = c[w];
            if (w + 1 < K) v |= (uint64_t)c[w + 1] << 32;
            canon = (uint32_t)(v >> sh) & 0xFFFFFFu;
        } else {
            canon = (c[0] << (24 - nbits)) & 0xFFFFFFu;
        }
        my_hits += proposal == canon ? 1u : 0u;
    }
    if (my_hits) atomicAdd(hits, my_hits);
}

// ------------------------------------------------------------ workspace
struct LearnedPlan {
    uint32_t B, bucket_bits, max_buckets, id_bits, passes, K, nbits;
    uint64_t S, ld_s, n, ld, div, chunk;
    uint32_t cap, epochs, train_blocks, flags, max_over;
    float lr;
    SortPlan sample_sort, plain;
    size_t off_sample, off_sample_sorted, off_sample_rid, off_sample_ws, off_xs, off_params, off_partial,
        off_misc, off_start, off_over, off_codes, off_spl, off_bkt, off_alt_bkt, off_alt_ck, off_alt_rid, off_hist,
        off_lookback, off_plain_ws, total;
};

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

static bool make_learned_plan(uint64_t n, uint32_t K, uint32_t nbits, const ck_learned_opts* o, LearnedPlan* p) {
    memset(p, 0, sizeof(*p));
    // bucket capacity of one block: K key words, two 16-bit indices, a 16-bit
    // rank and an 8-bit digit per pair in <= 200 KB, a multiple of 512
    uint32_t cap = (uint32_t)((200 * 1024) / (4 * K + 7)) / 512 * 512;
    if (cap > 16384) cap = 16384;
    p->cap = cap;
    // default bucket count: about 0.6 cap pairs per bucket (headroom for the
    // sampling noise of the quantiles), between 2^8 and 2^16 buckets
    uint32_t auto_bits = 8;
    while (auto_bits < 16 && (n >> auto_bits) > cap * 6 / 10) ++auto_bits;
    if (auto_bits == 16 && (n >> 15) <= cap * 3 / 4) auto_bits = 15;  // keeps the splitter table in shared memory
    p->bucket_bits = o && o->bucket_bits ? o->bucket_bits : auto_bits;
    if (p->bucket_bits < 8 || p->bucket_bits > 16) return false;
    p->B = 1u << p->bucket_bits;
    // heavy values add up to one bucket each; the bucket ids stay below 2^16
    p->max_buckets = p->bucket_bits <= 15 ? min(2 * p->B, p->B + 8192u) : p->B;
    p->id_bits = p->max_buckets > p->B ? p->bucket_bits + 1 : p->bucket_bits;
    p->passes = p->id_bits > 8 ? 2 : 1;
    p->div = o && o->sample_div ? o->sample_div : 100;
    p->epochs = o && o->epochs ? o->epochs : 100;
    p->lr = o && o->lr > 0.0f ? o->lr : 1e-3f;
    p->flags = o ? o->flags : 0u;
    p->K = K;
    p->nbits = nbits;
    p->n = n;
    p->ld = CK_LD(n);
    p->S = n / p->div;
    if (p->S < 2) p->S = n < 2 ? n : 2;
    p->ld_s = CK_LD(p->S);
    p->chunk = 4096;
    p->train_blocks = (uint32_t)min(num_sms(), 32);
    if (!make_sort_plan(p->S, K, nbits, 8, &p->sample_sort)) return false;
    if (!make_sort_plan(n, K, nbits, 8, &p->plain)) return false;
    const uint64_t tiles = (n + kPassTile - 1) / kPassTile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = a256(off + bytes);
        return at;
    };
    p->off_sample = take(4ull * K * p->ld_s);
    p->off_sample_sorted = take(4ull * K * p->ld_s);
    p->off_sample_rid = take(4ull * p->S);
    p->off_sample_ws = take(p->sample_sort.total);
    p->off_xs = take(4ull * p->S);
    p->off_params = take(4ull * kParams);
    p->off_partial = take(4ull * 2 * p->train_blocks * kRed);
    p->off_misc = take(256);  // barrier, loss, flags[2], counts[3], queue, steps[2] (u64)
    p->max_over = 4096;
    p->off_start = take(4ull * (p->max_buckets + 1));
    p->off_over = take(4ull * 2 * p->max_over);
    p->off_codes = take(p->B);
    p->off_spl = take(4ull * K * p->max_buckets);
    p->off_bkt = take(4ull * n);
    p->off_alt_bkt = take(4ull * n);
    p->off_alt_ck = take(4ull * K * p->ld);
    p->off_alt_rid = take(4ull * n);
    p->off_hist = take(4ull * 512);
    p->off_lookback = take(4ull * 256 * tiles * p->passes + 4 * p->passes);
    p->off_plain_ws = take(p->plain.total);
    p->total = off;
    return true;
}

}  // namespace ck

using namespace ck;

namespace {
struct Misc {  // layout of the misc block of the learned workspace
    unsigned barrier;
    float loss;
    uint32_t flags[2];   // oversize buckets, order violations
    uint32_t counts[3];  // buckets sorted, constant buckets, max bucket
    uint32_t next;       // bucket queue of the local sorts
    uint32_t nsplit;     // number of splitters
    unsigned long long steps[2];
};
}  // namespace

extern "C" {

size_t ck_mlp_workspace_bytes(void) { return (size_t)4 * 1024 * kRed; }

ck_status ck_mlp_loss_grad(const float* params, const float* x, const float* t, uint64_t S, float* grad_out,
                           float* loss_out, void* ws, size_t ws_bytes, ck_stream stream) {
    if (!params || !x || !grad_out || S == 0) return CK_EINVAL;
    if (!ws || ws_bytes < ck_mlp_workspace_bytes()) return CK_ENOMEM;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t want = (S + kTrainThreads - 1) / kTrainThreads;
    const uint32_t blocks = (uint32_t)(want < 1024 ? want : 1024);
    float* partial = static_cast<float*>(ws);
    mlp_grad_kernel<<<blocks, kTrainThreads, 0, s>>>(params, x, t, S, partial);
    mlp_grad_sum_kernel<<<1, 64, 0, s>>>(partial, blocks, S, grad_out, loss_out);
    count_launch(2);
    return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

size_t ck_sort_learned_workspace_bytes(uint64_t n, uint32_t ck_words, uint32_t nbits, const ck_learned_opts* opts) {
    LearnedPlan p;
    if (ck_words == 0 || ck_words > kMaxLearnedWords || !make_learned_plan(n, ck_words, nbits, opts, &p)) return 0;
    return p.total;
}

ck_status ck_sort_learned(const uint32_t* ck_in, uint32_t* ck_out, uint32_t* rid_out, uint64_t n, uint32_t ck_words,
                          uint32_t nbits, const ck_learned_opts* opts, ck_learned_stats* stats, float* params_out,
                          void* ws_v, size_t ws_bytes, ck_stream stream) {
    if (n > CK_MAX_ROWS || ck_words == 0 || ck_words > kMaxLearnedWords || nbits > 32u * ck_words) return CK_EINVAL;
    if (opts && (opts->reserved != 0 || (opts->flags & ~3u))) return CK_EINVAL;
    if (stats) memset(stats, 0, sizeof(*stats));
    if (n == 0) return CK_OK;
    if (!ck_in || !ck_out || !rid_out || ck_in == ck_out) return CK_EINVAL;
    LearnedPlan P;
    if (!make_learned_plan(n, ck_words, nbits, opts, &P)) return CK_EINVAL;
    if (!ws_v || ws_bytes < P.total || (reinterpret_cast<uintptr_t>(ws_v) & 255)) return CK_ENOMEM;
    unsigned long long* status = status_ptr();
    if (!status) return CK_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* ws = static_cast<unsigned char*>(ws_v);
    auto at = [&](size_t off) { return reinterpret_cast<uint32_t*>(ws + off); };
    const uint32_t K = ck_words;
    const bool use_model = !(P.flags & CK_LEARNED_NO_MODEL);
#define CK_TRY(x)                                    \
    do {                                             \
        if ((x) != cudaSuccess) return CK_ECUDA;     \
    } while (0)
    Misc* misc = reinterpret_cast<Misc*>(ws + P.off_misc);
    CK_TRY(cudaMemsetAsync(misc, 0, sizeof(Misc), s));
    CK_TRY(cudaMemsetAsync(ws + P.off_hist, 0, 4ull * 512, s));
    CK_TRY(cudaMemsetAsync(ws + P.off_lookback, 0, P.off_plain_ws - P.off_lookback, s));
    const int sms = num_sms();

    // 1. sample, sort the sample, features
    sample_kernel<<<sms * 4, 256, 0, s>>>(ck_in, P.ld, K, P.div, P.S, at(P.off_sample), P.ld_s);
    count_launch();
    CK_TRY(run_sort(P.sample_sort, at(P.off_sample), nullptr, at(P.off_sample_sorted), at(P.off_sample_rid), P.S,
                    nbits, kDefaultSpin, 0, 0, nullptr, ws + P.off_sample_ws, s));
    float* xs = reinterpret_cast<float*>(ws + P.off_xs);
    features_kernel<<<sms * 4, 256, 0, s>>>(at(P.off_sample_sorted), P.ld_s, P.S, K, nbits, xs);
    count_launch();

    // 2. model: spline initialisation, full-batch Adam (cooperative launch)
    float* params = reinterpret_cast<float*>(ws + P.off_params);
    if (use_model) {
        mlp_init_kernel<<<1, 32, 0, s>>>(xs, P.S, params);
        count_launch();
        TrainArgs ta;
        ta.xs = xs;
        ta.S = P.S;
        ta.stride = (P.S + kMaxTrainPoints - 1) / kMaxTrainPoints;
        ta.T = (P.S + ta.stride - 1) / ta.stride;
        ta.params = params;
        ta.partial = reinterpret_cast<float*>(ws + P.off_partial);
        ta.barrier = &misc->barrier;
        ta.loss = &misc->loss;
        ta.epochs = P.epochs;
        ta.lr = P.lr;
        ta.spin_limit = kDefaultSpin;
        ta.status = status;
        void* args[] = {&ta};
        CK_TRY(cudaLaunchCooperativeKernel((const void*)mlp_train_kernel, dim3(P.train_blocks), dim3(kTrainThreads),
                                           args, 0, s));
        count_launch();
    }
    // 3. splitters: sample quantiles (they cut through long shared prefixes that
    //    a 24-bit feature cannot see) moved to run ends, heavy values isolated
    const uint64_t heavy = std::max<uint64_t>(2, (P.S + 2ull * P.B - 1) / (2ull * P.B));
    uint8_t* codes = reinterpret_cast<uint8_t*>(ws + P.off_codes);
    quantile_kernel<<<(P.B + 255) / 256, 256, 0, s>>>(at(P.off_sample_sorted), P.ld_s, P.S, K, P.B, nbits, heavy,
                                                      codes);
    emit_splitters_kernel<<<1, 1024, 0, s>>>(at(P.off_sample_sorted), P.ld_s, P.S, K, P.B, P.max_buckets, codes,
                                             at(P.off_spl), &misc->nsplit);
    count_launch(2);

    // 4. bucket id of every key (model guess + exact correction), digit histograms
    BucketArgs ba;
    ba.ck = ck_in;
    ba.ld = P.ld;
    ba.n = n;
    ba.K = K;
    ba.nbits = nbits;
    ba.max_buckets = P.max_buckets;
    ba.nsplit = &misc->nsplit;
    ba.use_model = use_model ? 1u : 0u;
    ba.spl = at(P.off_spl);
    ba.params = use_model ? params : nullptr;
    ba.loss = &misc->loss;
    ba.bkt = at(P.off_bkt);
    ba.hist = at(P.off_hist);
    ba.steps = misc->steps;
    const size_t top_bytes = 4ull * (P.max_buckets - 1) + 4ull * ((1u << kPrefixBits) + 1);
    const bool staged = top_bytes <= 200 * 1024;
    CK_TRY(launch_bucket(ba, staged, top_bytes, sms, s));
    count_launch();
    CK_TRY(launch_bucket_scan(at(P.off_hist), P.passes, 8, s));

    // 5. stable partition by bucket id: radix passes over its low 8 bits, then the rest
    auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    const uint32_t bulk = al16(ck_in) && al16(ck_out) && al16(rid_out) ? 1u : 0u;
    const uint64_t tiles = (n + kPassTile - 1) / kPassTile;
    uint32_t* counters = at(P.off_lookback) + 256ull * tiles * P.passes;
    static thread_local PassArrays arr;
    for (uint32_t q = 0; q < P.passes; ++q) {
        const bool last = q + 1 == P.passes;
        uint32_t m = 0;
        const uint32_t* src_ck = q == 0 ? ck_in : at(P.off_alt_ck);
        uint32_t* dst_ck = last ? ck_out : at(P.off_alt_ck);
        // bucket ids: read by every pass, kept for the next pass only
        arr.src[m] = q == 0 ? at(P.off_bkt) : at(P.off_alt_bkt);
        arr.dst[m] = last ? nullptr : at(P.off_alt_bkt);
        ++m;
        for (uint32_t w = 0; w < K; ++w, ++m) {
            arr.src[m] = src_ck + (uint64_t)w * P.ld;
            arr.dst[m] = dst_ck + (uint64_t)w * P.ld;
        }
        arr.src[m] = q == 0 ? nullptr : at(P.off_alt_rid);
        arr.dst[m] = last ? rid_out : at(P.off_alt_rid);
        ++m;
        PassArgs a;
        a.n = n;
        a.narr = m;
        a.sh = 8 * q;
        a.bits = last ? P.id_bits - 8 * q : 8;
        a.straddle = 0;
        a.pass = q;
        a.bulk = bulk;
        a.bucket_base = at(P.off_hist) + 256 * q;
        a.lookback = at(P.off_lookback) + 256ull * tiles * q;
        a.tile_counter = counters + q;
        a.spin_limit = kDefaultSpin;
        a.inject = 0;
        a.status = status;
        CK_TRY(launch_onesweep_pass(8, a, arr, (uint32_t)tiles, s));
    }

    // 6. bucket starts (binary search of the splitters in the partitioned
    //    keys), then every bucket sorted in shared memory, in place
    uint32_t* start = at(P.off_start);
    bucket_bounds_kernel<<<(P.max_buckets + 256) / 256, 256, 0, s>>>(ck_out, P.ld, n, K, at(P.off_spl),
                                                                     &misc->nsplit, P.max_buckets, start);
    count_launch();
    LocalArgs la;
    la.ck = ck_out;
    la.rid = rid_out;
    la.start = start;
    la.spl = at(P.off_spl);
    la.nsplit = &misc->nsplit;
    la.ld = P.ld;
    la.K = K;
    la.B = P.max_buckets;
    la.cap = P.cap;
    la.next = &misc->next;
    la.flags = misc->flags;
    la.counts = misc->counts;
    la.over = at(P.off_over);
    la.max_over = P.max_over;
    const size_t lsmem = (size_t)P.cap * (4 * K + 7) + 16;
    CK_TRY(cudaFuncSetAttribute(local_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsmem));
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, local_sort_kernel, kLocalThreads, lsmem);
    local_sort_kernel<<<sms * (per_sm > 0 ? per_sm : 1), kLocalThreads, lsmem, s>>>(la);
    count_launch();
    Misc host;
    CK_TRY(cudaMemcpyAsync(&host, misc, sizeof(Misc), cudaMemcpyDeviceToHost, s));
    CK_TRY(cudaStreamSynchronize(s));
    // 7. buckets too large for a block (keys not all equal): the plain radix
    //    sort on just that segment, in place (the partition order is stable)
    bool failed = host.flags[0] > P.max_over;
    if (!failed && host.flags[0] > 0) {
        static thread_local uint32_t over[2 * 4096];
        CK_TRY(cudaMemcpy(over, at(P.off_over), 8ull * host.flags[0], cudaMemcpyDeviceToHost));
        for (uint32_t k = 0; k < host.flags[0] && !failed; ++k) {
            const uint64_t b0 = over[2 * k], m = over[2 * k + 1] - b0;
            SortPlan sp;
            if (!make_sort_plan(m, K, nbits, 8, &sp, P.ld) || sp.total > P.plain.total) {
                failed = true;
                break;
            }
            CK_TRY(run_sort(sp, ck_out + b0, rid_out + b0, ck_out + b0, rid_out + b0, m, nbits, kDefaultSpin, 0, 0,
                            nullptr, ws + P.off_plain_ws, s));
        }
    }

    // 8. verification of every adjacent pair
    verify_kernel<<<sms * 8, 256, 0, s>>>(ck_out, rid_out, P.ld, n, K, misc->flags);
    count_launch();
    CK_TRY(cudaMemcpyAsync(&host, misc, sizeof(Misc), cudaMemcpyDeviceToHost, s));
    CK_TRY(cudaStreamSynchronize(s));
    if (params_out && use_model) CK_TRY(cudaMemcpy(params_out, params, 4 * kParams, cudaMemcpyDeviceToHost));
    failed = failed || host.flags[1] != 0 || (P.flags & CK_LEARNED_INJECT_VERIFY_FAIL);
    if (stats) {
        stats->train_loss = use_model ? host.loss : 0.0f;
        stats->mean_search_steps = (float)((double)host.steps[0] / (double)n);
        stats->max_search_steps = (uint32_t)host.steps[1];
        stats->buckets = host.nsplit + 1;
        stats->sample_size = (uint32_t)P.S;
        stats->max_bucket = host.counts[2];
        stats->sorted_segments = host.counts[0];
        stats->constant_buckets = host.counts[1];
        stats->oversize_buckets = host.flags[0];
        stats->fell_back = failed ? 1u : 0u;
    }
    if (!failed) return CK_OK;
    // fallback: the plain radix sort from the untouched input
    CK_TRY(run_sort(P.plain, ck_in, nullptr, ck_out, rid_out, n, nbits, kDefaultSpin, 0, 0, nullptr,
                    ws + P.off_plain_ws, s));
#undef CK_TRY
    return CK_EVERIFY;
}

ck_status ck_model_separators(const float* params, const ck_btree* tree, uint32_t ck_words, uint32_t nbits,
                              uint32_t* proposals, uint32_t* hits, ck_stream stream) {
    if (!params || !tree || ck_words == 0 || ck_words > kMaxLearnedWords || nbits > 32u * ck_words || !hits)
        return CK_EINVAL;
    const ck_btree_shape& sh = tree->shape;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(hits, 0, sizeof(uint32_t), s) != cudaSuccess) return CK_ECUDA;
    if (sh.inner_entries == 0) return CK_OK;
    if (!proposals || !tree->inner_high_ck) return CK_EINVAL;
    InnerLevels lv;
    memset(&lv, 0, sizeof(lv));
    lv.levels = sh.levels;
    lv.inner_entries = sh.inner_entries;
    for (uint32_t l = 0; l < CK_MAX_LEVELS; ++l) lv.offset[l] = sh.inner_offset[l];
    const uint64_t want = (sh.inner_entries + 255) / 256, cap = (uint64_t)num_sms() * 8;
    separators_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, s>>>(params, lv, sh.n, sh.entries_per_node,
                                                                        tree->inner_high_ck, ck_words, nbits,
                                                                        proposals, hits);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

}  // extern "C"

// ck_learned.cu -- the learned-partition sort (not in the paper): a tiny fp32
// CDF model, trained on the GPU on a sample of the compressed keys, proposes
// the bucket boundaries of a stable partition; every bucket is then sorted in
// shared memory (ck_local_sort.cu).  The result is the same permutation as the
// plain radix sort:
//
//  * the buckets are key ranges between strictly increasing splitters: the
//    model's crossings of b / B over the sorted sample (moved to the start of
//    their run of equal keys), a bucket [v, v + 1) of its own for every heavy
//    key value, and sample quantiles inside any model bucket too large for a
//    shared-memory sort.  A stable partition by bucket followed by a stable
//    sort inside each bucket is a stable sort of the whole column;
//  * the model also proposes each key's bucket; a short search against the
//    splitters makes the assignment exact, so a poor model costs time, never
//    correctness;
//  * every check and decision runs on the device: when a check fails, the
//    plain radix sort -- launched gated on a device flag by every call, and
//    idle otherwise -- recomputes the output from the untouched input, and the
//    device status word records CK_EVERIFY.  Nothing waits for the host, so
//    the call can be captured in a CUDA graph.
//
// The model: y(x) = b2 + sum_j w2_j relu(w1_j x + b1_j), 16 hidden units, on
// x = the top 24 bits of the compressed key / 2^24, fitted by full-batch Adam
// to the empirical CDF (rank + 0.5) / S of the sorted sample.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ck_learned.cuh"

namespace ck {

constexpr int kHidden = CK_MLP_HIDDEN;
constexpr int kParams = CK_MLP_PARAMS;  // [w1(16), b1(16), w2(16), b2]
constexpr int kRed = kParams + 1;       // gradient + loss
constexpr int kTrainThreads = 256;
constexpr uint64_t kTrainPoints = 2048;  // training points: a stride subsample of the sorted sample
constexpr int kScanBlock = 1024;         // elements per block of the sample scans and gap compactions
constexpr uint32_t kMaxModelBuckets = 1u << 15;
constexpr uint32_t kMaxBucketIds = 1u << 16;  // bucket ids of two 8-bit partition passes
constexpr uint32_t kMaxConst = 1024;          // large constant buckets listed for the chunked check
constexpr uint32_t kStagedSplitters = 48 * 1024;  // splitters whose bits 16..31 the bucket kernel stages
constexpr uint32_t kPrefixCells = 1u << 16;        // prefix table over the top 16 bits of a key
constexpr uint32_t kPrefixEntries = kPrefixCells + 8;  // kPrefixCells + 1, rounded up to 16 bytes

// flags of a boundary gap g (between sample keys g - 1 and g)
constexpr uint32_t kGapModel = 1, kGapQuant = 2, kGapHeavyStart = 4, kGapHeavyEnd = 8;

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
// Full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8) by one block on T points
// of the sorted sample (indices 0, stride, 2 stride, ...; targets (i + 0.5) /
// S): the features sit in shared memory, the gradient is summed in a fixed
// order, so the same input trains the same bits.
__global__ void __launch_bounds__(kTrainThreads) mlp_train_kernel(const float* __restrict__ xs, uint64_t S,
                                                                   uint64_t T, uint64_t stride, float* params,
                                                                   float* loss, uint32_t epochs, float lr) {
    __shared__ float p[kParams], m1[kParams], m2[kParams];
    __shared__ float red[(kTrainThreads / 32) * kRed];
    __shared__ float out[kRed];
    __shared__ float xt[kTrainPoints];
    const int tid = threadIdx.x;
    for (uint64_t i = tid; i < T; i += kTrainThreads) xt[i] = xs[i * stride];
    if (tid < kParams) {
        p[tid] = params[tid];
        m1[tid] = 0.0f;
        m2[tid] = 0.0f;
    }
    __syncthreads();
    const float scale = 1.0f / (float)T, tscale = 1.0f / (float)S;
    float b1t = 1.0f, b2t = 1.0f, last = 0.0f;
    for (uint32_t ep = 0; ep < epochs; ++ep) {
        float g[kRed];
#pragma unroll
        for (int q = 0; q < kRed; ++q) g[q] = 0.0f;
        for (uint64_t i = tid; i < T; i += kTrainThreads)
            g[kParams] += mlp_accumulate(p, xt[i], ((float)(i * stride) + 0.5f) * tscale, scale, g);
        block_reduce_red(g, red, out);
        b1t *= 0.9f;
        b2t *= 0.999f;
        if (tid < kParams) {
            const float s = out[tid];
            m1[tid] = 0.9f * m1[tid] + 0.1f * s;
            m2[tid] = 0.999f * m2[tid] + 0.001f * s * s;
            const float mh = m1[tid] / (1.0f - b1t), vh = m2[tid] / (1.0f - b2t);
            p[tid] -= lr * mh / (sqrtf(vh) + 1e-8f);
        } else if (tid == kParams) {
            last = out[kParams] * scale;
        }
        __syncthreads();
    }
    if (tid < kParams) params[tid] = p[tid];
    if (tid == kParams) *loss = last;
}

// ------------------------------------------------------------ sample keys
// Sample key i against the K words v: -1, 0, 1.
__device__ __forceinline__ int cmp_sample(const uint32_t* smp, uint64_t ld_s, uint32_t K, uint64_t i,
                                          const uint32_t* v) {
    for (int w = (int)K - 1; w >= 0; --w) {
        const uint32_t x = smp[(uint64_t)w * ld_s + i];
        if (x != v[w]) return x < v[w] ? -1 : 1;
    }
    return 0;
}

__device__ __forceinline__ void load_sample(const uint32_t* smp, uint64_t ld_s, uint32_t K, uint64_t i, uint32_t* v) {
    for (uint32_t w = 0; w < K; ++w) v[w] = smp[(uint64_t)w * ld_s + i];
}

// First position in [a, c] whose key equals sample key c (the start of its run).
__device__ uint64_t run_start(const uint32_t* smp, uint64_t ld_s, uint32_t K, uint64_t a, uint64_t c) {
    uint32_t v[kMaxLearnedWords];
    load_sample(smp, ld_s, K, c, v);
    uint64_t lo = a, hi = c;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (cmp_sample(smp, ld_s, K, mid, v) < 0) lo = mid + 1;
        else hi = mid;
    }
    return lo;
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

// ------------------------------------------------------------ boundaries
// 1. the model over the sorted sample and the running maximum of its output,
//    block by block (ys = block-local running maximum, bmax = block maximum).
__global__ void __launch_bounds__(256) model_ys_kernel(const float* __restrict__ xs, uint64_t S,
                                                       const float* __restrict__ params, float* __restrict__ ys,
                                                       float* __restrict__ bmax) {
    __shared__ float p[kParams];
    __shared__ float wtot[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kParams) p[tid] = params[tid];
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kScanBlock + 4 * (uint64_t)tid;
    float y[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        y[k] = base + k < S ? mlp_eval(p, xs[base + k]) : -INFINITY;
        if (k) y[k] = fmaxf(y[k], y[k - 1]);
    }
    float inc = y[3];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc = fmaxf(inc, t);
    }
    if (lane == 31) wtot[warp] = inc;
    __syncthreads();
    float before = -INFINITY;
    for (int w = 0; w < warp; ++w) before = fmaxf(before, wtot[w]);
    float excl = __shfl_up_sync(kFull, inc, 1);
    excl = fmaxf(before, lane ? excl : -INFINITY);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < S) ys[base + k] = fmaxf(excl, y[k]);
    if (tid == 0) {
        float m = wtot[0];
        for (int w = 1; w < 8; ++w) m = fmaxf(m, wtot[w]);
        bmax[blockIdx.x] = m;
    }
}

// 2. the maximum of all earlier blocks (one block).
__global__ void __launch_bounds__(1024) max_carry_kernel(const float* __restrict__ bmax, uint32_t nblk,
                                                         float* __restrict__ carry) {
    __shared__ float part[1024];
    const uint32_t tid = threadIdx.x, per = (nblk + 1023) / 1024, lo = tid * per, hi = min(nblk, lo + per);
    float m = -INFINITY;
    for (uint32_t j = lo; j < hi; ++j) m = fmaxf(m, bmax[j]);
    part[tid] = m;
    __syncthreads();
    if (tid == 0) {
        float run = -INFINITY;
        for (int t = 0; t < 1024; ++t) {
            const float x = part[t];
            part[t] = run;
            run = fmaxf(run, x);
        }
    }
    __syncthreads();
    float run = part[tid];
    for (uint32_t j = lo; j < hi; ++j) {
        carry[j] = run;
        run = fmaxf(run, bmax[j]);
    }
}

// 3. model boundary b (0 < b < B): the first sample position where the running
//    maximum of y reaches b / B, moved to the start of its run of equal keys.
__global__ void model_cross_kernel(const float* __restrict__ ys, const float* __restrict__ bmax,
                                   const float* __restrict__ carry, uint32_t nblk, uint64_t S, uint32_t B,
                                   const uint32_t* __restrict__ smp, uint64_t ld_s, uint32_t K,
                                   uint32_t* __restrict__ mgap, uint32_t* __restrict__ flag) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= B; b += gridDim.x * blockDim.x) {
        if (b == 0 || b == B) {
            mgap[b] = b == 0 ? 0u : (uint32_t)S;
            continue;
        }
        const float target = (float)b / (float)B;
        uint32_t lo = 0, hi = nblk;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (fmaxf(carry[mid], bmax[mid]) >= target) hi = mid;
            else lo = mid + 1;
        }
        uint64_t c = S;
        if (lo < nblk) {
            const uint64_t b0 = (uint64_t)lo * kScanBlock;
            if (carry[lo] >= target) {
                c = b0;
            } else {
                uint64_t l = b0, h = min(S, b0 + kScanBlock) - 1;  // ys[h] >= target
                while (l < h) {
                    const uint64_t mid = (l + h) >> 1;
                    if (ys[mid] >= target) h = mid;
                    else l = mid + 1;
                }
                c = l;
            }
        }
        const uint64_t p = c >= S ? S : run_start(smp, ld_s, K, 0, c);
        mgap[b] = (uint32_t)p;
        if (p > 0 && p < S) atomicOr(&flag[p], kGapModel);
    }
}

// Without the model: the B-quantiles of the sample, moved to run starts.
__global__ void quantile_flag_kernel(uint64_t S, uint32_t B, const uint32_t* __restrict__ smp, uint64_t ld_s,
                                     uint32_t K, uint32_t* __restrict__ flag) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x + 1; b < B; b += gridDim.x * blockDim.x) {
        const uint64_t c = (uint64_t)b * S / B;
        const uint64_t p = run_start(smp, ld_s, K, 0, c);
        if (p > 0 && p < S) atomicOr(&flag[p], kGapQuant);
    }
}

// 4. heavy keys: a run of at least h equal sample keys [i, r1) gets the bucket
//    [v, v + 1): boundary gaps i (value v) and r1 (value v + 1).
__global__ void heavy_kernel(uint64_t S, uint64_t h, const uint32_t* __restrict__ smp, uint64_t ld_s, uint32_t K,
                             uint32_t nbits, uint32_t* __restrict__ flag, LearnedMisc* misc) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i + h <= S;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t v[kMaxLearnedWords];
        load_sample(smp, ld_s, K, i, v);
        if (i > 0 && cmp_sample(smp, ld_s, K, i - 1, v) == 0) continue;  // not a run start
        if (cmp_sample(smp, ld_s, K, i + h - 1, v) != 0) continue;       // run shorter than h
        uint64_t lo = i + h, hi = S;  // first position past the run
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (cmp_sample(smp, ld_s, K, mid, v) <= 0) lo = mid + 1;
            else hi = mid;
        }
        atomicOr(&flag[i], kGapHeavyStart);
        if (!is_max_key(v, K, nbits)) atomicOr(&flag[lo], kGapHeavyEnd);
        atomicAdd(&misc->counts[5], 1u);
    }
}

// Splitter values at gap g: an end value (sample g - 1 plus one) for a heavy
// run ending there, a start value (sample g) for any other boundary; one value
// when the two coincide.
__device__ __forceinline__ void gap_values(const uint32_t* smp, uint64_t ld_s, uint32_t K, uint32_t nbits, uint64_t S,
                                           uint64_t g, uint32_t f, bool* has_end, bool* has_start) {
    *has_start = (f & (kGapModel | kGapQuant | kGapHeavyStart)) && g < S;
    *has_end = false;
    if ((f & kGapHeavyEnd) && g >= 1) {
        uint32_t a[kMaxLearnedWords];
        load_sample(smp, ld_s, K, g - 1, a);
        if (!is_max_key(a, K, nbits)) {
            *has_end = true;
            if (*has_start) {  // a + 1 == sample g ?
                uint32_t carry = 1;
                bool eq = true;
                for (uint32_t w = 0; w < K; ++w) {
                    const uint64_t sum = (uint64_t)a[w] + carry;
                    eq &= (uint32_t)sum == smp[(uint64_t)w * ld_s + g];
                    carry = (uint32_t)(sum >> 32);
                }
                if (eq) *has_end = false;
            }
        }
    }
}

// Gap compaction, one gap per thread, kScanBlock gaps per block.
// mode 0: count flagged gaps; mode 1: count splitter values.
template <int MODE>
__device__ __forceinline__ uint32_t gap_weight(const uint32_t* flag, uint64_t g, uint64_t S, const uint32_t* smp,
                                               uint64_t ld_s, uint32_t K, uint32_t nbits) {
    if (g > S) return 0;
    const uint32_t f = flag[g];
    if (!f) return 0;
    if (MODE == 0) return 1;
    bool e, s;
    gap_values(smp, ld_s, K, nbits, S, g, f, &e, &s);
    return (e ? 1u : 0u) + (s ? 1u : 0u);
}

// Block-wide exclusive prefix of one small value per thread (1024 threads).
__device__ __forceinline__ uint32_t block_excl_1024(uint32_t x, uint32_t* wsum /*[33]*/, uint32_t* total) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, inc, o);
        if (lane >= (uint32_t)o) inc += t;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t v = wsum[lane];
        uint32_t vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, vi, o);
            if (lane >= (uint32_t)o) vi += t;
        }
        wsum[lane] = vi - v;
        if (lane == 31) wsum[32] = vi;
    }
    __syncthreads();
    const uint32_t r = wsum[warp] + inc - x;
    *total = wsum[32];
    __syncthreads();
    return r;
}

template <int MODE>
__global__ void __launch_bounds__(kScanBlock) gap_count_kernel(const uint32_t* __restrict__ flag, uint64_t S,
                                                               const uint32_t* __restrict__ smp, uint64_t ld_s,
                                                               uint32_t K, uint32_t nbits, uint32_t* __restrict__ bcnt) {
    __shared__ uint32_t wsum[33];
    const uint64_t g = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x;
    uint32_t total;
    block_excl_1024(gap_weight<MODE>(flag, g, S, smp, ld_s, K, nbits), wsum, &total);
    if (threadIdx.x == 0) bcnt[blockIdx.x] = total;
}

// Single-block exclusive scan of cnt[0, *len or len) in place; the total goes
// to *total; with limit > 0, a total >= limit sets *gate.
__global__ void __launch_bounds__(1024) scan_counts_kernel(uint32_t* cnt, uint32_t len, const uint32_t* len_dev,
                                                           uint32_t* total, uint32_t limit, uint32_t* gate) {
    __shared__ uint32_t wsum[33];
    const uint32_t L = len_dev ? *len_dev + 1 : len;
    const uint32_t per = (L + 1023) / 1024, lo = threadIdx.x * per, hi = min(L, lo + per);
    uint32_t s = 0;
    for (uint32_t j = lo; j < hi; ++j) s += cnt[j];
    uint32_t tot;
    uint32_t run = block_excl_1024(s, wsum, &tot);
    for (uint32_t j = lo; j < hi; ++j) {
        const uint32_t x = cnt[j];
        cnt[j] = run;
        run += x;
    }
    if (threadIdx.x == 0) {
        *total = tot;
        if (limit && tot >= limit) *gate = 1;
    }
}

// Flagged gaps in order.
__global__ void __launch_bounds__(kScanBlock) gap_write_kernel(const uint32_t* __restrict__ flag, uint64_t S,
                                                               const uint32_t* __restrict__ boff,
                                                               uint32_t* __restrict__ gaps) {
    __shared__ uint32_t wsum[33];
    const uint64_t g = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const uint32_t x = gap_weight<0>(flag, g, S, nullptr, 0, 0, 0);
    uint32_t total;
    const uint32_t r = block_excl_1024(x, wsum, &total) + boff[blockIdx.x];
    if (x) gaps[r] = (uint32_t)g;
}

// 5. model buckets with more sample keys than a bucket may hold (u) are cut
//    into pieces of about t sample keys: the number of cuts of every segment.
__device__ __forceinline__ void segment_of(const uint32_t* gaps, uint32_t g1, uint64_t S, uint32_t j, uint64_t* a,
                                           uint64_t* e) {
    *a = j ? gaps[j - 1] : 0;
    *e = j < g1 ? gaps[j] : S;
}

__device__ __forceinline__ uint32_t segment_cuts(const uint32_t* smp, uint64_t ld_s, uint32_t K, uint64_t a, uint64_t e,
                                                 float t_s, uint32_t u_s) {
    if (e <= a || e - a <= u_s) return 0;
    uint32_t v[kMaxLearnedWords];
    load_sample(smp, ld_s, K, a, v);
    if (cmp_sample(smp, ld_s, K, e - 1, v) == 0) return 0;  // one key value (a heavy run)
    const uint64_t pieces = (uint64_t)ceilf((float)(e - a) / t_s);
    return (uint32_t)(pieces > 1 ? pieces - 1 : 0);
}

__global__ void subdiv_count_kernel(const uint32_t* __restrict__ gaps, const LearnedMisc* misc, uint64_t S,
                                    const uint32_t* __restrict__ smp, uint64_t ld_s, uint32_t K, float t_s,
                                    uint32_t u_s, uint32_t* __restrict__ segcnt) {
    const uint32_t g1 = misc->g1;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= g1; j += gridDim.x * blockDim.x) {
        uint64_t a, e;
        segment_of(gaps, g1, S, j, &a, &e);
        segcnt[j] = segment_cuts(smp, ld_s, K, a, e, t_s, u_s);
    }
}

__global__ void subdiv_flag_kernel(const uint32_t* __restrict__ gaps, const LearnedMisc* misc, uint64_t S,
                                   const uint32_t* __restrict__ smp, uint64_t ld_s, uint32_t K, float t_s,
                                   uint32_t u_s, const uint32_t* __restrict__ segoff, uint32_t* __restrict__ flag) {
    const uint32_t g1 = misc->g1, nsub = misc->nsub;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nsub; q += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = g1;  // last segment with segoff <= q
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (segoff[mid] <= q) lo = mid;
            else hi = mid - 1;
        }
        uint64_t a, e;
        segment_of(gaps, g1, S, lo, &a, &e);
        const uint64_t pieces = segment_cuts(smp, ld_s, K, a, e, t_s, u_s) + 1ull;
        const uint64_t k = q - segoff[lo] + 1;
        const uint64_t pos = a + k * (e - a) / pieces;
        const uint64_t p = run_start(smp, ld_s, K, a, pos);
        if (p > a && p < S) atomicOr(&flag[p], kGapQuant);
    }
}

// 6. splitter values in order; gidx[g] = index of gap g's start value.
__global__ void __launch_bounds__(kScanBlock) value_write_kernel(const uint32_t* __restrict__ flag, uint64_t S,
                                                                 const uint32_t* __restrict__ smp, uint64_t ld_s,
                                                                 uint32_t K, uint32_t nbits,
                                                                 const uint32_t* __restrict__ boff,
                                                                 uint32_t max_splitters, uint32_t* __restrict__ spl,
                                                                 uint32_t* __restrict__ gidx, LearnedMisc* misc) {
    __shared__ uint32_t wsum[33];
    const uint64_t g = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const uint32_t f = g <= S ? flag[g] : 0u;
    bool e = false, s = false;
    if (f) gap_values(smp, ld_s, K, nbits, S, g, f, &e, &s);
    const uint32_t x = (e ? 1u : 0u) + (s ? 1u : 0u);
    uint32_t total;
    uint32_t r = block_excl_1024(x, wsum, &total) + boff[blockIdx.x];
    if (e && r < max_splitters) {
        uint32_t carry = 1;
        for (uint32_t w = 0; w < K; ++w) {
            const uint64_t sum = (uint64_t)smp[(uint64_t)w * ld_s + g - 1] + carry;
            spl[(uint64_t)r * K + w] = (uint32_t)sum;
            carry = (uint32_t)(sum >> 32);
        }
        ++r;
    }
    if (s && r < max_splitters) {
        for (uint32_t w = 0; w < K; ++w) spl[(uint64_t)r * K + w] = smp[(uint64_t)w * ld_s + g];
        gidx[g] = r;
        if (f & kGapModel) atomicAdd(&misc->counts[4], 1u);
    }
}

// 7. the model's guess: model bucket b starts at final bucket map[b].
__global__ void guess_map_kernel(const uint32_t* __restrict__ mgap, const uint32_t* __restrict__ gidx, uint64_t S,
                                 uint32_t B, const LearnedMisc* misc, uint32_t* __restrict__ map) {
    const uint32_t ns = misc->nsplit;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= B; b += gridDim.x * blockDim.x) {
        const uint32_t p = mgap[b];
        map[b] = p == 0 ? 0u : (p >= S ? ns : min(gidx[p] + 1, ns));
    }
}

// ------------------------------------------------------------ bucket ids
struct BucketArgs {
    const uint32_t* ck;
    uint64_t ld, n;
    uint32_t K, nbits, max_buckets, B, use_model, passes;
    const float* params;
    const uint32_t* spl;  // strictly increasing, entry-major
    const uint32_t* map;  // [B + 1]
    const uint16_t* pre;  // [kPrefixEntries] prefix table (prefix_table_kernel)
    LearnedMisc* misc;
    uint32_t* bkt;        // [n]
    uint32_t* hist;       // [2][256] digit counts of the bucket id (low byte, high byte)
};

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

// Comparison of key x (top32 value t) with splitter m of the key's prefix
// cell (the same top 16 bits): with `staged`, the shared table of the
// splitters' bits 16..31 decides unless they are equal too.
template <int KW>
__device__ __forceinline__ int cmp_at(const uint32_t (&key)[KW], uint32_t t, const uint16_t* low, bool staged,
                                      const uint32_t* spl, uint32_t m) {
    if (staged) {
        const uint32_t u = low[m], tl = t & 0xFFFFu;
        if (tl != u) return tl < u ? -1 : 1;
    }
    return cmp_key<KW>(key, spl + (uint64_t)m * KW);
}

// Number of splitters <= x within [lo, hi] (binary search).
template <int KW>
__device__ __forceinline__ uint32_t search_range(const uint32_t (&key)[KW], uint32_t t, const uint16_t* top,
                                                 bool staged, const uint32_t* spl, uint32_t lo, uint32_t hi,
                                                 uint32_t* cmp) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        ++*cmp;
        if (cmp_at<KW>(key, t, top, staged, spl, mid) >= 0) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Exact bucket from a guess g in [lo, hi] (the key's bucket is known to lie
// there): check the guess's range, then gallop away from it (1, 2, 4, ...
// buckets) and finish with a binary search, so a guess that is e buckets off
// costs about 2 log2(e) + 2 comparisons.
template <int KW>
__device__ __forceinline__ uint32_t search_from_guess(const uint32_t (&key)[KW], uint32_t t, const uint16_t* top,
                                                      bool staged, const uint32_t* spl, uint32_t lo, uint32_t hi,
                                                      uint32_t g, uint32_t* cmp) {
    ++*cmp;
    if (g > lo && cmp_at<KW>(key, t, top, staged, spl, g - 1) < 0) {  // below: gallop down
        uint32_t h = g - 1, step = 1;
        while (true) {
            const uint32_t probe = h >= lo + step ? h - step : lo;
            ++*cmp;
            if (cmp_at<KW>(key, t, top, staged, spl, probe) >= 0)
                return search_range<KW>(key, t, top, staged, spl, probe + 1, h, cmp);
            if (probe == lo) return lo;
            h = probe;
            step <<= 1;
        }
    }
    ++*cmp;
    if (g < hi && cmp_at<KW>(key, t, top, staged, spl, g) >= 0) {  // above: gallop up
        uint32_t l = g + 1, step = 1;
        while (true) {
            const uint32_t probe = l + step - 1 < hi ? l + step - 1 : hi - 1;
            ++*cmp;
            if (cmp_at<KW>(key, t, top, staged, spl, probe) < 0)
                return search_range<KW>(key, t, top, staged, spl, l, probe, cmp);
            l = probe + 1;
            if (probe == hi - 1) return hi;
            step <<= 1;
        }
    }
    return g;
}

// Prefix table over the top 16 bits of a key: pre[q] = the first splitter
// whose top 16 bits are >= q (q = 0 .. 2^16), so the splitters of cell q --
// those sharing the top 16 bits q -- are [pre[q], pre[q + 1]).
__global__ void prefix_table_kernel(const uint32_t* __restrict__ spl, uint32_t K, uint32_t nbits,
                                    const LearnedMisc* misc, uint32_t max_buckets, uint16_t* __restrict__ pre) {
    if (*(volatile const uint32_t*)&misc->gate) return;
    const uint32_t ns = min(misc->nsplit, max_buckets - 1);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < kPrefixEntries; q += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = ns;
        if (q <= kPrefixCells)
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if ((top32_mem(spl + (uint64_t)mid * K, K, nbits) >> 16) >= q) hi = mid;
                else lo = mid + 1;
            }
        pre[q] = (uint16_t)(q <= kPrefixCells ? lo : ns);
    }
}

// Bucket id of every key, the digit counts of the two partition passes, and
// the hash sum of the input pairs (key, row id = position).  The prefix table
// over the top 16 bits sits in shared memory, and when the splitters fit,
// bits 16..31 of each: a key's bucket lies in the range of its prefix cell,
// where those 16 bits decide every comparison unless they are equal too.  The
// model's guess (its bucket b maps to final bucket map[b]), clamped into that
// range, starts a galloping search where that is expected to be cheaper than
// a binary search of the range: the model's error is about e = sqrt(loss) B
// buckets, so galloping costs about 2 log2(e + 1) + 2 comparisons against
// log2(range + 1).
template <int KW>
__global__ void __launch_bounds__(1024) bucket_kernel(const BucketArgs a) {
    extern __shared__ uint16_t sm16[];
    uint16_t* pre = sm16;                    // [kPrefixEntries]
    uint16_t* low = sm16 + kPrefixEntries;   // [kStagedSplitters]
    __shared__ float p[kParams];
    __shared__ uint32_t hlo[256], hhi[256];
    LearnedMisc* misc = a.misc;
    if (*(volatile uint32_t*)&misc->gate) return;
    const int tid = threadIdx.x;
    const uint32_t ns = min(misc->nsplit, a.max_buckets - 1), nbits = a.nbits, B = a.B;
    const bool staged = ns <= kStagedSplitters;
    const float err = a.use_model ? sqrtf(fmaxf(misc->loss, 0.0f)) * (float)(ns + 1) + 1.0f : 0.0f;
    const float model_min_range = 4.0f * err * err;  // use the model on ranges wider than this
    if (tid < kParams) p[tid] = a.params ? a.params[tid] : 0.0f;
    if (tid < 256) {
        hlo[tid] = 0;
        hhi[tid] = 0;
    }
    for (uint32_t i = tid; i < kPrefixEntries / 8; i += blockDim.x)
        reinterpret_cast<uint4*>(pre)[i] = reinterpret_cast<const uint4*>(a.pre)[i];
    if (staged)
        for (uint32_t m = tid; m < ns; m += blockDim.x)
            low[m] = (uint16_t)(top32_mem(a.spl + (uint64_t)m * KW, KW, nbits) & 0xFFFFu);
    __syncthreads();
    unsigned long long my_sum = 0, my_max = 0;
    uint64_t my_hash = 0;
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
        uint32_t g, steps = 0;
        const uint32_t lo = pre[t >> 16], hi = pre[(t >> 16) + 1];
        if (a.use_model && (float)(hi - lo) + 1.0f > model_min_range) {
            const float x = (float)(t >> 8) * (1.0f / 16777216.0f);  // the top 24 bits, as in training
            const float y = mlp_eval(p, x) * (float)B;
            const uint32_t mb = y <= 0.0f ? 0u : (y >= (float)(B - 1) ? B - 1 : (uint32_t)y);
            uint32_t guess = a.map[mb];
            guess = guess < lo ? lo : (guess > hi ? hi : guess);
            g = search_from_guess<KW>(key, t, low, staged, a.spl, lo, hi, guess, &steps);
        } else {
            g = search_range<KW>(key, t, low, staged, a.spl, lo, hi, &steps);
        }
        a.bkt[i] = g;
        atomicAdd(&hlo[g & 255u], 1u);
        if (a.passes > 1) atomicAdd(&hhi[g >> 8], 1u);
        my_sum += steps;
        my_max = my_max > steps ? my_max : steps;
        uint64_t h = pair_hash_start((uint32_t)i);
#pragma unroll
        for (int w = 0; w < KW; ++w) h = pair_hash_word(h, key[w]);
        my_hash += pair_hash_end(h);
    }
    for (int o = 16; o > 0; o >>= 1) {
        my_sum += __shfl_xor_sync(kFull, my_sum, o);
        my_max = max(my_max, __shfl_xor_sync(kFull, my_max, o));
        my_hash += __shfl_xor_sync(kFull, my_hash, o);
    }
    if ((tid & 31) == 0) {
        atomicAdd(&misc->steps[0], my_sum);
        atomicMax(&misc->steps[1], my_max);
        atomicAdd(&misc->hash_in, (unsigned long long)my_hash);
    }
    __syncthreads();
    if (tid < 256) {
        if (hlo[tid]) atomicAdd(&a.hist[tid], hlo[tid]);
        if (hhi[tid]) atomicAdd(&a.hist[256 + tid], hhi[tid]);
    }
}

template <int KW>
static cudaError_t launch_bucket_kw(const BucketArgs& ba, size_t smem, int sms, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(bucket_kernel<KW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    bucket_kernel<KW><<<sms, 1024, smem, s>>>(ba);
    return cudaGetLastError();
}

static cudaError_t launch_bucket(const BucketArgs& ba, int sms, cudaStream_t s) {
    const size_t smem = 2ull * kPrefixEntries + 2ull * kStagedSplitters;
    switch (ba.K) {
        case 1: return launch_bucket_kw<1>(ba, smem, sms, s);
        case 2: return launch_bucket_kw<2>(ba, smem, sms, s);
        case 3: return launch_bucket_kw<3>(ba, smem, sms, s);
        case 4: return launch_bucket_kw<4>(ba, smem, sms, s);
        case 5: return launch_bucket_kw<5>(ba, smem, sms, s);
        case 6: return launch_bucket_kw<6>(ba, smem, sms, s);
        case 7: return launch_bucket_kw<7>(ba, smem, sms, s);
        default: return launch_bucket_kw<8>(ba, smem, sms, s);
    }
}

// start[b] = first position of bucket b in the partitioned keys: the first
// position whose key is >= spl[b - 1].  The partition is by key range, so
// that predicate is monotone in the position and a binary search finds it.
// start[0] = 0; buckets past the last splitter are empty (start = n).
__global__ void bucket_bounds_kernel(const uint32_t* __restrict__ ck, uint64_t ld, uint64_t n, uint32_t K,
                                     const uint32_t* __restrict__ spl, const LearnedMisc* misc, uint32_t max_buckets,
                                     uint32_t* __restrict__ start) {
    if (*(volatile const uint32_t*)&misc->gate) return;
    const uint32_t ns = min(misc->nsplit, max_buckets - 1);
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

// Last step: the checks' verdict (the gate of the plain fallback), the
// status word, the statistics and the trained parameters.
__global__ void finalize_kernel(LearnedMisc* misc, uint32_t force_fail, uint32_t use_model, uint32_t B, uint64_t S,
                                uint64_t n, uint32_t cap, unsigned long long* status, ck_learned_stats* stats,
                                const float* params, float* params_out) {
    if (threadIdx.x == 0) {
        if (!misc->gate && (misc->fail || misc->hash_in != misc->hash_out || force_fail)) misc->gate = 1;
        if (misc->gate) report(status, CK_EVERIFY, misc->fail);
        if (stats) {
            const uint32_t ns = misc->nsplit;
            stats->train_loss = use_model ? misc->loss : 0.0f;
            stats->mean_search_steps = (float)((double)misc->steps[0] / (double)n);
            stats->max_search_steps = (uint32_t)misc->steps[1];
            stats->buckets = ns + 1;
            stats->sample_size = (uint32_t)S;
            stats->max_bucket = misc->counts[2];
            stats->sorted_segments = misc->counts[0];
            stats->constant_buckets = misc->counts[1];
            stats->oversize_buckets = misc->counts[3];
            stats->fell_back = misc->gate;
            stats->model_buckets = B;
            stats->model_boundaries = use_model ? misc->counts[4] : 0u;
            stats->model_boundary_frac = use_model && ns ? (float)misc->counts[4] / (float)ns : 0.0f;
            stats->heavy_keys = misc->counts[5];
            stats->capacity = cap;
            stats->reserved = 0;
        }
    }
    if (params_out && use_model && threadIdx.x < kParams) params_out[threadIdx.x] = params[threadIdx.x];
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

__global__ void identity_rid_kernel(uint32_t* rid, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        rid[i] = (uint32_t)i;
}

// ------------------------------------------------------------ workspace
struct LearnedPlan {
    uint32_t B, max_buckets, passes, K, nbits, cap, epochs, flags, u_s;
    uint32_t nblk_s, nblk_g;  // blocks of the sample scans (S entries) and of the gap scans (S + 1 gaps)
    uint64_t S, ld_s, n, ld, div, T, tstride, h_s;
    float lr, t_s;
    SortPlan sample_sort, plain;
    size_t off_sample, off_sample_sorted, off_sample_rid, off_sample_ws, off_xs, off_ys, off_bmax, off_carry, off_flag,
        off_bcnt, off_gaps, off_seg, off_mgap, off_gidx, off_map, off_params, off_misc, off_spl, off_start, off_const,
        off_bkt, off_alt_bkt, off_alt_ck, off_alt_rid, off_hist, off_lookback, off_plain_ws, off_pre, total;
};

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

static bool make_learned_plan(uint64_t n, uint32_t K, uint32_t nbits, const ck_learned_opts* o, LearnedPlan* p) {
    memset(p, 0, sizeof(*p));
    if (K == 0 || K > kMaxLearnedWords || n < 2) return false;
    p->K = K;
    p->nbits = nbits;
    p->n = n;
    p->ld = CK_LD(n);
    p->cap = local_sort_cap(K);
    // model buckets: about 0.55 of a block's capacity per bucket on average
    uint32_t B = 2;
    if (o && o->bucket_bits) {
        if (o->bucket_bits > 15) return false;
        B = 1u << o->bucket_bits;
    } else {
        const double want = (double)n / (0.55 * p->cap);
        while (B < kMaxModelBuckets && (double)B < want) B <<= 1;
    }
    p->B = B;
    p->div = o && o->sample_div ? o->sample_div : 100;
    p->epochs = o && o->epochs ? o->epochs : 100;
    p->lr = o && o->lr > 0.0f ? o->lr : 1e-3f;
    p->flags = o ? o->flags : 0u;
    p->S = n / p->div;
    if (p->S < 2) {  // at least two sample keys: a stride that keeps both inside the column
        p->S = 2;
        p->div = n / 2;
    }
    p->ld_s = CK_LD(p->S);
    p->tstride = (p->S + kTrainPoints - 1) / kTrainPoints;
    p->T = (p->S + p->tstride - 1) / p->tstride;
    // u_s: most sample keys a bucket may hold so that its pairs (about
    // u_s * n / S, with a relative spread of 1 / sqrt(u_s)) stay within the
    // capacity at five standard deviations
    const double per = (double)n / (double)p->S;
    uint32_t u = 1;
    while ((double)(u + 1) * per * (1.0 + 5.0 / std::sqrt((double)(u + 1))) <= (double)p->cap && u < (1u << 30)) ++u;
    p->u_s = u;
    // t_s: sample keys per piece of an over-capacity model bucket -- those of
    // an average model bucket, or 2 u_s / 3 when an average model bucket is
    // itself over capacity (few model buckets, a small B): a cut moves back to
    // the start of its run of equal keys, and runs shorter than the heavy
    // threshold h_s = t_s / 2 stay in the piece, so such a piece holds at most
    // t_s + h_s <= u_s sample keys
    p->t_s = (float)((double)p->S / (double)B > (double)u ? 2.0 * (double)u / 3.0 : (double)p->S / (double)B);
    p->h_s = std::max<uint64_t>(2, std::min<uint64_t>(u, (uint64_t)(p->t_s / 2.0f)));
    // bucket id space: room for four times the buckets of a column cut into
    // pieces of t_s sample keys throughout (4 B when t_s = S / B), heavy keys
    // and model boundaries included; more needs the fallback
    const double pieces = std::ceil((double)p->S / (double)p->t_s);
    p->max_buckets = (uint32_t)std::min<double>(kMaxBucketIds, std::max<double>(256.0, 4.0 * pieces));
    p->passes = p->max_buckets > 256 ? 2 : 1;
    p->nblk_s = (uint32_t)((p->S + kScanBlock - 1) / kScanBlock);
    p->nblk_g = (uint32_t)((p->S + 1 + kScanBlock - 1) / kScanBlock);
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
    p->off_ys = take(4ull * p->nblk_s * kScanBlock);
    p->off_bmax = take(4ull * p->nblk_s);
    p->off_carry = take(4ull * p->nblk_s);
    p->off_flag = take(4ull * (p->S + 1));
    p->off_bcnt = take(4ull * p->nblk_g);
    p->off_gaps = take(4ull * (p->S + 1));
    p->off_seg = take(4ull * (p->S + 2));
    p->off_mgap = take(4ull * (B + 1));
    p->off_gidx = take(4ull * (p->S + 1));
    p->off_map = take(4ull * (B + 1));
    p->off_params = take(4ull * kParams);
    p->off_misc = take(sizeof(LearnedMisc));
    p->off_spl = take(4ull * K * p->max_buckets);
    p->off_start = take(4ull * (p->max_buckets + 1));
    p->off_const = take(4ull * 3 * kMaxConst);
    p->off_bkt = take(4ull * n);
    p->off_alt_bkt = take(4ull * n);
    p->off_alt_ck = take(4ull * K * p->ld);
    p->off_alt_rid = take(4ull * n);
    p->off_hist = take(4ull * 512);
    p->off_lookback = take(4ull * 256 * tiles * p->passes + 4 * p->passes);
    p->off_plain_ws = take(p->plain.total);
    p->off_pre = take(2ull * kPrefixEntries);
    p->total = off;
    return true;
}

}  // namespace ck

using namespace ck;

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
    if (ck_words == 0 || ck_words > kMaxLearnedWords) return 0;
    if (n < 2) return 256;
    if (!make_learned_plan(n, ck_words, nbits, opts, &p)) return 0;
    return p.total;
}

ck_status ck_sort_learned(const uint32_t* ck_in, uint32_t* ck_out, uint32_t* rid_out, uint64_t n, uint32_t ck_words,
                          uint32_t nbits, const ck_learned_opts* opts, ck_learned_stats* stats, float* params_out,
                          void* ws_v, size_t ws_bytes, ck_stream stream) {
    if (n > CK_MAX_ROWS || ck_words == 0 || ck_words > kMaxLearnedWords || nbits > 32u * ck_words) return CK_EINVAL;
    if (opts && (opts->reserved != 0 || (opts->flags & ~7u) || opts->bucket_bits > 15)) return CK_EINVAL;
    if (n == 0) return CK_OK;
    if (!ck_in || !ck_out || !rid_out || ck_in == ck_out) return CK_EINVAL;
    unsigned long long* status = status_ptr();
    if (!status) return CK_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
#define CK_TRY(x)                                    \
    do {                                             \
        if ((x) != cudaSuccess) return CK_ECUDA;     \
    } while (0)
    const uint32_t K = ck_words;
    const uint64_t ld = CK_LD(n);
    if (n < 2 || nbits == 0) {  // nothing to order: the keys as they are, row ids 0 .. n - 1
        CK_TRY(cudaMemcpy2DAsync(ck_out, 4 * ld, ck_in, 4 * ld, 4 * n, K, cudaMemcpyDeviceToDevice, s));
        identity_rid_kernel<<<num_sms() * 4, 256, 0, s>>>(rid_out, n);
        count_launch();
        if (stats) CK_TRY(cudaMemsetAsync(stats, 0, sizeof(ck_learned_stats), s));
        return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
    }
    LearnedPlan P;
    if (!make_learned_plan(n, K, nbits, opts, &P)) return CK_EINVAL;
    if (!ws_v || ws_bytes < P.total || (reinterpret_cast<uintptr_t>(ws_v) & 255)) return CK_ENOMEM;
    unsigned char* ws = static_cast<unsigned char*>(ws_v);
    auto at = [&](size_t off) { return reinterpret_cast<uint32_t*>(ws + off); };
    auto atf = [&](size_t off) { return reinterpret_cast<float*>(ws + off); };
    const bool use_model = !(P.flags & CK_LEARNED_NO_MODEL);
    LearnedMisc* misc = reinterpret_cast<LearnedMisc*>(ws + P.off_misc);
    const uint64_t tiles = (n + kPassTile - 1) / kPassTile;
    CK_TRY(cudaMemsetAsync(misc, 0, sizeof(LearnedMisc), s));
    CK_TRY(cudaMemsetAsync(ws + P.off_flag, 0, 4ull * (P.S + 1), s));
    CK_TRY(cudaMemsetAsync(ws + P.off_hist, 0, 4ull * 512, s));
    CK_TRY(cudaMemsetAsync(ws + P.off_lookback, 0, 4ull * 256 * tiles * P.passes + 4 * P.passes, s));
    const int sms = num_sms();
    const uint32_t* smp = at(P.off_sample_sorted);
    cudaEvent_t* ev = opts ? static_cast<cudaEvent_t*>(opts->phase_events) : nullptr;
    auto mark = [&](int k) { return ev ? cudaEventRecord(ev[k], s) : cudaSuccess; };
    CK_TRY(mark(0));

    // 1. sample, sort the sample, features
    sample_kernel<<<sms * 4, 256, 0, s>>>(ck_in, ld, K, P.div, P.S, at(P.off_sample), P.ld_s);
    count_launch();
    CK_TRY(run_sort(P.sample_sort, at(P.off_sample), nullptr, at(P.off_sample_sorted), at(P.off_sample_rid), P.S,
                    nbits, kDefaultSpin, 0, 0, nullptr, ws + P.off_sample_ws, s));
    float* xs = atf(P.off_xs);
    features_kernel<<<sms * 4, 256, 0, s>>>(smp, P.ld_s, P.S, K, nbits, xs);
    count_launch();

    // 2. model: spline initialisation, full-batch Adam
    float* params = atf(P.off_params);
    if (use_model) {
        mlp_init_kernel<<<1, 32, 0, s>>>(xs, P.S, params);
        mlp_train_kernel<<<1, kTrainThreads, 0, s>>>(xs, P.S, P.T, P.tstride, params, &misc->loss, P.epochs, P.lr);
        count_launch(2);
    }

    // 3. boundaries: the model's crossings (or plain quantiles), heavy keys,
    //    quantile cuts inside oversized model buckets; then the splitter values
    uint32_t* flag = at(P.off_flag);
    const uint32_t gb = (P.B + 256) / 256;
    if (use_model) {
        model_ys_kernel<<<P.nblk_s, 256, 0, s>>>(xs, P.S, params, atf(P.off_ys), atf(P.off_bmax));
        max_carry_kernel<<<1, 1024, 0, s>>>(atf(P.off_bmax), P.nblk_s, atf(P.off_carry));
        model_cross_kernel<<<gb, 256, 0, s>>>(atf(P.off_ys), atf(P.off_bmax), atf(P.off_carry), P.nblk_s, P.S, P.B,
                                              smp, P.ld_s, K, at(P.off_mgap), flag);
        count_launch(3);
    } else {
        quantile_flag_kernel<<<gb, 256, 0, s>>>(P.S, P.B, smp, P.ld_s, K, flag);
        count_launch();
    }
    heavy_kernel<<<sms * 4, 256, 0, s>>>(P.S, P.h_s, smp, P.ld_s, K, nbits, flag, misc);
    gap_count_kernel<0><<<P.nblk_g, kScanBlock, 0, s>>>(flag, P.S, smp, P.ld_s, K, nbits, at(P.off_bcnt));
    scan_counts_kernel<<<1, 1024, 0, s>>>(at(P.off_bcnt), P.nblk_g, nullptr, &misc->g1, 0, nullptr);
    gap_write_kernel<<<P.nblk_g, kScanBlock, 0, s>>>(flag, P.S, at(P.off_bcnt), at(P.off_gaps));
    subdiv_count_kernel<<<sms * 4, 256, 0, s>>>(at(P.off_gaps), misc, P.S, smp, P.ld_s, K, P.t_s, P.u_s,
                                                 at(P.off_seg));
    scan_counts_kernel<<<1, 1024, 0, s>>>(at(P.off_seg), 0, &misc->g1, &misc->nsub, 0, nullptr);
    subdiv_flag_kernel<<<sms * 4, 256, 0, s>>>(at(P.off_gaps), misc, P.S, smp, P.ld_s, K, P.t_s, P.u_s,
                                                at(P.off_seg), flag);
    gap_count_kernel<1><<<P.nblk_g, kScanBlock, 0, s>>>(flag, P.S, smp, P.ld_s, K, nbits, at(P.off_bcnt));
    scan_counts_kernel<<<1, 1024, 0, s>>>(at(P.off_bcnt), P.nblk_g, nullptr, &misc->nsplit, P.max_buckets,
                                          &misc->gate);
    value_write_kernel<<<P.nblk_g, kScanBlock, 0, s>>>(flag, P.S, smp, P.ld_s, K, nbits, at(P.off_bcnt),
                                                       P.max_buckets - 1, at(P.off_spl), at(P.off_gidx), misc);
    count_launch(9);
    if (use_model) {
        guess_map_kernel<<<gb, 256, 0, s>>>(at(P.off_mgap), at(P.off_gidx), P.S, P.B, misc, at(P.off_map));
        count_launch();
    }

    prefix_table_kernel<<<(kPrefixEntries + 255) / 256, 256, 0, s>>>(at(P.off_spl), K, nbits, misc, P.max_buckets,
                                                                     reinterpret_cast<uint16_t*>(ws + P.off_pre));
    count_launch();

    CK_TRY(mark(1));
    // 4. bucket id of every key (model guess + exact correction), digit
    //    counts, input hash
    BucketArgs ba;
    ba.ck = ck_in;
    ba.ld = ld;
    ba.n = n;
    ba.K = K;
    ba.nbits = nbits;
    ba.max_buckets = P.max_buckets;
    ba.B = P.B;
    ba.use_model = use_model ? 1u : 0u;
    ba.passes = P.passes;
    ba.params = use_model ? params : nullptr;
    ba.spl = at(P.off_spl);
    ba.map = at(P.off_map);
    ba.pre = reinterpret_cast<const uint16_t*>(ws + P.off_pre);
    ba.misc = misc;
    ba.bkt = at(P.off_bkt);
    ba.hist = at(P.off_hist);
    CK_TRY(launch_bucket(ba, sms, s));
    count_launch();
    CK_TRY(launch_bucket_scan(at(P.off_hist), P.passes, 8, s));

    CK_TRY(mark(2));
    // 5. stable partition by bucket id: radix passes over its low byte, then its high byte
    auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    const uint32_t bulk = al16(ck_in) && al16(ck_out) && al16(rid_out) ? 1u : 0u;
    uint32_t* counters = at(P.off_lookback) + 256ull * tiles * P.passes;
    for (uint32_t q = 0; q < P.passes; ++q) {
        PassArrays arr;
        const bool last = q + 1 == P.passes;
        uint32_t m = 0;
        const uint32_t* src_ck = q == 0 ? ck_in : at(P.off_alt_ck);
        uint32_t* dst_ck = last ? ck_out : at(P.off_alt_ck);
        // bucket ids: read by every pass, kept for the next pass only
        arr.src[m] = q == 0 ? at(P.off_bkt) : at(P.off_alt_bkt);
        arr.dst[m] = last ? nullptr : at(P.off_alt_bkt);
        ++m;
        for (uint32_t w = 0; w < K; ++w, ++m) {
            arr.src[m] = src_ck + (uint64_t)w * ld;
            arr.dst[m] = dst_ck + (uint64_t)w * ld;
        }
        arr.src[m] = q == 0 ? nullptr : at(P.off_alt_rid);
        arr.dst[m] = last ? rid_out : at(P.off_alt_rid);
        ++m;
        PassArgs a;
        a.n = n;
        a.narr = m;
        a.sh = 8 * q;
        a.bits = 8;
        a.straddle = 0;
        a.pass = q;
        a.bulk = bulk;
        a.bucket_base = at(P.off_hist) + 256 * q;
        a.lookback = at(P.off_lookback) + 256ull * tiles * q;
        a.tile_counter = counters + q;
        a.spin_limit = kDefaultSpin;
        a.inject = 0;
        a.status = status;
        a.gate = &misc->gate;
        a.gate_run = 0;
        CK_TRY(launch_onesweep_pass(8, a, arr, (uint32_t)tiles, s));
    }

    CK_TRY(mark(3));
    // 6. bucket starts, then every bucket sorted and checked
    uint32_t* start = at(P.off_start);
    bucket_bounds_kernel<<<(P.max_buckets + 256) / 256, 256, 0, s>>>(ck_out, ld, n, K, at(P.off_spl), misc,
                                                                     P.max_buckets, start);
    count_launch();
    LocalSortArgs la;
    la.ck = ck_out;
    la.rid = rid_out;
    la.ld = ld;
    la.n = n;
    la.K = K;
    la.cap = P.cap;
    la.max_buckets = P.max_buckets;
    la.start = start;
    la.spl = at(P.off_spl);
    la.misc = misc;
    la.const_list = at(P.off_const);
    la.max_const = kMaxConst;
    la.inject = P.flags;
    CK_TRY(launch_local_sort(la, s));

    CK_TRY(mark(4));
    // 7. verdict, statistics; the plain radix sort runs only if the verdict says so
    finalize_kernel<<<1, 64, 0, s>>>(misc, (P.flags & CK_LEARNED_INJECT_VERIFY_FAIL) ? 1u : 0u, use_model ? 1u : 0u,
                                     P.B, P.S, n, P.cap, status, stats, params, params_out);
    count_launch();
    CK_TRY(run_sort(P.plain, ck_in, nullptr, ck_out, rid_out, n, nbits, kDefaultSpin, 0, 0, nullptr,
                    ws + P.off_plain_ws, s, nullptr, &misc->gate));
    CK_TRY(mark(5));
#undef CK_TRY
    return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
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

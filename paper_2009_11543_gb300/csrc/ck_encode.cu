// ck_encode.cu -- index keys from several columns (Sec. 4.1, "Index Key
// Format"): the concatenation of each column's binary-comparable index key,
// so that a byte comparison of two rows is the lexicographic comparison of
// their tuples.  One thread per row; each part's bytes go to its offset.
#include <cstring>

#include "ck_internal.cuh"

namespace ck {

namespace {

struct Part {
    const unsigned char* values;
    const uint8_t* nulls;
    uint32_t kind, width, stride, offset;
};

struct EncodeParts {
    Part p[CK_MAX_KEY_PARTS];
    uint32_t nparts;
};

// The order-preserving form of a 32- or 64-bit value (see ck_column).
__device__ __forceinline__ uint32_t map32(uint32_t kind, uint32_t x) {
    if (kind == CK_KIND_I32) return x ^ 0x80000000u;
    if (kind == CK_KIND_F32) return (x >> 31) ? ~x : (x ^ 0x80000000u);
    return x;
}

__device__ __forceinline__ uint64_t map64(uint32_t kind, uint64_t x) {
    if (kind == CK_KIND_I64) return x ^ 0x8000000000000000ull;
    if (kind == CK_KIND_F64) return (x >> 63) ? ~x : (x ^ 0x8000000000000000ull);
    return x;
}

__device__ __forceinline__ void put_be(uint8_t* dst, uint64_t v, uint32_t bytes) {
    for (uint32_t b = 0; b < bytes; ++b) dst[b] = (uint8_t)(v >> (8 * (bytes - 1 - b)));
}

__global__ void encode_kernel(const __grid_constant__ EncodeParts ps, uint64_t n, uint8_t* __restrict__ out,
                              uint32_t out_stride, unsigned long long* status) {
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
        uint8_t* row = out + r * out_stride;
        for (uint32_t q = 0; q < ps.nparts; ++q) {
            const Part& p = ps.p[q];
            const unsigned char* src = p.values + r * p.stride;
            uint8_t* dst = row + p.offset;
            switch (p.kind) {
                case CK_KIND_BYTES:
                    for (uint32_t b = 0; b < p.width; ++b) dst[b] = src[b];
                    break;
                case CK_KIND_U32:
                case CK_KIND_I32:
                case CK_KIND_F32:
                    put_be(dst, map32(p.kind, *reinterpret_cast<const uint32_t*>(src)), 4);
                    break;
                case CK_KIND_U64:
                case CK_KIND_I64:
                case CK_KIND_F64:
                    put_be(dst, map64(p.kind, *reinterpret_cast<const uint64_t*>(src)), 8);
                    break;
                default: {  // CK_KIND_DECIMAL: header (not-null, sign) + magnitude, mapped (Sec. 4.1 A)
                    const int64_t v = *reinterpret_cast<const int64_t*>(src);
                    const bool null = p.nulls && p.nulls[r];
                    const bool neg = !null && v < 0;
                    const uint64_t mag = null ? 0ull : (neg ? 0ull - (uint64_t)v : (uint64_t)v);
                    const uint32_t mb = p.width - 1;  // magnitude bytes, 1 .. 8
                    if (mb < 8 && (mag >> (8 * mb)) != 0) report(status, CK_EOVERFLOW, r);
                    const uint32_t header = (null ? 0u : 2u) | (neg ? 1u : 0u);
                    dst[0] = (uint8_t)(header ^ 1u);  // the sign bit toggled
                    put_be(dst + 1, neg ? ~mag : mag, mb);
                    break;
                }
            }
        }
    }
}

}  // namespace
}  // namespace ck

using namespace ck;

extern "C" {

ck_status ck_encode_key(const ck_key_part* parts, uint32_t nparts, uint64_t n, uint8_t* out, uint32_t out_stride,
                        ck_stream stream) {
    if (!parts || nparts == 0 || nparts > CK_MAX_KEY_PARTS || n > CK_MAX_ROWS) return CK_EINVAL;
    EncodeParts ps;
    memset(&ps, 0, sizeof(ps));
    ps.nparts = nparts;
    uint32_t offset = 0;
    for (uint32_t q = 0; q < nparts; ++q) {
        const ck_key_part& a = parts[q];
        const uint32_t k = a.kind;
        uint32_t size;  // bytes read per row
        if (k == CK_KIND_BYTES) {
            if (a.width == 0) return CK_EINVAL;
            size = a.width;
        } else if (k == CK_KIND_U32 || k == CK_KIND_I32 || k == CK_KIND_F32) {
            if (a.width != 4) return CK_EINVAL;
            size = 4;
        } else if (k == CK_KIND_U64 || k == CK_KIND_I64 || k == CK_KIND_F64) {
            if (a.width != 8) return CK_EINVAL;
            size = 8;
        } else if (k == CK_KIND_DECIMAL) {
            if (a.width < 2 || a.width > 9) return CK_EINVAL;
            size = 8;
        } else {
            return CK_EINVAL;
        }
        if (a.stride < size || (n > 0 && !a.values)) return CK_EINVAL;
        if (k != CK_KIND_BYTES &&
            ((reinterpret_cast<uintptr_t>(a.values) % size) != 0 || (a.stride % size) != 0))
            return CK_EINVAL;
        ps.p[q] = Part{static_cast<const unsigned char*>(a.values), a.nulls, k, a.width, a.stride, offset};
        offset += a.width;
    }
    if (offset > CK_MAX_KEY_BYTES || out_stride < offset || (n > 0 && !out)) return CK_EINVAL;
    if (n == 0) return CK_OK;
    unsigned long long* status = status_ptr();
    if (!status) return CK_ECUDA;
    const uint64_t want = (n + 255) / 256, cap = (uint64_t)num_sms() * 8;
    encode_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        ps, n, out, out_stride, status);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? CK_OK : CK_ECUDA;
}

}  // extern "C"

// ck_sort_static.cu -- ck_sort_static: the radix sort of ck_sort with its
// scratch in a fixed device array of this library instead of a workspace the
// caller allocates.
//
// Some callers cannot allocate device memory on the path that rebuilds an
// index.  A database engine that owns every byte of device memory through its
// own memory manager may forbid its components to call cudaMalloc at all, and
// cudaMalloc / cudaFree can synchronise the whole device, which a caller in a
// latency-bound restart or replication path cannot afford.  Such a caller
// still owns its inputs and outputs; only the sort's scratch (digit
// histograms, look-back words, the second buffer of the ping-pong passes)
// comes from here.
//
// The scratch is one file-scope device array of CK_SORT_STATIC_SCRATCH_BYTES
// bytes.  Every GPU that loads this code holds it until the process exits;
// with CUDA's lazy module loading (the default) the code, and with it the
// array, is loaded on a device at the latest by the first call there, so a
// caller that must see no allocation on its path makes one call at start-up.
// All calls on a device share it and it keeps the previous call's contents;
// the sort clears the parts that must start at zero (histograms, tile
// counters, look-back words) at the start of every call.  Two calls whose
// execution overlaps on the GPU (different streams, or another thread) race on
// the array and give wrong results.
#include <mutex>

#include "ck_internal.cuh"

namespace ck {

static __device__ __align__(256) unsigned char g_sort_scratch[CK_SORT_STATIC_SCRATCH_BYTES];

static constexpr int kStaticMaxDevices = 64;
static std::mutex g_static_mu;
static unsigned char* g_static_addr[kStaticMaxDevices];

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device (with that device current) and cached.
static unsigned char* static_scratch(ck_status* st) {
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kStaticMaxDevices) {
        *st = CK_ECUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[d]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess || !p) {  // the module (and the array) could not be loaded on this device
            *st = e == cudaErrorMemoryAllocation ? CK_ENOMEM : CK_ECUDA;
            return nullptr;
        }
        g_static_addr[d] = static_cast<unsigned char*>(p);
    }
    *st = CK_OK;
    return g_static_addr[d];
}

}  // namespace ck

using namespace ck;

extern "C" ck_status ck_sort_static(const uint32_t* ck_in, const uint32_t* rid_in, uint32_t* ck_out,
                                    uint32_t* rid_out, uint64_t n, uint32_t ck_words, uint32_t nbits,
                                    const ck_sort_opts* opts, ck_stream stream) {
    if (n > CK_MAX_ROWS || ck_words == 0 || nbits > 32u * ck_words) return CK_EINVAL;
    if (opts && ((opts->flags & ~CK_SORT_FLAGS_ALL) != 0 || opts->reserved != 0 ||
                 (opts->digit_bits != 0 && (opts->digit_bits < 4 || opts->digit_bits > 11)) ||
                 (opts->tile != 0 && opts->tile != 2048 && opts->tile != 4096 && opts->tile != 8192)))
        return CK_EINVAL;
    if (n == 0) return CK_OK;
    if (!ck_in || !ck_out || !rid_out) return CK_EINVAL;
    SortPlan p;
    if (!make_sort_plan(n, ck_words, nbits, opts ? opts->digit_bits : 0, &p, 0, opts ? opts->tile : 0))
        return CK_EINVAL;
    if (p.passes > 0 && p.total > (size_t)CK_SORT_STATIC_SCRATCH_BYTES) return CK_ENOMEM;  // beyond the fixed array
    ck_status st = CK_OK;
    unsigned char* ws = static_scratch(&st);
    if (st != CK_OK) return st;
    if (!status_ptr()) return CK_ECUDA;
    const uint32_t spin = (opts && opts->spin_limit) ? opts->spin_limit : kDefaultSpin;
    const uint32_t inject = opts ? opts->inject : 0u;
    const uint32_t flags = opts ? opts->flags : 0u;
    cudaEvent_t* ev = opts ? static_cast<cudaEvent_t*>(opts->pass_events) : nullptr;
    const cudaError_t e = run_sort(p, ck_in, rid_in, ck_out, rid_out, n, nbits, spin, inject, flags, ev, ws,
                                   reinterpret_cast<cudaStream_t>(stream), opts ? opts->hist : nullptr);
    return e == cudaSuccess ? CK_OK : CK_ECUDA;
}

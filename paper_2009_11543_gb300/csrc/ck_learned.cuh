// ck_learned.cuh -- declarations shared by the learned-partition sort's files
// (ck_learned.cu: sample, model, bucket boundaries, partition and the host
// driver; ck_local_sort.cu: sorting and checking every bucket).
#pragma once

#include "ck_internal.cuh"

namespace ck {

constexpr uint32_t kMaxLearnedWords = 8;

// Order-independent check of the sort's output against its input: the sum
// (mod 2^64) of a 64-bit hash of every (compressed key, row id) pair.  Equal
// sums on both sides say that the output holds the input's pairs -- every
// row id once, each with its own key -- unless two different multisets of
// pairs collide in 64 bits.  The hash starts from the row id and folds in
// every key word by xor-then-multiply with an odd constant (nonlinear, so a
// key paired with another pair's row id hashes to an unrelated value), then
// avalanches with the SplitMix64 finaliser's last two rounds (Steele, Lea and
// Flood, "Fast splittable pseudorandom number generators", 2014).
__device__ __forceinline__ uint64_t pair_hash_start(uint32_t rid) {
    return (uint64_t)rid * 0x9E3779B97F4A7C15ull + 0xD1B54A32D192ED03ull;
}
__device__ __forceinline__ uint64_t pair_hash_word(uint64_t h, uint32_t word) {
    return (h ^ word) * 0xBF58476D1CE4E5B9ull;
}
__device__ __forceinline__ uint64_t pair_hash_end(uint64_t h) {
    h = (h ^ (h >> 31)) * 0x94D049BB133111EBull;
    return h ^ (h >> 29);
}

// Device counters and flags of one learned sort (part of its workspace).
struct LearnedMisc {
    uint32_t gate;          // 0: learned result stands; 1: the plain sort recomputes the output
    uint32_t fail;          // violations found by the checks (order, range, capacity)
    uint32_t nsplit;        // number of splitters (buckets - 1)
    uint32_t queue;         // bucket queue of the local sort
    uint32_t const_queue;   // chunk queue of the constant-bucket check
    uint32_t nconst;        // constant buckets listed for the chunked check
    uint32_t counts[6];     // sorted buckets, constant buckets, max bucket, oversize buckets, model boundaries,
                            // heavy keys isolated
    float loss;             // training loss of the model
    uint32_t g1;            // boundary gaps placed by the model and the heavy keys
    uint32_t nsub;          // boundaries added inside oversized model buckets
    uint32_t pad;
    unsigned long long hash_in, hash_out;
    unsigned long long steps[2];  // total and max splitter comparisons of the bucket search
};

struct LocalSortArgs {
    uint32_t* ck;            // partitioned keys (word-major, leading dimension ld); sorted per bucket in place
    uint32_t* rid;           // partitioned row ids
    uint64_t ld, n;
    uint32_t K;              // key words
    uint32_t cap;            // most pairs one block sorts in shared memory
    uint32_t max_buckets;    // bucket id space (start has max_buckets + 1 entries)
    const uint32_t* start;   // first position of every bucket
    const uint32_t* spl;     // splitters, entry-major K words, strictly increasing
    LearnedMisc* misc;
    uint32_t* const_list;    // [2 * max_const]: start, size of constant buckets left for the chunked check
    uint32_t max_const;
    uint32_t inject;         // CK_LEARNED_INJECT_* bits
};

// Dynamic shared memory of the local sort for a given capacity and key width.
size_t local_sort_smem(uint32_t cap, uint32_t K);
// Largest capacity (pairs per block) that fits shared memory, a multiple of 256.
uint32_t local_sort_cap(uint32_t K);
// Sorts every non-constant bucket (persistent blocks), checks every bucket
// (order, key range, row-id order of equal keys) and adds the pair hashes of
// the output; then checks the listed large constant buckets in chunks.
cudaError_t launch_local_sort(const LocalSortArgs& a, cudaStream_t s);

}  // namespace ck

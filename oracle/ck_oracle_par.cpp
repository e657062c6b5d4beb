/*
 * ck_oracle_par.cpp -- the compressed key sort of Sec. 3.2 on every host core:
 * the rows ordered by their compressed value, equal values in row-id order,
 * by GCC's parallel-mode stable sort (libstdc++ parallel mode on OpenMP), the
 * multi-threaded CPU sort the paper's evaluation compares with (Sec. 6).
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY, like ck_oracle.c: only tests/ and
 * the cpu_baseline leg of bench.py load it.  It shares no code with the CUDA
 * path and never calls into it.  The library sort is the whole algorithm;
 * this file only lays the pairs out for it and reads the order back.
 *
 * Layout as in ck_oracle.c: compressed keys row-major, K uint32 words per row,
 * least significant word first.
 */
#include <parallel/algorithm>
#include <omp.h>

#include <cstdint>
#include <cstring>
#include <vector>

namespace {

template <uint32_t K>
struct Pair {
    uint32_t w[K];  // most significant word first
    uint32_t rid;
};

template <uint32_t K>
bool pair_less(const Pair<K>& a, const Pair<K>& b) {
    for (uint32_t i = 0; i < K; ++i)
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i];
    return false;  // equal values: the stable sort keeps row-id order
}

template <uint32_t K>
void sort_k(const uint32_t* ck, uint64_t n, uint32_t* perm) {
    std::vector<Pair<K>> v(n);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < (int64_t)n; ++r) {
        for (uint32_t i = 0; i < K; ++i) v[r].w[i] = ck[(uint64_t)r * K + (K - 1 - i)];
        v[r].rid = (uint32_t)r;
    }
    __gnu_parallel::stable_sort(v.begin(), v.end(), pair_less<K>);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < (int64_t)n; ++r) perm[r] = v[r].rid;
}

}  // namespace

extern "C" {

/* Sorts rows 0..n-1 by compressed value (ties by row id) into perm on
 * `threads` threads (0: all of omp_get_num_procs()).  Returns the thread count
 * used, or -1 for an unsupported K (1..8 are). */
int cko_par_sort_compressed(const uint32_t* ck, uint64_t n, uint32_t K, uint32_t* perm, int threads) {
    const int t = threads > 0 ? threads : omp_get_num_procs();
    omp_set_num_threads(t);
    switch (K) {
        case 1: sort_k<1>(ck, n, perm); break;
        case 2: sort_k<2>(ck, n, perm); break;
        case 3: sort_k<3>(ck, n, perm); break;
        case 4: sort_k<4>(ck, n, perm); break;
        case 5: sort_k<5>(ck, n, perm); break;
        case 6: sort_k<6>(ck, n, perm); break;
        case 7: sort_k<7>(ck, n, perm); break;
        case 8: sort_k<8>(ck, n, perm); break;
        default: return -1;
    }
    return t;
}

}  // extern "C"

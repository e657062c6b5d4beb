// ck_batch.cu -- batched rebuild of all the indexes of one table, its CUDA
// graph capture, and the per-index autotuner of the radix digit width.
//
// The batch forks each job onto an internal stream of this library (events
// recorded on the caller's stream, waited on by the job streams, and the job
// streams' completion events waited on by the caller's stream), so the jobs'
// kernels overlap and a small index fills the SMs a large one leaves idle.
// Recorded inside stream capture, the whole table rebuild becomes one graph.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "ck_internal.cuh"

namespace ck {

namespace {

constexpr int kMaxDev = 64;

struct DeviceStreams {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
};

std::mutex g_batch_mu;
DeviceStreams g_dev[kMaxDev];
// Held by a batched call from its fork event through its last join, and by a
// capture from its begin to its end: every call shares the internal streams
// and the fork event, so two calls (or a call and a capture) must not
// interleave their records and waits.
std::mutex g_batch_call_mu;

// Internal non-blocking streams and events of the current device (created once).
DeviceStreams* device_streams(uint32_t need) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDev) return nullptr;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    DeviceStreams& ds = g_dev[d];
    if (!ds.fork && cudaEventCreateWithFlags(&ds.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    while (ds.streams.size() < need) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        ds.streams.push_back(st);
        ds.done.push_back(ev);
    }
    return &ds;
}

uint32_t popcount_mask(const uint64_t* m, uint32_t key_bits) {
    uint32_t c = 0;
    for (uint32_t w = 0; w < (key_bits + 63) / 64; ++w) c += (uint32_t)__builtin_popcountll(m[w]);
    return c;
}

}  // namespace
}  // namespace ck

using namespace ck;

struct ck_graph_st {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

// The batched rebuild; the caller holds g_batch_call_mu.
ck_status build_batched_locked(const ck_index_job* jobs, uint32_t njobs, ck_stream stream) {
    if (!jobs || njobs == 0 || njobs > CK_MAX_JOBS) return CK_EINVAL;
    for (uint32_t j = 0; j < njobs; ++j)
        if (!jobs[j].dmask || !jobs[j].tree) return CK_EINVAL;
    DeviceStreams* ds = device_streams(njobs);
    if (!ds) return CK_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaEventRecord(ds->fork, s) != cudaSuccess) return CK_ECUDA;
    ck_status first_error = CK_OK;
    for (uint32_t j = 0; j < njobs; ++j) {
        const ck_index_job& jb = jobs[j];
        cudaStream_t js = ds->streams[j];
        if (cudaStreamWaitEvent(js, ds->fork, 0) != cudaSuccess) return CK_ECUDA;
        ck_stream jst = reinterpret_cast<ck_stream>(js);
        const uint32_t key_bits = 8 * jb.col.key_bytes;
        const uint32_t nbits = popcount_mask(jb.dmask, key_bits);
        ck_sort_opts o;
        memset(&o, 0, sizeof(o));
        o.digit_bits = jb.digit_bits;
        o.tile = jb.tile;
        // room after the sort's workspace for the digit counts: take them while extracting
        const uint32_t rb = jb.digit_bits ? jb.digit_bits : 8u;
        const size_t sort_bytes = (ck_sort_workspace_bytes(jb.col.n, jb.ck_words, nbits, &o) + 255) & ~(size_t)255;
        const size_t hist_bytes = sizeof(uint32_t) * ((size_t)((nbits + rb - 1) / rb) << rb);
        uint32_t* hist = nullptr;
        if (nbits > 0 && jb.ws && jb.ws_bytes >= sort_bytes + hist_bytes)
            hist = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(jb.ws) + sort_bytes);
        ck_status st = hist ? ck_extract_hist(&jb.col, jb.dmask, jb.ck_words, jb.ck, rb, hist, jst)
                            : ck_extract(&jb.col, jb.dmask, jb.ck_words, jb.ck, jst);
        if (st == CK_OK) {
            o.hist = hist;
            st = ck_sort(jb.ck, nullptr, jb.ck_sorted, jb.rid_sorted, jb.col.n, jb.ck_words, nbits, &o, jb.ws,
                         hist ? sort_bytes : jb.ws_bytes, jst);
        }
        if (st == CK_OK)
            st = ck_build_index(jb.ck_sorted, jb.rid_sorted, jb.col.n, jb.ck_words, jb.dmask, key_bits, jb.fanout,
                                jb.fill, jb.tree, jb.refined_mask, jst);
        if (st != CK_OK && first_error == CK_OK) first_error = st;
        if (cudaEventRecord(ds->done[j], js) != cudaSuccess) return CK_ECUDA;
        if (cudaStreamWaitEvent(s, ds->done[j], 0) != cudaSuccess) return CK_ECUDA;
    }
    return first_error;
}

}  // namespace

extern "C" {

ck_status ck_build_batched(const ck_index_job* jobs, uint32_t njobs, ck_stream stream) {
    std::lock_guard<std::mutex> lk(g_batch_call_mu);
    return build_batched_locked(jobs, njobs, stream);
}

ck_status ck_graph_capture_batched(const ck_index_job* jobs, uint32_t njobs, ck_graph* graph_out) {
    if (!graph_out) return CK_EINVAL;
    *graph_out = nullptr;
    std::lock_guard<std::mutex> lk(g_batch_call_mu);
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return CK_ECUDA;
    ck_status st = CK_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return CK_ECUDA;
    }
    st = build_batched_locked(jobs, njobs, reinterpret_cast<ck_stream>(cs));
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st != CK_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess || !g) return CK_ECUDA;
    cudaGraphExec_t ex;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return CK_ECUDA;
    }
    ck_graph h = new ck_graph_st{g, ex};
    *graph_out = h;
    return CK_OK;
}

ck_status ck_graph_launch(ck_graph graph, ck_stream stream) {
    if (!graph) return CK_EINVAL;
    count_launch();
    return cudaGraphLaunch(graph->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? CK_OK : CK_ECUDA;
}

ck_status ck_graph_destroy(ck_graph graph) {
    if (!graph) return CK_EINVAL;
    cudaGraphExecDestroy(graph->exec);
    cudaGraphDestroy(graph->graph);
    delete graph;
    return CK_OK;
}

ck_status ck_autotune_sort(const uint32_t* ck_in, uint32_t* ck_out, uint32_t* rid_out, uint64_t n, uint32_t ck_words,
                           uint32_t nbits, void* ws, size_t ws_bytes, uint32_t reps, const char* cache_path,
                           uint32_t* best_digit_bits, uint32_t* best_tile, float* best_ms, ck_stream stream) {
    if (!best_digit_bits || !ck_in || !ck_out || !rid_out || ck_words == 0 || n == 0) return CK_EINVAL;
    if (reps == 0) reps = 3;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return CK_ECUDA;
    uint64_t nb = 1;
    while (nb < n) nb <<= 1;
    const bool tune_tile = best_tile != nullptr;
    char key[384];
    snprintf(key, sizeof(key), "%s|%llu|%u|%u|%s", prop.name, (unsigned long long)nb, ck_words, nbits,
             tune_tile ? "tile" : "width");
    if (cache_path) {  // cached choice?  lines: key|digit bits|tile
        if (FILE* f = fopen(cache_path, "r")) {
            char line[512];
            while (fgets(line, sizeof(line), f)) {
                char* bar2 = strrchr(line, '|');
                if (!bar2) continue;
                *bar2 = 0;
                char* bar1 = strrchr(line, '|');
                if (!bar1) continue;
                *bar1 = 0;
                if (strcmp(line, key) == 0) {
                    const unsigned d = (unsigned)strtoul(bar1 + 1, nullptr, 10);
                    const unsigned t = (unsigned)strtoul(bar2 + 1, nullptr, 10);
                    if (d >= 4 && d <= 11 && (t == 2048 || t == 4096 || t == 8192)) {
                        fclose(f);
                        *best_digit_bits = d;
                        if (best_tile) *best_tile = t;
                        if (best_ms) *best_ms = 0.0f;
                        return CK_OK;
                    }
                }
            }
            fclose(f);
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CK_ECUDA;
    uint32_t best = 0, best_t_tile = CK_SORT_TILE;
    float best_t = 0.0f;
    const uint32_t tiles[3] = {CK_SORT_TILE, 2048u, 8192u};
    for (uint32_t ti = 0; ti < (tune_tile ? 3u : 1u); ++ti)
        for (uint32_t d = 4; d <= 11; ++d) {
            ck_sort_opts o;
            memset(&o, 0, sizeof(o));
            o.digit_bits = d;
            o.tile = tiles[ti];
            const size_t need = ck_sort_workspace_bytes(n, ck_words, nbits, &o);
            if (need == 0 || need > ws_bytes) continue;
            ck_status st = ck_sort(ck_in, nullptr, ck_out, rid_out, n, ck_words, nbits, &o, ws, ws_bytes, stream);
            if (st != CK_OK) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st;
            }
            std::vector<float> t;
            for (uint32_t r = 0; r < reps; ++r) {
                cudaEventRecord(e0, s);
                ck_sort(ck_in, nullptr, ck_out, rid_out, n, ck_words, nbits, &o, ws, ws_bytes, stream);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    return CK_ECUDA;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                t.push_back(ms);
            }
            std::sort(t.begin(), t.end());
            const float med = t[t.size() / 2];
            if (best == 0 || med < best_t) {
                best = d;
                best_t_tile = tiles[ti];
                best_t = med;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best == 0) return CK_ENOMEM;
    *best_digit_bits = best;
    if (best_tile) *best_tile = best_t_tile;
    if (best_ms) *best_ms = best_t;
    if (cache_path)
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s|%u|%u\n", key, best, best_t_tile);
            fclose(f);
        }
    return CK_OK;
}

}  // extern "C"

// Autotuner: per (kernel, shape class) the fastest implementation variant, measured with CUDA
// events on the caller's stream the first time the class is seen (when tuning is on), cached for
// the process and exportable as text.
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "common.cuh"
#include "internal.h"
#include "tune.h"
#include "variants.h"

namespace glu {

namespace {

using Key = std::tuple<int, int, int, int, int, int>;
struct Entry {
    int variant;
    float ms;
};

std::mutex g_mu;
std::map<Key, Entry> g_cache;
bool g_on = false;
int g_forced[kTuneKernels] = {-1, -1};
thread_local bool t_timing_off = false;

int nvariants(int kernel) {
    if (kernel == kTuneSearch) return kNumSearchVariants;
    if (kernel == kTuneApply) return kNumApplyVariants;
    return 0;
}

Key make_key(int kernel, const int k[5]) { return Key(kernel, k[0], k[1], k[2], k[3], k[4]); }

}  // namespace

TuneTimingOff::TuneTimingOff() : prev(t_timing_off) { t_timing_off = true; }
TuneTimingOff::~TuneTimingOff() { t_timing_off = prev; }

int tune_size_class(long long n) {
    int c = 0;
    while ((1LL << c) < n && c < 62) ++c;
    return c;
}

int tune_choose(int kernel, const int key[5], int n, const std::function<int(int)>& run,
                cudaStream_t st, int* chosen) {
    *chosen = 0;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        const int f = g_forced[kernel];
        if (f >= 0 && f < n) {
            *chosen = f;
            return GLU_OK;
        }
        auto it = g_cache.find(make_key(kernel, key));
        if (it != g_cache.end()) {
            *chosen = it->second.variant;
            return GLU_OK;
        }
        if (!g_on || t_timing_off) return GLU_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return GLU_OK;  // no timing inside a graph capture: the default variant
    cudaEvent_t e0, e1;
    GLU_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GLU_ERR_CUDA;
    }
    constexpr int kReps = 3;
    int best = -1;
    float best_ms = 0.f;
    int rc = GLU_OK;
    for (int v = 0; v < n && rc == GLU_OK; ++v) {
        if (run(v) != GLU_OK) continue;  // a variant that cannot launch here is skipped
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = GLU_ERR_CUDA; break; }
        int vr = GLU_OK;
        for (int k = 0; k < kReps && vr == GLU_OK; ++k) vr = run(v);
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            rc = GLU_ERR_CUDA;
            break;
        }
        if (vr != GLU_OK) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= kReps;
        if (best < 0 || ms < best_ms) {
            best = v;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != GLU_OK) return rc;
    if (best < 0) return GLU_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[make_key(kernel, key)] = Entry{best, best_ms};
    *chosen = best;
    return GLU_OK;
}

}  // namespace glu

using namespace glu;

extern "C" {

int glu_tune_mode(int32_t on) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_on = on != 0;
    return GLU_OK;
}

int32_t glu_tune_variants(int32_t kernel) {
    const int n = nvariants(kernel);
    return n > 0 ? n : GLU_ERR_INVALID_ARG;
}

int glu_tune_variant_name(int32_t kernel, int32_t variant, char* buf, int32_t cap) {
    if (!buf || cap <= 0 || variant < 0 || variant >= nvariants(kernel)) return GLU_ERR_INVALID_ARG;
    if (kernel == kTuneSearch) {
        const SearchVariant& sv = kSearchVariants[variant];
        snprintf(buf, (size_t)cap, "tile %dx%d, %d CTAs/SM, %s candidate loops", kTileW, sv.tile_h,
                 sv.min_blocks, sv.compact ? "rolled" : "row-unrolled");
    } else {
        snprintf(buf, (size_t)cap, "tile 128x%d%s", kApplyVariants[variant].rows,
                 kApplyVariants[variant].tma == 2   ? ", TMA pipeline (persistent)"
                 : kApplyVariants[variant].tma == 1 ? ", TMA loads and stores"
                                                    : "");
    }
    return GLU_OK;
}

int glu_tune_force(int32_t kernel, int32_t variant) {
    if (nvariants(kernel) == 0 || variant < -1 || variant >= nvariants(kernel))
        return GLU_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mu);
    g_forced[kernel] = variant;
    return GLU_OK;
}

int glu_tune_clear(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache.clear();
    return GLU_OK;
}

int64_t glu_tune_export(char* buf, int64_t cap) {
    std::string out;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        char line[160];
        for (const auto& kv : g_cache) {
            const Key& k = kv.first;
            snprintf(line, sizeof(line), "%d %d %d %d %d %d %d %.6f\n", std::get<0>(k),
                     std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k),
                     kv.second.variant, (double)kv.second.ms);
            out += line;
        }
    }
    const int64_t need = (int64_t)out.size() + 1;
    if (buf && cap >= need) memcpy(buf, out.c_str(), (size_t)need);
    return need;
}

int glu_tune_import(const char* text) {
    if (!text) return GLU_ERR_INVALID_ARG;
    std::map<Key, Entry> add;
    const char* p = text;
    while (*p) {
        int k[6], v, used = 0;
        float ms;
        if (sscanf(p, "%d %d %d %d %d %d %d %f%n", &k[0], &k[1], &k[2], &k[3], &k[4], &k[5], &v,
                   &ms, &used) != 8)
            return GLU_ERR_INVALID_ARG;
        if (nvariants(k[0]) == 0 || v < 0 || v >= nvariants(k[0])) return GLU_ERR_INVALID_ARG;
        add[Key(k[0], k[1], k[2], k[3], k[4], k[5])] = Entry{v, ms};
        p += used;
        while (*p == '\n' || *p == ' ' || *p == '\r' || *p == '\t') ++p;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    for (const auto& kv : add) g_cache[kv.first] = kv.second;
    return GLU_OK;
}

}  // extern "C"

// Plan-time tuning of the cyclic grid p (the analogue of FFTW's measured planning,
// which the paper's FFTU relies on for its local FFTs, Sec. 4.1).
//
// For a problem with p left to the library, every candidate grid is planned, run on
// scratch buffers and timed with CUDA events in the plan's own direction; the fastest wins.
// Candidates: p_l = min(q, pmax_l) for q = 1, 2, 4, ..., where pmax_l is the largest
// power of two with p_l^2 | n_l (Algorithm 2.3's condition); the untuned default grid
// (q = 8) is one of them.
// Results are kept per (shape, dtype, direction, schedule, GPU name) in an in-process
// table that can be written to and read from a text file ("wisdom").
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fftu_internal.h"

namespace fftu {

namespace {

std::mutex g_wisdom_mutex;
std::map<std::string, std::vector<int64_t>> g_wisdom;

std::string wisdom_key(int d, const int64_t *n, int dtype, int dir, int sched) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char &c : name)
        if (c == ' ') c = '_';
    std::string k = std::to_string(d) + ":";
    for (int l = 0; l < d; ++l) k += (l ? "," : "") + std::to_string(n[l]);
    k += ":" + std::to_string(dtype) + ":" + std::to_string(dir) + ":" + std::to_string(sched) + ":" + name;
    return k;
}

// Time one candidate: best of three executions after one warm-up; < 0 on failure.
float time_candidate(int d, const int64_t *n, const int64_t *p, fftu_dtype dtype, fftu_dir dir, int sched,
                     void *in, void *out) {
    fftu_options o;
    std::memset(&o, 0, sizeof(o));
    o.schedule = sched;
    fftu_handle h = nullptr;
    if (fftu_plan_ex(d, n, p, dtype, dir, &o, &h) != FFTU_OK) return -1.f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = -1.f;
    bool ok = fftu_exec(h, in, out, nullptr) == FFTU_OK;
    for (int r = 0; ok && r < 3; ++r) {
        cudaEventRecord(e0, nullptr);
        ok = fftu_exec(h, in, out, nullptr) == FFTU_OK;
        cudaEventRecord(e1, nullptr);
        if (ok && cudaEventSynchronize(e1) == cudaSuccess) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (best < 0.f || ms < best) best = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (fftu_check_device_status(h) != FFTU_OK) best = -1.f;
    fftu_destroy(h);
    return ok ? best : -1.f;
}

}  // namespace

// p_out receives the chosen grid; returns true when tuning ran (or wisdom answered),
// false when the caller should fall back to the default grid (no memory, no candidates).
bool autotune_grid(int d, const int64_t *n, fftu_dtype dtype, fftu_dir dir, int sched, int64_t *p_out) {
    const std::string key = wisdom_key(d, n, dtype, dir, sched);
    {
        std::lock_guard<std::mutex> lock(g_wisdom_mutex);
        auto it = g_wisdom.find(key);
        if (it != g_wisdom.end() && (int)it->second.size() == d) {
            for (int l = 0; l < d; ++l) p_out[l] = it->second[l];
            return true;
        }
    }
    int64_t N = 1, pmax[FFTU_MAX_DIMS];
    for (int l = 0; l < d; ++l) {
        N *= n[l];
        int64_t q = 1;
        while (n[l] % ((2 * q) * (2 * q)) == 0) q *= 2;
        pmax[l] = q;
    }
    std::vector<std::vector<int64_t>> cands;
    for (int64_t q = 1;; q *= 2) {
        std::vector<int64_t> c(d);
        bool grew = false;
        for (int l = 0; l < d; ++l) {
            c[l] = q < pmax[l] ? q : pmax[l];
            if (q <= pmax[l]) grew = true;
        }
        cands.push_back(c);
        if (!grew) break;
    }
    const size_t bytes = (size_t)N * (dtype == FFTU_C128 ? 16 : 8);
    void *in = nullptr, *out = nullptr;
    if (cudaMalloc(&in, bytes) != cudaSuccess || cudaMalloc(&out, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (in) cudaFree(in);
        return false;
    }
    cudaMemset(in, 0, bytes);
    float best = -1.f;
    std::vector<int64_t> best_p;
    for (const auto &c : cands) {
        const float ms = time_candidate(d, n, c.data(), dtype, dir, sched, in, out);
        if (ms >= 0.f && (best < 0.f || ms < best)) {
            best = ms;
            best_p = c;
        }
    }
    cudaFree(in);
    cudaFree(out);
    if (best_p.empty()) return false;
    for (int l = 0; l < d; ++l) p_out[l] = best_p[l];
    std::lock_guard<std::mutex> lock(g_wisdom_mutex);
    g_wisdom[key] = best_p;
    return true;
}

}  // namespace fftu

extern "C" {

fftu_status fftu_wisdom_export(const char *path) {
    if (!path) return FFTU_ERR_ARG;
    FILE *f = std::fopen(path, "w");
    if (!f) {
        fftu::record_error("wisdom: cannot open the file for writing");
        return FFTU_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(fftu::g_wisdom_mutex);
    for (const auto &kv : fftu::g_wisdom) {
        std::fprintf(f, "fftu-wisdom-v1 %s", kv.first.c_str());
        for (size_t l = 0; l < kv.second.size(); ++l) std::fprintf(f, "%s%lld", l ? "," : " ", (long long)kv.second[l]);
        std::fprintf(f, "\n");
    }
    std::fclose(f);
    return FFTU_OK;
}

fftu_status fftu_wisdom_import(const char *path) {
    if (!path) return FFTU_ERR_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f) {
        fftu::record_error("wisdom: cannot open the file for reading");
        return FFTU_ERR_ARG;
    }
    char tag[32], key[512], vals[256];
    std::lock_guard<std::mutex> lock(fftu::g_wisdom_mutex);
    while (std::fscanf(f, "%31s %511s %255s", tag, key, vals) == 3) {
        if (std::strcmp(tag, "fftu-wisdom-v1") != 0) continue;
        std::vector<int64_t> p;
        for (char *tok = std::strtok(vals, ","); tok; tok = std::strtok(nullptr, ",")) p.push_back(std::atoll(tok));
        fftu::g_wisdom[key] = p;
    }
    std::fclose(f);
    return FFTU_OK;
}

fftu_status fftu_wisdom_forget(void) {
    std::lock_guard<std::mutex> lock(fftu::g_wisdom_mutex);
    fftu::g_wisdom.clear();
    return FFTU_OK;
}

}  // extern "C"

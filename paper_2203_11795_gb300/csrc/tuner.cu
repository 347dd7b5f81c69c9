// Plan-time tuning (the analogue of FFTW's measured planning, which the paper's FFTU relies on
// for its local FFTs, Sec. 4.1), over the choices this library adds: the cyclic grid p, the
// kernel schedule, and the strided passes' tile size and stage radix.
//
// Every candidate is planned, run once on scratch buffers, then timed with CUDA events (best of
// three executions, the plan's own direction).  The search takes one coordinate at a time:
//   1. p: p_l = min(q, pmax_l) for q = 1, 2, 4, ..., where pmax_l is the largest power of two with
//      p_l^2 | n_l (Algorithm 2.3's condition), each also with the last axis at q / 2 (e.g. 16 x 16 x 8);
//      the untuned default (q = 8) is one of them;
//   2. for that p, the schedule (AUTO, GENERIC_A, GENERIC), unless the caller fixed one;
//   3. the whole-line tile target of the strided passes, unless fixed;
//   4. their stage radix (8 or 16), unless fixed.
// Results are kept per (shape, dtype, direction, requested schedule, precision, GPU name) in an
// in-process table that can be written to and read from a text file ("wisdom").
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fftu_internal.h"

namespace fftu {

namespace {

struct Wise {
    std::vector<int64_t> p;
    int schedule = 0, tile = 0, radix = 0;  // 0: not chosen (the plan's default)
};

std::mutex g_wisdom_mutex;
std::map<std::string, Wise> g_wisdom;

std::string gpu_name() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::string name = "unknown";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    else cudaGetLastError();
    for (char &c : name)
        if (c == ' ') c = '_';
    return name;
}

std::string wisdom_key(int d, const int64_t *n, int dtype, int dir, int sched, int precision) {
    std::string k = std::to_string(d) + ":";
    for (int l = 0; l < d; ++l) k += (l ? "," : "") + std::to_string(n[l]);
    k += ":" + std::to_string(dtype) + ":" + std::to_string(dir) + ":" + std::to_string(sched) + ":" +
         std::to_string(precision) + ":" + gpu_name();
    return k;
}

// Time one candidate: best of three executions after one warm-up; < 0 on failure.
float time_candidate(int d, const int64_t *n, const int64_t *p, fftu_dtype dtype, fftu_dir dir,
                     const fftu_options &o, void *in, void *out) {
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

// An imported line is kept only if its key and choices describe a plan fftu_plan_ex would accept:
// key d:n_0,...,n_{d-1}:dtype:dir:schedule:precision:gpu with power-of-two n_l, and a grid with
// p_l^2 | n_l, a known schedule, a tile of 0 or a power of two in [1024, 8192] (4096 for complex128)
// and a radix of 0, 8 or 16.  A file is input from outside the process: a bad line must not reach a
// plan.
bool valid_entry(const std::string &key, const Wise &w) {
    const std::vector<std::string> f = [&] {
        std::vector<std::string> parts;
        size_t start = 0;
        for (size_t i = 0; i <= key.size(); ++i)
            if (i == key.size() || key[i] == ':') {
                parts.push_back(key.substr(start, i - start));
                start = i + 1;
            }
        return parts;
    }();
    if (f.size() < 7) return false;  // fields 6.. are the GPU name
    char *end = nullptr;
    const long d = std::strtol(f[0].c_str(), &end, 10);
    if (*end || d < 1 || d > FFTU_MAX_DIMS || (long)w.p.size() != d) return false;
    std::vector<long long> n;
    for (size_t start = 0; start <= f[1].size();) {
        size_t stop = f[1].find(',', start);
        if (stop == std::string::npos) stop = f[1].size();
        const std::string tok = f[1].substr(start, stop - start);
        const long long v = std::strtoll(tok.c_str(), &end, 10);
        if (tok.empty() || *end || v < 1 || v > (1ll << 40) || (v & (v - 1))) return false;
        n.push_back(v);
        start = stop + 1;
    }
    if ((long)n.size() != d) return false;
    const long dtype = std::strtol(f[2].c_str(), &end, 10);
    if (*end || (dtype != FFTU_C64 && dtype != FFTU_C128)) return false;
    const long dir = std::strtol(f[3].c_str(), &end, 10);
    if (*end || (dir != FFTU_FORWARD && dir != FFTU_INVERSE)) return false;
    const long sched = std::strtol(f[4].c_str(), &end, 10);
    if (*end || sched < FFTU_SCHED_AUTO || sched > FFTU_SCHED_GENERIC_A) return false;
    const long prec = std::strtol(f[5].c_str(), &end, 10);
    if (*end || prec < FFTU_PREC_NATIVE || prec > FFTU_PREC_SPLIT_FP16) return false;
    for (long l = 0; l < d; ++l) {
        const long long q = w.p[l];
        if (q < 1 || q > n[l] / q || (q & (q - 1)) || n[l] % (q * q) != 0) return false;
    }
    if (w.schedule < FFTU_SCHED_AUTO || w.schedule > FFTU_SCHED_GENERIC_A) return false;
    const int tmax = dtype == FFTU_C128 ? 4096 : 8192;
    if (w.tile != 0 && (w.tile < 1024 || w.tile > tmax || (w.tile & (w.tile - 1)))) return false;
    return w.radix == 0 || w.radix == 8 || w.radix == 16;
}

}  // namespace

// The wisdom entry for the problem, if any (no measurement).
bool wisdom_lookup(int d, const int64_t *n, fftu_dtype dtype, fftu_dir dir, const fftu_options &base, TuneChoice *t) {
    const std::string key = wisdom_key(d, n, dtype, dir, base.schedule, base.precision);
    std::lock_guard<std::mutex> lock(g_wisdom_mutex);
    auto it = g_wisdom.find(key);
    if (it == g_wisdom.end() || (int)it->second.p.size() != d) return false;
    for (int l = 0; l < d; ++l) t->p[l] = it->second.p[l];
    t->schedule = it->second.schedule ? it->second.schedule : base.schedule;
    t->tile = it->second.tile ? it->second.tile : base.tile;
    t->radix = it->second.radix ? it->second.radix : base.radix;
    return true;
}

// Fills `t` (p, and schedule / tile / radix where the caller left them open); returns true when
// tuning ran or wisdom answered, false when the caller should use the defaults.
bool autotune(int d, const int64_t *n, fftu_dtype dtype, fftu_dir dir, const fftu_options &base, TuneChoice *t) {
    const std::string key = wisdom_key(d, n, dtype, dir, base.schedule, base.precision);
    if (wisdom_lookup(d, n, dtype, dir, base, t)) return true;
    int64_t N = 1, pmax[FFTU_MAX_DIMS];
    for (int l = 0; l < d; ++l) {
        N *= n[l];
        int64_t q = 1;
        while (n[l] % ((2 * q) * (2 * q)) == 0) q *= 2;
        pmax[l] = q;
    }
    const size_t bytes = (size_t)N * (dtype == FFTU_C128 ? 16 : 8);
    void *in = nullptr, *out = nullptr;
    if (cudaMalloc(&in, bytes) != cudaSuccess || cudaMalloc(&out, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (in) cudaFree(in);
        return false;
    }
    cudaMemset(in, 0, bytes);

    fftu_options cur = base;
    cur.tune = 0;
    std::vector<int64_t> best_p;
    float best = -1.f;
    // 1. the grid: q on every axis, and q with the last (contiguous) axis at q / 2
    auto try_grid = [&](const std::vector<int64_t> &c) {
        const float ms = time_candidate(d, n, c.data(), dtype, dir, cur, in, out);
        if (ms >= 0.f && (best < 0.f || ms < best)) {
            best = ms;
            best_p = c;
        }
    };
    for (int64_t q = 1;; q *= 2) {
        std::vector<int64_t> c(d);
        bool grew = false;
        for (int l = 0; l < d; ++l) {
            c[l] = q < pmax[l] ? q : pmax[l];
            if (q <= pmax[l]) grew = true;
        }
        try_grid(c);
        if (d > 1 && c[d - 1] >= 2 && c[d - 1] == q) {
            std::vector<int64_t> h = c;
            h[d - 1] /= 2;
            if (h != c) try_grid(h);
        }
        if (!grew) break;
    }
    if (best_p.empty()) {
        cudaFree(in);
        cudaFree(out);
        return false;
    }
    // 2-4. schedule, tile, radix, each with the others at their best so far
    auto try_field = [&](int *field, std::initializer_list<int> values) {
        const int keep = *field;
        int best_v = keep;
        for (int v : values) {
            if (v == keep) continue;
            *field = v;
            const float ms = time_candidate(d, n, best_p.data(), dtype, dir, cur, in, out);
            if (ms >= 0.f && ms < best) {
                best = ms;
                best_v = v;
            }
        }
        *field = best_v;
    };
    if (base.schedule == FFTU_SCHED_AUTO && base.precision == FFTU_PREC_NATIVE)
        try_field(&cur.schedule, {FFTU_SCHED_GENERIC_A, FFTU_SCHED_GENERIC});
    if (base.tile == 0) {
        if (dtype == FFTU_C128) try_field(&cur.tile, {1024, 4096});
        else try_field(&cur.tile, {2048, 8192});
    }
    if (base.radix == 0 && base.precision == FFTU_PREC_NATIVE) try_field(&cur.radix, {16});
    cudaFree(in);
    cudaFree(out);
    for (int l = 0; l < d; ++l) t->p[l] = best_p[l];
    t->schedule = cur.schedule;
    t->tile = cur.tile;
    t->radix = cur.radix;
    Wise w;
    w.p = best_p;
    w.schedule = cur.schedule;
    w.tile = cur.tile;
    w.radix = cur.radix;
    std::lock_guard<std::mutex> lock(g_wisdom_mutex);
    g_wisdom[key] = w;
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
        std::fprintf(f, "fftu-wisdom-v2 %s", kv.first.c_str());
        for (size_t l = 0; l < kv.second.p.size(); ++l)
            std::fprintf(f, "%s%lld", l ? "," : " ", (long long)kv.second.p[l]);
        std::fprintf(f, " %d %d %d\n", kv.second.schedule, kv.second.tile, kv.second.radix);
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
    std::lock_guard<std::mutex> lock(fftu::g_wisdom_mutex);
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
        char tag[32], key[512], vals[256];
        int sched = 0, tile = 0, radix = 0;
        const int got = std::sscanf(line, "%31s %511s %255s %d %d %d", tag, key, vals, &sched, &tile, &radix);
        if (got < 3) continue;
        std::string k = key;
        if (std::strcmp(tag, "fftu-wisdom-v1") == 0) {
            // v1 keys carry no precision field: d:n:dtype:dir:sched:gpu -> d:n:dtype:dir:sched:0:gpu
            const size_t pos = k.rfind(':');
            if (pos == std::string::npos) continue;
            k.insert(pos, ":0");
            sched = tile = radix = 0;
        } else if (!(got == 6 && std::strcmp(tag, "fftu-wisdom-v2") == 0)) {
            continue;
        }
        fftu::Wise w;
        for (char *tok = std::strtok(vals, ","); tok; tok = std::strtok(nullptr, ",")) w.p.push_back(std::atoll(tok));
        w.schedule = sched;
        w.tile = tile;
        w.radix = radix;
        if (!fftu::valid_entry(k, w)) continue;  // never let a malformed line reach a plan
        fftu::g_wisdom[k] = w;
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

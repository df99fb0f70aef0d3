// lbm_tune.cu -- autotuner for the launch shape of the step kernels.
//
// Candidates are timed with CUDA events on the context stream in "dry" runs
// that read the current state and write the other buffer without making it
// current, so tuning never advances or alters the simulation.  The winner is
// applied to the context and cached in a small JSON file:
//   { "<device>|<physics>|<precision>|<geometry>": {"threads": 256, ...}, ... }
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "lbm_internal.h"

namespace {

using Entry = std::map<std::string, double>;
using Cache = std::map<std::string, Entry>;

void skip_ws(const std::string& s, size_t& i) {
    while (i < s.size() && (s[i] == ' ' || s[i] == '\n' || s[i] == '\r' || s[i] == '\t' || s[i] == ',')) ++i;
}

bool parse_string(const std::string& s, size_t& i, std::string& out) {
    skip_ws(s, i);
    if (i >= s.size() || s[i] != '"') return false;
    ++i;
    out.clear();
    while (i < s.size() && s[i] != '"') {
        if (s[i] == '\\' && i + 1 < s.size()) ++i;
        out += s[i++];
    }
    if (i >= s.size()) return false;
    ++i;
    return true;
}

bool expect(const std::string& s, size_t& i, char ch) {
    skip_ws(s, i);
    if (i >= s.size() || s[i] != ch) return false;
    ++i;
    return true;
}

// Reads the cache format written by save_cache; anything else yields an
// empty cache (the tuner then re-times and rewrites the file).
Cache load_cache(const char* path) {
    Cache c;
    if (!path) return c;
    std::ifstream f(path);
    if (!f) return c;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    size_t i = 0;
    if (!expect(s, i, '{')) return Cache();
    while (true) {
        skip_ws(s, i);
        if (i < s.size() && s[i] == '}') break;
        std::string key;
        if (!parse_string(s, i, key) || !expect(s, i, ':') || !expect(s, i, '{')) return Cache();
        Entry e;
        while (true) {
            skip_ws(s, i);
            if (i < s.size() && s[i] == '}') {
                ++i;
                break;
            }
            std::string k;
            if (!parse_string(s, i, k) || !expect(s, i, ':')) return Cache();
            skip_ws(s, i);
            char* end = nullptr;
            const double v = std::strtod(s.c_str() + i, &end);
            if (end == s.c_str() + i) return Cache();
            i = (size_t)(end - s.c_str());
            e[k] = v;
        }
        c[key] = e;
    }
    return c;
}

bool save_cache(const char* path, const Cache& c) {
    if (!path) return true;
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream f(tmp);
        if (!f) return false;
        f << "{\n";
        size_t k = 0;
        for (const auto& kv : c) {
            f << "  \"" << kv.first << "\": {";
            size_t j = 0;
            for (const auto& e : kv.second) {
                char num[64];
                std::snprintf(num, sizeof(num), "%.6g", e.second);
                f << "\"" << e.first << "\": " << num << (++j < kv.second.size() ? ", " : "");
            }
            f << "}" << (++k < c.size() ? ",\n" : "\n");
        }
        f << "}\n";
    }
    return std::rename(tmp.c_str(), path) == 0;
}

const char* phys_name(lbm_physics p) {
    return p == LBM_PHYS_FLUID ? "fluid" : (p == LBM_PHYS_MHD ? "mhd" : (p == LBM_PHYS_CGM ? "cgm" : "sc"));
}
const char* prec_name(lbm_precision p) {
    return p == LBM_FP64 ? "fp64" : (p == LBM_FP32 ? "fp32" : (p == LBM_FP16_SHIFTED ? "fp16" : "bf16"));
}

std::string cache_key(const lbm_ctx* c, const std::vector<long>& domain_sizes) {
    cudaDeviceProp prop;
    std::string dev = "gpu";
    if (cudaGetDeviceProperties(&prop, c->device) == cudaSuccess) dev = prop.name;
    char buf[256];
    if (!c->batch) {
        std::snprintf(buf, sizeof(buf), "%s|%s|%s|%dx%dx%d|p%u%s%s%s", dev.c_str(), phys_name(c->physics),
                      prec_name(c->prec), c->box.nx, c->box.ny, c->box.nz, c->box.periodic,
                      c->grid.wall_model == LBM_WALL_REGULARIZED ? "|reg" : "",
                      c->relax.moment_space == LBM_MOMENTS_RAW ? "|rm" : "", c->q == 27 ? "|q27" : "");
        return buf;
    }
    unsigned long long h = 1469598103934665603ull;  // FNV-1a over the domain sizes
    for (long v : domain_sizes) {
        h ^= (unsigned long long)v;
        h *= 1099511628211ull;
    }
    std::snprintf(buf, sizeof(buf), "%s|%s|%s|batch%zu|h%016llx", dev.c_str(), phys_name(c->physics),
                  prec_name(c->prec), domain_sizes.size(), h);
    return buf;
}

float time_dry_steps(lbm_ctx* c, long reps, cudaError_t* err) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = -1.f;
    cudaError_t e = cudaEventRecord(a, c->stream);
    if (e == cudaSuccess) e = lbm_internal_step(c, reps, true);
    if (e == cudaSuccess) e = cudaEventRecord(b, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *err = e;
    return ms;
}

}  // namespace

extern "C" lbm_status lbm_set_launch_shape(lbm_ctx* c, int variant, int threads, int stages, int ctas) {
    if (!c || c->batch || !c->owns) return LBM_ERR_ARG;
    if (variant == 3) {  // fused Shan-Chen step: 32 x 8 or 32 x 16 threads, `stages` planes per CTA
        if (c->physics != LBM_PHYS_SC) return LBM_ERR_UNSUPPORTED;
        if ((threads != 256 && threads != 512) || stages < 0 || stages > 4096) return LBM_ERR_ARG;
        if (threads == 512 && c->prec == LBM_FP64) return LBM_ERR_UNSUPPORTED;
        c->variant = 3;
        c->fused_threads = threads;
        c->zchunk = stages > 0 ? stages : 32;
        return LBM_OK;
    }
    if (threads < 32 || threads > 256 || threads % 32 != 0) return LBM_ERR_ARG;
    if (variant == 0 || variant == 2 || variant == 4) {
        if (variant == 2 && !(lbm::packed16_ok(c) && c->box.nx % 2 == 0)) return LBM_ERR_UNSUPPORTED;
        if (variant == 4 && !lbm::packed16_ok(c)) return LBM_ERR_UNSUPPORTED;
        if (variant == 4 && threads > lbm::ZPAIR_MAX_THREADS) return LBM_ERR_UNSUPPORTED;
        c->variant = variant;
        c->block_x = threads;
        return LBM_OK;
    }
    if (variant != 1) return LBM_ERR_ARG;
    if (ctas < 1 || stages < 2) return LBM_ERR_ARG;
    if (stages > lbm::fluid_tma_max_stages(c, ctas)) return LBM_ERR_UNSUPPORTED;
    c->variant = 1;
    c->block_x = threads;
    c->tma_stages = stages;
    c->tma_ctas = ctas;
    return LBM_OK;
}

extern "C" lbm_status lbm_get_launch_shape(const lbm_ctx* c, int* variant, int* threads, int* stages, int* ctas) {
    if (!c || c->batch) return LBM_ERR_ARG;
    if (variant) *variant = c->variant;
    if (threads) *threads = c->variant == 3 ? c->fused_threads : c->block_x;
    if (stages) *stages = c->variant == 1 ? c->tma_stages : (c->variant == 3 ? c->zchunk : 0);
    if (ctas) *ctas = c->variant == 1 ? c->tma_ctas : 0;
    return LBM_OK;
}

extern "C" lbm_status lbm_autotune(lbm_ctx* c, const char* cache_path, int force, double* mlups) {
    if (!c) return LBM_ERR_ARG;
    if (!c->owns) return LBM_ERR_UNSUPPORTED;
    std::vector<long> sizes;
    if (c->batch) {
        for (int d = 0;; ++d) {
            lbm_ctx* v = nullptr;
            if (lbm_batch_domain(c, d, &v) != LBM_OK) break;
            sizes.push_back(v->box.nx);
            sizes.push_back(v->box.ny);
            sizes.push_back(v->box.nz);
        }
    }
    const std::string key = cache_key(c, sizes);
    Cache cache = load_cache(cache_path);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    const double cells = (double)c->box.n;

    auto hit = cache.find(key);
    if (!force && hit != cache.end() && hit->second.count("threads")) {
        Entry& h = hit->second;
        const int threads = (int)h["threads"];
        if (c->batch) {
            const int cps = h.count("ctas_per_sm") ? (int)h["ctas_per_sm"] : 0;
            if (lbm::batch_apply_config(c, threads, cps) != cudaSuccess) return LBM_ERR_CUDA;
        } else {
            const int variant = h.count("variant") ? (int)h["variant"] : 0;
            const int stages = h.count("stages") ? (int)h["stages"] : 0;
            const int ctas = h.count("ctas") ? (int)h["ctas"] : 1;
            if (variant == 3 && c->physics == LBM_PHYS_SC) {
                c->variant = 3;
                c->fused_threads = threads;
                c->zchunk = stages > 0 ? stages : 32;
                if (mlups) *mlups = h.count("mlups") ? h["mlups"] : 0.0;
                return LBM_OK;
            }
            c->block_x = threads;
            if (variant == 1 && stages >= 2 && stages <= lbm::fluid_tma_max_stages(c, ctas)) {
                c->variant = 1;
                c->tma_stages = stages;
                c->tma_ctas = ctas;
            } else {
                c->variant = (variant == 2 && c->box.nx % 2 == 0) || variant == 4 ? variant : 0;
            }
        }
        if (mlups) *mlups = h.count("mlups") ? h["mlups"] : 0.0;
        return LBM_OK;
    }

    Entry best;
    double best_ms = 1e30;
    if (c->batch) {
        const long steps = 6;
        const int threads_c[] = {128, 256};
        const int cps_c[] = {1, 2, 3, 4, 0};
        for (int th : threads_c)
            for (int cps : cps_c) {
                float ms = 0.f;
                e = lbm::batch_time_config(c, th, cps, steps, &ms);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                const double per = ms / steps;
                if (per < best_ms) {
                    best_ms = per;
                    best = Entry{{"threads", (double)th}, {"ctas_per_sm", (double)cps}};
                }
            }
        if (best.empty()) return LBM_ERR_CUDA;
        if (lbm::batch_apply_config(c, (int)best["threads"], (int)best["ctas_per_sm"]) != cudaSuccess)
            return LBM_ERR_CUDA;
    } else {
        struct Cand {
            int variant, threads, stages, ctas;
        };
        std::vector<Cand> cands;
        for (int bx : {32, 64, 128, 256}) cands.push_back({0, bx, 0, 1});  // 32: small grids over all SMs
        if (lbm::packed16_ok(c)) {
            if (c->box.nx % 2 == 0)
                for (int bx : {128, 256}) cands.push_back({2, bx, 0, 1});
            for (int bx : {64, 128}) cands.push_back({4, bx, 0, 1});  // z-pairs: at most 128 threads
        }
        for (int ctas : {1, 2, 3, 4}) {
            const int smax = lbm::fluid_tma_max_stages(c, ctas);
            for (int st : {2, 3, 4, 6, 8})
                if (st <= smax) cands.push_back({1, c->block_x, st, ctas});
        }
        if (c->physics == LBM_PHYS_SC)
            for (int th : {256, 512})
                for (int lz : {16, 32, 64})
                    if (th == 256 || c->prec != LBM_FP64) cands.push_back({3, th, lz, 1});
        const int saved_bx = c->block_x, saved_var = c->variant, saved_st = c->tma_stages, saved_ct = c->tma_ctas;
        const int saved_ft = c->fused_threads, saved_lz = c->zchunk;
        for (const Cand& k : cands) {
            c->variant = k.variant;
            if (k.variant == 3) {
                c->fused_threads = k.threads;
                c->zchunk = k.stages;
            } else {
                c->block_x = k.threads;
            }
            c->tma_stages = k.variant == 1 && k.stages > 0 ? k.stages : saved_st;
            c->tma_ctas = k.ctas;
            float one = time_dry_steps(c, 1, &e);  // warm-up and size estimate
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            long reps = one > 0.f ? (long)(30.0f / one) : 10;
            if (reps < 3) reps = 3;
            if (reps > 200) reps = 200;
            const float ms = time_dry_steps(c, reps, &e);
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            const double per = ms / reps;
            if (per < best_ms) {
                best_ms = per;
                best = Entry{{"variant", (double)k.variant},
                             {"threads", (double)k.threads},
                             {"stages", (double)k.stages},
                             {"ctas", (double)k.ctas}};
            }
        }
        c->block_x = saved_bx;
        c->fused_threads = saved_ft;
        c->zchunk = saved_lz;
        if (best.empty()) {
            c->variant = saved_var;
            c->tma_stages = saved_st;
            c->tma_ctas = saved_ct;
            return LBM_ERR_CUDA;
        }
        c->variant = (int)best["variant"];
        if (c->variant == 3) {
            c->fused_threads = (int)best["threads"];
            c->zchunk = (int)best["stages"];
        } else {
            c->block_x = (int)best["threads"];
        }
        if (c->variant == 1) {
            c->tma_stages = (int)best["stages"];
            c->tma_ctas = (int)best["ctas"];
        }
    }
    best["mlups"] = cells / (best_ms * 1e-3) / 1e6;
    if (mlups) *mlups = best["mlups"];
    cache[key] = best;
    if (!save_cache(cache_path, cache)) {
        c->err = "autotune: could not write the cache file";
    }
    return LBM_OK;
}

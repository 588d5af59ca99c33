// Batched X-engine: many independent sub-arrays (different numbers of inputs,
// channels and spectra) correlated by ONE persistent tensor-core launch, replayed
// from a captured CUDA graph.
//
// Host runtime (this file):
//   planner   every (sub-array, channel pack, lower-triangle tile) work item is
//             costed by its spectra and spread over one CTA per SM by longest-
//             processing-time-first assignment; ties keep (sub, channel) order so
//             that CTAs running together share channel data in L2.
//   tuner     for each sub-array, the tile shape -- how many channels share one
//             128-row tile (1, 2 or 4, for sub-arrays of <= 128, 64 or 32 inputs)
//             -- is timed on the GPU and the fastest kept; choices are cached in a
//             JSON file keyed by (inputs, spectra).
//   graph     the launch is captured once into a CUDA graph and replayed; a new
//             plan (after tuning) invalidates it.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <new>
#include <queue>
#include <sstream>
#include <string>
#include <vector>

#include "internal.h"

namespace corr {
namespace {

struct Plan {
    std::vector<int4> items;
    std::vector<int> cta_off;
};

int max_cpt(int n_in) { return n_in <= 32 ? 4 : (n_in <= 64 ? 2 : 1); }

// Items of one sub-array with a given channel packing.
void sub_items(int s, const corr_sub_desc &d, int cpt, std::vector<std::pair<long long, int4>> &out) {
    if (cpt > 1) {
        for (int c = 0; c < d.n_chan; c += cpt) out.push_back({(long long)d.n_spectra, make_int4(s, c, 0, 0)});
        return;
    }
    const int nb = (d.n_in + 127) / 128;
    for (int c = 0; c < d.n_chan; ++c)
        for (int bi = 0; bi < nb; ++bi)
            for (int bj = 0; bj <= bi; ++bj)
                out.push_back({(long long)d.n_spectra, make_int4(s, c, bi | (bj << 16), 0)});
}

// Longest-processing-time-first assignment of the items to `grid` CTAs.
Plan make_plan(const std::vector<corr_sub_desc> &subs, const std::vector<int> &cpt, const std::vector<int> &which,
               int grid) {
    std::vector<std::pair<long long, int4>> all;
    for (int s : which) sub_items(s, subs[(size_t)s], cpt[(size_t)s], all);
    std::stable_sort(all.begin(), all.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    if ((int)all.size() < grid) grid = std::max<int>(1, (int)all.size());
    std::vector<std::vector<int4>> per(grid);
    using L = std::pair<long long, int>;
    std::priority_queue<L, std::vector<L>, std::greater<L>> heap;
    for (int g = 0; g < grid; ++g) heap.push({0, g});
    for (const auto &it : all) {
        L top = heap.top();
        heap.pop();
        per[(size_t)top.second].push_back(it.second);
        heap.push({top.first + it.first, top.second});
    }
    Plan p;
    p.cta_off.push_back(0);
    for (auto &v : per) {
        p.items.insert(p.items.end(), v.begin(), v.end());
        p.cta_off.push_back((int)p.items.size());
    }
    return p;
}

std::string cache_key(const corr_sub_desc &d) {
    return std::to_string(d.n_in) + "," + std::to_string(d.n_spectra);
}

// Minimal reader/writer for the tuning cache: {"n_in,K": cpt, ...}
std::map<std::string, int> read_cache(const char *path) {
    std::map<std::string, int> m;
    if (!path) return m;
    std::ifstream f(path);
    if (!f) return m;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string t = ss.str();
    size_t i = 0;
    while ((i = t.find('"', i)) != std::string::npos) {
        const size_t j = t.find('"', i + 1);
        if (j == std::string::npos) break;
        const std::string key = t.substr(i + 1, j - i - 1);
        const size_t c = t.find(':', j);
        if (c == std::string::npos) break;
        m[key] = std::atoi(t.c_str() + c + 1);
        i = t.find_first_of(",}", c);
        if (i == std::string::npos) break;
    }
    return m;
}

void write_cache(const char *path, const std::map<std::string, int> &m) {
    if (!path) return;
    std::ofstream f(path);
    f << "{";
    bool first = true;
    for (const auto &kv : m) {
        f << (first ? "" : ", ") << "\"" << kv.first << "\": " << kv.second;
        first = false;
    }
    f << "}\n";
}

}  // namespace
}  // namespace corr

struct corr_batch_s {
    std::vector<corr_sub_desc> subs;
    std::vector<int> cpt;  // tuned channels per tile, per sub-array
    int device = 0, n_sm = 0;
    void *d_tmaps = nullptr;  // [n_sub][3] tensor maps (box heights 128, 64, 32)
    corr::BatchSub *d_subs = nullptr;
    int4 *d_items = nullptr;
    int *d_cta_off = nullptr;
    size_t items_cap = 0, off_cap = 0;
    int grid = 0;
    int *d_status = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool planned = false;
};

namespace corr {
namespace {

// Upload the per-sub descriptors (with the chosen packing) and a plan.
corr_status upload(corr_batch_s &b, const Plan &p) {
    std::vector<BatchSub> hs(b.subs.size());
    for (size_t s = 0; s < b.subs.size(); ++s) {
        const corr_sub_desc &d = b.subs[s];
        hs[s] = BatchSub{d.vis, (long long)d.n_in * (d.n_in + 1) / 2, d.n_in, d.n_spectra, d.n_chan, b.cpt[s]};
    }
    CORR_CUDA_TRY(cudaMemcpy(b.d_subs, hs.data(), sizeof(BatchSub) * hs.size(), cudaMemcpyHostToDevice));
    if (p.items.size() > b.items_cap) {
        cudaFree(b.d_items);
        b.d_items = nullptr;
        b.items_cap = 0;
        if (cudaMalloc(&b.d_items, sizeof(int4) * p.items.size()) != cudaSuccess) {
            cudaGetLastError();
            return CORR_ENOMEM;
        }
        b.items_cap = p.items.size();
    }
    if (p.cta_off.size() > b.off_cap) {
        cudaFree(b.d_cta_off);
        b.d_cta_off = nullptr;
        b.off_cap = 0;
        if (cudaMalloc(&b.d_cta_off, sizeof(int) * p.cta_off.size()) != cudaSuccess) {
            cudaGetLastError();
            return CORR_ENOMEM;
        }
        b.off_cap = p.cta_off.size();
    }
    CORR_CUDA_TRY(cudaMemcpy(b.d_items, p.items.data(), sizeof(int4) * p.items.size(), cudaMemcpyHostToDevice));
    CORR_CUDA_TRY(cudaMemcpy(b.d_cta_off, p.cta_off.data(), sizeof(int) * p.cta_off.size(), cudaMemcpyHostToDevice));
    b.grid = (int)p.cta_off.size() - 1;
    return CORR_OK;
}

// The tensor map a sub-array's items use depends on its packing (box height 128 / cpt);
// point each sub's slot at the right one by reordering: slot s holds the map in use.
corr_status set_maps(corr_batch_s &b) {
    std::vector<unsigned char> maps(128 * b.subs.size());
    for (size_t s = 0; s < b.subs.size(); ++s) {
        const corr_sub_desc &d = b.subs[s];
        corr_status st = tma_encode_planar(maps.data() + 128 * s, d.planes, d.n_in, d.n_chan, d.n_spectra, 2,
                                           128 / b.cpt[s]);
        if (st != CORR_OK) return st;
    }
    CORR_CUDA_TRY(cudaMemcpy(b.d_tmaps, maps.data(), maps.size(), cudaMemcpyHostToDevice));
    return CORR_OK;
}

corr_status plan_all(corr_batch_s &b) {
    std::vector<int> all(b.subs.size());
    for (size_t s = 0; s < all.size(); ++s) all[s] = (int)s;
    corr_status st = set_maps(b);
    if (st != CORR_OK) return st;
    st = upload(b, make_plan(b.subs, b.cpt, all, b.n_sm));
    if (st != CORR_OK) return st;
    if (b.exec) {
        cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
    }
    b.planned = true;
    return CORR_OK;
}

}  // namespace
}  // namespace corr

using corr::Plan;

extern "C" {

corr_status corr_batch_create(int32_t n_sub, const corr_sub_desc *subs, const corr_opts *opts, corr_batch_t **out) {
    if (!out) return CORR_EINVAL;
    *out = nullptr;
    if (n_sub <= 0 || !subs) return CORR_EINVAL;
    // the batched X-engine is the exact INT8 one on tensor cores, fed planar FP16 codes
    int device = -1;
    if (opts) {
        if (opts->precision != CORR_PREC_INT8 || opts->xengine == CORR_XENG_CUDACORE ||
            (opts->flags & ~CORR_FLAG_PLANAR) != 0) {
            corr::set_error_text("corr_batch_create: only INT8 on the tensor-core X-engine (planar codes) is batched");
            return CORR_EUNSUPPORTED;
        }
        if (opts->xengine < CORR_XENG_AUTO || opts->xengine > CORR_XENG_TCGEN05) return CORR_EINVAL;
        device = opts->device;
    }
    for (int s = 0; s < n_sub; ++s) {
        const corr_sub_desc &d = subs[s];
        if (d.n_in <= 0 || d.n_in > 65535 || d.n_chan <= 0 || d.n_spectra <= 0 || d.reserved != 0 || !d.planes || !d.vis)
            return CORR_EINVAL;
        if ((reinterpret_cast<uintptr_t>(d.planes) & 15u) || (reinterpret_cast<uintptr_t>(d.vis) & 7u))
            return CORR_EINVAL;
        if (d.n_spectra % 8 != 0) return CORR_EUNSUPPORTED;
        // INT32 guard: |V| <= n_spectra * 2 * 128^2 (int8 codes include -128)
        if ((int64_t)d.n_spectra * 2 * 128 * 128 >= (int64_t)1 << 31) return CORR_EOVERFLOW;
    }
    if (device < 0 && cudaGetDevice(&device) != cudaSuccess) {
        corr::set_cuda_error(cudaGetLastError(), "cudaGetDevice");
        return CORR_ECUDA;
    }
    corr::DeviceGuard dg(device);
    if (!dg.ok) {
        corr::set_cuda_error(cudaGetLastError(), "cudaSetDevice");
        return CORR_ECUDA;
    }
    corr_batch_s *b = new (std::nothrow) corr_batch_s();
    if (!b) return CORR_ENOMEM;
    b->subs.assign(subs, subs + n_sub);
    b->cpt.assign((size_t)n_sub, 1);
    b->device = device;
    bool ok = 
              cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device) == cudaSuccess &&
              cudaMalloc(&b->d_tmaps, 128 * (size_t)n_sub) == cudaSuccess &&
              cudaMalloc(&b->d_subs, sizeof(corr::BatchSub) * (size_t)n_sub) == cudaSuccess &&
              cudaMalloc(&b->d_status, sizeof(int)) == cudaSuccess &&
              cudaMemset(b->d_status, 0, sizeof(int)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    corr_status st = ok ? corr::plan_all(*b) : CORR_ENOMEM;
    if (st != CORR_OK) {
        cudaGetLastError();
        corr_batch_destroy(b);
        return st;
    }
    *out = b;
    return CORR_OK;
}

corr_status corr_batch_destroy(corr_batch_t *b) {
    if (!b) return CORR_OK;
    corr::DeviceGuard dg(b->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaFree(b->d_tmaps);
    cudaFree(b->d_subs);
    cudaFree(b->d_items);
    cudaFree(b->d_cta_off);
    cudaFree(b->d_status);
    delete b;
    return CORR_OK;
}

int32_t corr_batch_channels_per_tile(const corr_batch_t *b, int32_t sub) {
    if (!b || sub < 0 || sub >= (int32_t)b->subs.size()) return -1;
    return b->cpt[(size_t)sub];
}

corr_status corr_batch_run(corr_batch_t *b, void *stream) {
    if (!b) return CORR_EINVAL;
    corr::DeviceGuard dg(b->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!b->exec) {
        // capture the single persistent launch on a private stream, then replay it
        cudaGraph_t g = nullptr;
        CORR_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        corr_status s = corr::launch_xengine_tma_batch(b->d_tmaps, b->d_subs, b->d_items, b->d_cta_off, b->grid,
                                                       b->d_status, b->cap_stream);
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
        if (s != CORR_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) {
            corr::set_cuda_error(e, "cudaStreamEndCapture");
            return CORR_ECUDA;
        }
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            corr::set_cuda_error(e, "cudaGraphInstantiate");
            b->exec = nullptr;
            return CORR_ECUDA;
        }
    }
    CORR_CUDA_TRY(cudaGraphLaunch(b->exec, st));
    return CORR_OK;
}

corr_status corr_batch_check_status(corr_batch_t *b, void *stream) {
    if (!b) return CORR_EINVAL;
    corr::DeviceGuard dg(b->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int v = 0;
    CORR_CUDA_TRY(cudaMemcpyAsync(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CORR_CUDA_TRY(cudaStreamSynchronize(st));
    if (v != 0) {
        CORR_CUDA_TRY(cudaMemset(b->d_status, 0, sizeof(int)));
        return (corr_status)v;
    }
    return CORR_OK;
}

corr_status corr_batch_tune(corr_batch_t *b, const char *cache_path, void *stream) {
    if (!b) return CORR_EINVAL;
    corr::DeviceGuard dg(b->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::map<std::string, int> cache = corr::read_cache(cache_path);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CORR_CUDA_TRY(cudaEventCreate(&e0));
    CORR_CUDA_TRY(cudaEventCreate(&e1));
    corr_status result = CORR_OK;
    for (size_t s = 0; s < b->subs.size() && result == CORR_OK; ++s) {
        const corr_sub_desc &d = b->subs[s];
        const std::string key = corr::cache_key(d);
        auto hit = cache.find(key);
        if (hit != cache.end() && hit->second >= 1 && hit->second <= corr::max_cpt(d.n_in)) {
            b->cpt[s] = hit->second;
            continue;
        }
        // time each valid packing on this sub-array alone (a window of <= 64 channels)
        corr_sub_desc w = d;
        w.n_chan = std::min(d.n_chan, 64);
        std::vector<corr_sub_desc> one{w};
        float best_ms = 1e30f;
        int best = 1;
        for (int cpt = 1; cpt <= corr::max_cpt(d.n_in) && result == CORR_OK; cpt *= 2) {
            corr_batch_s tmp;
            tmp.subs = one;
            tmp.cpt = {cpt};
            tmp.n_sm = b->n_sm;
            tmp.d_tmaps = b->d_tmaps;  // borrow the device buffers (slot 0)
            tmp.d_subs = b->d_subs;
            tmp.d_status = b->d_status;
            result = corr::set_maps(tmp);
            if (result != CORR_OK) break;
            result = corr::upload(tmp, corr::make_plan(tmp.subs, tmp.cpt, {0}, b->n_sm));
            float ms = 0.f;
            for (int rep = 0; rep < 3 && result == CORR_OK; ++rep) {
                cudaEventRecord(e0, st);
                result = corr::launch_xengine_tma_batch(tmp.d_tmaps, tmp.d_subs, tmp.d_items, tmp.d_cta_off,
                                                        tmp.grid, tmp.d_status, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    corr::set_cuda_error(cudaGetLastError(), "corr_batch_tune");
                    result = CORR_ECUDA;
                }
                if (result == CORR_OK && rep > 0) {
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms += t;
                }
            }
            cudaFree(tmp.d_items);
            cudaFree(tmp.d_cta_off);
            tmp.d_tmaps = nullptr;
            tmp.d_subs = nullptr;
            tmp.d_status = nullptr;
            if (result == CORR_OK && ms < best_ms) {
                best_ms = ms;
                best = cpt;
            }
        }
        b->cpt[s] = best;
        cache[key] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (result != CORR_OK) return result;
    corr::write_cache(cache_path, cache);
    return corr::plan_all(*b);
}

}  // extern "C"

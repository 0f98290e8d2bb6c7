// Launch-shape autotuner: for each bucket width of an ensemble, time candidate
// (warps per block, paths per block, staged sub-chunk, node-group width, private
// per-warp tiles or not) of the
// forward kernel and candidate work-item sizes of the fused forward+adjoint
// kernel on the caller's data, keep the fastest, and optionally merge them into
// a JSON cache keyed by (width, log2 F, log2 M).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <fstream>
#include <map>
#include <sstream>

#include "qts_internal.h"

namespace qts {

cudaError_t launch_bwd_bucket(const qts_ensemble* e, const Bucket& b, const float* X,
                              const float* grad, int64_t M, int F, const QuadF& q, double* g_val,
                              double* g_slot, double* phi, const Tune& tn, cudaStream_t st);
void batch_forget(const qts_ensemble* e);

static int ilog2(int64_t v) {
    int l = 0;
    while (v > 1) { v >>= 1; ++l; }
    return l;
}

static std::string cache_key(int D, int F, int64_t M) {
    return std::to_string(D) + "|" + std::to_string(ilog2(F)) + "|" + std::to_string(ilog2(std::max<int64_t>(M, 1)));
}

// The cache file is a flat JSON object:
//   {"D|logF|logM": [warps, paths, sub, np, bpaths, priv], ...}
static std::map<std::string, Tune> read_cache(const char* path) {
    std::map<std::string, Tune> out;
    std::ifstream in(path);
    if (!in) return out;
    std::stringstream ss;
    ss << in.rdbuf();
    const std::string s = ss.str();
    size_t i = 0;
    while ((i = s.find('"', i)) != std::string::npos) {
        const size_t j = s.find('"', i + 1);
        if (j == std::string::npos) break;
        const std::string key = s.substr(i + 1, j - i - 1);
        const size_t lb = s.find('[', j), rb = s.find(']', j);
        if (lb == std::string::npos || rb == std::string::npos) break;
        int v[6] = {0, 0, 0, 0, 0, 0};
        std::stringstream vs(s.substr(lb + 1, rb - lb - 1));
        std::string tok;
        int k = 0;
        while (k < 6 && std::getline(vs, tok, ',')) v[k++] = std::atoi(tok.c_str());
        if (k == 6) out[key] = Tune{v[0], v[1], v[2], v[3], v[4], v[5]};
        i = rb + 1;
    }
    return out;
}

static void write_cache(const char* path, const std::map<std::string, Tune>& m) {
    std::ofstream o(std::string(path) + ".tmp");
    o << "{\n";
    size_t n = 0;
    for (const auto& kv : m) {
        const Tune& t = kv.second;
        o << "  \"" << kv.first << "\": [" << t.warps << ", " << t.paths << ", " << t.sub << ", " << t.np
          << ", " << t.bpaths << ", " << t.priv << "]" << (++n < m.size() ? "," : "") << "\n";
    }
    o << "}\n";
    o.close();
    std::rename((std::string(path) + ".tmp").c_str(), path);
}

template <typename F>
static float time_ms(F&& fn, cudaStream_t st, int reps) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    fn();  // warm-up
    std::vector<float> ts;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a, st);
        fn();
        cudaEventRecord(b, st);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        ts.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
}

}  // namespace qts

using namespace qts;

extern "C" qts_status qts_autotune(qts_ensemble* e, const float* X, int64_t M, int32_t F,
                                   const char* cache_path, qts_stream_t stream) {
    qts_status st = check_call(e, X, M, F, 8);
    if (st != QTS_OK) return st;
    if (M == 0) return QTS_OK;
    if (e->flags & QTS_FLAG_FP64) return fail(QTS_ERR_UNSUPPORTED, "autotuning applies to the FP32 kernels");
    cudaStream_t s = (cudaStream_t)stream;
    std::map<std::string, Tune> cache;
    if (cache_path) cache = read_cache(cache_path);
    const int64_t Mt = std::min<int64_t>(M, 4096);  // tune on a leading slice of the samples
    QuadF qf;
    QuadD qd;
    make_quad(8, &qf, &qd);
    double* phi = nullptr;
    float* grad = nullptr;
    // the FP32 forward and adjoint run on the pair tables
    st = ensure_batch_tables(e);
    if (st != QTS_OK) return st;
    const Prepared& P = e->bprep;
    cudaError_t ce = cudaMalloc(&phi, sizeof(double) * Mt * (F + 1));
    if (ce == cudaSuccess) ce = cudaMalloc(&grad, sizeof(float) * Mt * (F + 1));
    if (ce == cudaSuccess) ce = cudaMemsetAsync(grad, 0, sizeof(float) * Mt * (F + 1), s);
    if (ce != cudaSuccess) {
        cudaFree(phi);
        cudaFree(grad);
        return cuda_fail(ce, "autotune scratch");
    }
    st = ensure_workspace(e, sizeof(double) * (size_t)(4 + 2 * P.n_paths + P.n_slots));
    if (st != QTS_OK) {
        cudaFree(phi);
        cudaFree(grad);
        return st;
    }
    double* g_val = (double*)e->d_work + 4;
    double* g_slot = g_val + 2 * P.n_paths;
    for (int D = 1; D <= kMaxD; ++D) {
        const Bucket* bf = nullptr;
        for (const Bucket& b : P.buckets)
            if (b.D == D) bf = &b;
        const Bucket* bb = bf;
        if (!bf) continue;
        const std::string key = cache_key(D, F, M);
        auto it = cache.find(key);
        if (it != cache.end()) {
            const Tune keep = e->tune[D];  // the batched-launch tuner's choices stay
            e->tune[D] = it->second;
            e->tune[D].bt_paths = keep.bt_paths;
            e->tune[D].bt_mode = keep.bt_mode;
            e->tune[D].bt_occ = keep.bt_occ;
            continue;
        }
        Tune best = e->tune[D];
        float best_ms = 1e30f;
        const int nps[3] = {8, 4, 2};
        for (int np : nps) {
            if (!bf) break;
            if ((np == 8 && D > 8) || (np == 4 && D > 24)) continue;
            for (int warps : {2, 4, 8}) {
                for (int paths : {128, 512, 2048}) {
                    for (int sub : {16, 32}) {
                      for (int priv : {1, 2, 0}) {
                        Tune t = best;
                        t.np = np;
                        t.warps = warps;
                        t.paths = paths;
                        t.sub = sub;
                        t.priv = priv;
                        cudaError_t le = cudaSuccess;
                        const float ms = time_ms([&] {
                            le = launch_fwd_bucket(e, *bf, X, Mt, F, qf, qd, phi, t, s);
                        }, s, 3);
                        if (le == cudaSuccess && ms < best_ms) {
                            best_ms = ms;
                            best = t;
                        }
                        cudaGetLastError();
                      }
                    }
                }
            }
        }
        // work-item size of the fused forward + adjoint pass (batched launches)
        float best_b = 1e30f;
        for (int paths : {32, 64, 128, 256, 512}) {
            if (!bb) break;
            Tune t = best;
            t.paths = paths;
            t.sub = 16;
            t.warps = 4;
            cudaError_t le = cudaSuccess;
            const float ms = time_ms([&] {
                le = launch_bwd_bucket(e, *bb, X, grad, Mt, F, qf, g_val, g_slot, phi, t, s);
            }, s, 3);
            if (le == cudaSuccess && ms < best_b) {
                best_b = ms;
                best.bpaths = paths;
            }
            cudaGetLastError();
        }
        e->tune[D] = best;
        cache[key] = best;
    }
    ce = cudaStreamSynchronize(s);
    cudaFree(phi);
    cudaFree(grad);
    if (ce != cudaSuccess) return cuda_fail(ce, "autotune");
    e->tuned = true;
    ++e->tune_gen;
    batch_forget(e);
    if (cache_path) write_cache(cache_path, cache);
    return QTS_OK;
}

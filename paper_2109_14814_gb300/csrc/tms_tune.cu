// Autotuner: picks the parameters the paper leaves to the implementation -- the
// grid cell size (Sec. 6.2.1 asks only for cells wider than the widest quad),
// the face level, the broad-phase level (faces or patches in the grid) and the
// bounds-pass tile shape -- by timing them on the caller's meshes, and keeps the
// choice in a text file read back by later searches (tms_params.autotune_cache).
//
// One pair: every setting of a small grid is timed with tms_search.
// A batch of uneven pairs (the continuation sweep): the settings that shape
// the whole launch sequence (face level, patch level, bounds-pass tile) are
// timed on the whole batch; then the cell multiplier is chosen per size class
// -- pairs grouped by their quad count, a class per factor of four -- by
// coordinate descent, each class's candidates timed on the whole batch with
// the other classes at their current choice, since the batch runs as one
// launch sequence.  Results are identical for every setting.
//
// Cache lines (text, one per key; the last line for a key wins):
//   G|<device>|pairs=<n>|sizes=<hash of every N, M>|<flags> fl patch bf tr cm ms
//   C|<device>|class=<c>|<flags> cm
// <flags> = prec/filter/narrow/moller of the search.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tms_common.cuh"

namespace {

std::mutex g_tune_mu;
// resolved cache lookups: (path, batch key) -> settings, read once per process
struct Resolved {
    bool found = false;
    int face_level = 1, patch = 1, block_faces = 128, tile_rows = 4;
    float cell_mult = 1.0625f;
    std::vector<float> cm;
};
std::map<std::string, Resolved> g_memo;

std::string device_name() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string k = prop.name;
    for (char &c : k)
        if (c == ' ' || c == '|') c = '_';
    return k;
}

std::string flags_key(const tms_params &b) {
    char buf[96];
    snprintf(buf, sizeof(buf), "prec=%d|filter=%d|narrow=%d|moller=%d", b.precision, b.cell_filter,
             b.narrow_filter, b.moller);
    return buf;
}

unsigned long long pair_quads(tms_mesh A, tms_mesh B) {
    tms::MeshDev a, b;
    int d;
    tms::mesh_view(A, &a, &d);
    tms::mesh_view(B, &b, &d);
    return (unsigned long long)a.nqi * a.nqk + (unsigned long long)b.nqi * b.nqk;
}

// size class: a factor of four in the pair's quad count
int size_class(tms_mesh A, tms_mesh B) {
    const unsigned long long q = std::max(pair_quads(A, B), 1ULL);
    int l = 0;
    while ((1ULL << (l + 1)) <= q) ++l;
    return l / 2;
}

std::string batch_key(const tms_mesh *A, const tms_mesh *B, int nPairs, const tms_params &base) {
    unsigned long long h = 1469598103934665603ULL;
    for (int i = 0; i < nPairs; ++i) {
        tms::MeshDev a, b;
        int d;
        tms::mesh_view(A[i], &a, &d);
        tms::mesh_view(B[i], &b, &d);
        const unsigned long long v[4] = {(unsigned long long)a.N, (unsigned long long)a.M,
                                         (unsigned long long)b.N, (unsigned long long)b.M};
        for (unsigned long long x : v) { h ^= x; h *= 1099511628211ULL; }
    }
    char buf[96];
    snprintf(buf, sizeof(buf), "|pairs=%d|sizes=%016llx|", nPairs, (unsigned long long)h);
    return "G|" + device_name() + buf + flags_key(base);
}

std::string class_key(int c, const tms_params &base) {
    return "C|" + device_name() + "|class=" + std::to_string(c) + "|" + flags_key(base);
}

// every line of the cache file as (key, rest)
std::vector<std::pair<std::string, std::string>> read_cache(const char *path) {
    std::vector<std::pair<std::string, std::string>> out;
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f) return out;
    char line[1024];
    while (fgets(line, sizeof(line), f)) {
        char k[600];
        int used = 0;
        if (sscanf(line, "%599s%n", k, &used) == 1) out.emplace_back(k, std::string(line + used));
    }
    fclose(f);
    return out;
}

Resolved resolve(const tms_mesh *A, const tms_mesh *B, int nPairs, const tms_params &base,
                 const char *path) {
    Resolved r;
    const std::string bk = batch_key(A, B, nPairs, base);
    std::map<std::string, float> class_cm;
    for (auto &kv : read_cache(path)) {
        if (kv.first == bk) {
            int fl, pa, bf, tr;
            float cm;
            double ms;
            if (sscanf(kv.second.c_str(), "%d %d %d %d %f %lf", &fl, &pa, &bf, &tr, &cm, &ms) == 6) {
                r.found = true;
                r.face_level = fl;
                r.patch = pa;
                r.block_faces = bf;
                r.tile_rows = tr;
                r.cell_mult = cm;
            }
        } else if (kv.first.compare(0, 2, "C|") == 0) {
            float cm;
            if (sscanf(kv.second.c_str(), "%f", &cm) == 1) class_cm[kv.first] = cm;
        }
    }
    if (!r.found) return r;
    bool any = false;
    std::vector<float> cm(nPairs, r.cell_mult);
    for (int i = 0; i < nPairs; ++i) {
        auto it = class_cm.find(class_key(size_class(A[i], B[i]), base));
        if (it != class_cm.end()) {
            cm[i] = it->second;
            any = true;
        }
    }
    if (any) r.cm = cm;
    return r;
}

void append_lines(const char *path, const std::vector<std::string> &lines) {
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    for (auto &l : lines) fprintf(f, "%s\n", l.c_str());
    fclose(f);
}

}  // namespace

namespace tms {

bool tune_lookup(const tms_mesh *A, const tms_mesh *B, int nPairs, const char *path, tms_params *p,
                 std::vector<float> *cm_pair) {
    if (!path) return false;
    const std::string mk = std::string(path) + "\n" + batch_key(A, B, nPairs, *p);
    Resolved r;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_memo.find(mk);
        if (it == g_memo.end()) it = g_memo.emplace(mk, resolve(A, B, nPairs, *p, path)).first;
        r = it->second;
    }
    if (!r.found) return false;
    p->face_level = r.face_level;
    p->patch = r.patch;
    p->block_faces = r.block_faces;
    p->tile_rows = r.tile_rows;
    p->cell_mult = r.cell_mult;
    *cm_pair = r.cm;
    return true;
}

}  // namespace tms

extern "C" tms_status tms_autotune(const tms_mesh *A, const tms_mesh *B, int nPairs,
                                   const tms_params *base, tms_params *best, const char *cache_path,
                                   double *best_ms, void *stream) {
    if (!A || !B || nPairs <= 0 || !best) return TMS_ERR_ARG;
    for (int i = 0; i < nPairs; ++i) {
        tms::MeshDev v;
        int d;
        if (tms::mesh_view(A[i], &v, &d) != TMS_OK || tms::mesh_view(B[i], &v, &d) != TMS_OK)
            return TMS_ERR_ARG;
    }
    tms_params p0;
    tms_params_default(&p0);
    if (base) p0 = *base;
    p0.timing = 0;
    p0.autotune_cache = nullptr;
    {
        // answered from the cache when it holds this batch
        tms_params q = p0;
        std::vector<float> cm;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        Resolved r = cache_path ? resolve(A, B, nPairs, p0, cache_path) : Resolved();
        if (r.found) {
            q.face_level = r.face_level;
            q.patch = r.patch;
            q.block_faces = r.block_faces;
            q.tile_rows = r.tile_rows;
            q.cell_mult = r.cell_mult;
            *best = q;
            if (best_ms) {
                const std::string bk = batch_key(A, B, nPairs, p0);
                for (auto &kv : read_cache(cache_path))
                    if (kv.first == bk) {
                        int fl, pa, bf, tr;
                        float c;
                        double ms;
                        if (sscanf(kv.second.c_str(), "%d %d %d %d %f %lf", &fl, &pa, &bf, &tr, &c, &ms) == 6)
                            *best_ms = ms;
                    }
            }
            return TMS_OK;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    long long n = 0;
    long long cap = 1 << 16;
    tms_hit *out = nullptr;
    long long *offs = nullptr;
    if (cudaMalloc((void **)&out, cap * sizeof(tms_hit)) != cudaSuccess) return TMS_ERR_CUDA;
    if (cudaMalloc((void **)&offs, (nPairs + 1) * sizeof(long long)) != cudaSuccess) {
        cudaFree(out);
        return TMS_ERR_CUDA;
    }
    std::vector<float> none;
    auto run = [&](const tms_params &p, const std::vector<float> &cm) -> tms_status {
        return tms::search_with_cm(A, B, nPairs, p, cm, out, cap, nPairs > 1 ? offs : nullptr, &n, stream);
    };
    tms_status s = run(p0, none);
    if (s == TMS_ERR_CAPACITY && n > cap) {
        cudaFree(out);
        cap = n + 1024;
        if (cudaMalloc((void **)&out, cap * sizeof(tms_hit)) != cudaSuccess) {
            cudaFree(offs);
            return TMS_ERR_CUDA;
        }
        s = run(p0, none);
    }
    if (s != TMS_OK) {
        cudaFree(out);
        cudaFree(offs);
        return s;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // median of three timed runs after one warm-up (plan, capture, growth)
    auto timed = [&](const tms_params &p, const std::vector<float> &cm) -> double {
        if (run(p, cm) != TMS_OK) return 1e300;
        std::vector<float> ts;
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0, st);
            const tms_status rs = run(p, cm);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            if (rs != TMS_OK) return 1e300;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ts.push_back(ms);
        }
        tms_release_workspace(stream);   // keep only one trial plan alive
        std::sort(ts.begin(), ts.end());
        return ts[1];
    };
    // the settings of the whole launch sequence
    const int levels[3][2] = {{1, 1}, {1, 0}, {0, 0}};   // (face_level, patch)
    const int shapes[3][2] = {{128, 4}, {64, 4}, {128, 8}};
    const float mults[3] = {1.0625f, 1.5f, 2.5f};
    double bestt = 1e300;
    tms_params bp = p0;
    for (auto &lv : levels)
        for (auto &sh : shapes)
            for (int m = 0; m < (nPairs == 1 ? 3 : 1); ++m) {
                tms_params p = p0;
                p.face_level = lv[0];
                p.patch = lv[1];
                p.block_faces = sh[0];
                p.tile_rows = sh[1];
                p.cell_mult = nPairs == 1 ? mults[m] : p0.cell_mult;
                const double t = timed(p, none);
                if (t < bestt) {
                    bestt = t;
                    bp = p;
                }
            }
    // per size class: the cell multiplier, by coordinate descent (batches)
    std::vector<float> cm;
    std::map<int, float> class_best;
    if (nPairs > 1 && bestt < 1e300) {
        std::map<int, unsigned long long> weight;
        std::vector<int> cls(nPairs);
        for (int i = 0; i < nPairs; ++i) {
            cls[i] = size_class(A[i], B[i]);
            weight[cls[i]] += pair_quads(A[i], B[i]);
        }
        std::vector<std::pair<unsigned long long, int>> order;
        for (auto &w : weight) order.emplace_back(w.second, w.first);
        std::sort(order.rbegin(), order.rend());   // heaviest class first
        cm.assign(nPairs, bp.cell_mult);
        const float cands[4] = {1.0625f, 1.5f, 2.5f, 4.0f};
        for (auto &o : order) {
            const int c = o.second;
            float keep = bp.cell_mult;
            for (float v : cands) {
                if (v == keep) continue;
                std::vector<float> trial = cm;
                for (int i = 0; i < nPairs; ++i)
                    if (cls[i] == c) trial[i] = v;
                const double t = timed(bp, trial);
                if (t < bestt) {
                    bestt = t;
                    keep = v;
                    cm = trial;
                }
            }
            class_best[c] = keep;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(offs);
    if (!(bestt < 1e300)) return TMS_ERR_CUDA;
    *best = bp;
    if (best_ms) *best_ms = bestt;
    if (cache_path) {
        std::vector<std::string> lines;
        char buf[128];
        snprintf(buf, sizeof(buf), " %d %d %d %d %.6g %.6g", bp.face_level, bp.patch, bp.block_faces,
                 bp.tile_rows, (double)bp.cell_mult, bestt);
        lines.push_back(batch_key(A, B, nPairs, p0) + buf);
        for (auto &cb : class_best) {
            snprintf(buf, sizeof(buf), " %.6g", (double)cb.second);
            lines.push_back(class_key(cb.first, p0) + buf);
        }
        std::lock_guard<std::mutex> lk(g_tune_mu);
        append_lines(cache_path, lines);
        g_memo.clear();   // later searches read the new lines
    }
    return TMS_OK;
}

// Autotuner: picks the face level (triangle or quad boxes), the grid cell size
// (cell_mult) and the bounds-pass tile shape for a search or a batch of searches
// by timing each candidate on the caller's meshes, and caches the choice in a
// text file keyed by the device name and the meshes' sizes.  Used to set up a
// sweep (the batched continuation search of many pairs replays one tuned plan).
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "tms_common.cuh"

namespace {

std::string tune_key(const tms_mesh *A, const tms_mesh *B, int nPairs, const tms_params &base) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    std::string k = prop.name;
    for (char &c : k)
        if (c == ' ') c = '_';
    // the size class: every mesh view's N x M (hashed for large batches)
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
    char buf[160];
    snprintf(buf, sizeof(buf), "|pairs=%d|sizes=%016llx|prec=%d|filter=%d|narrow=%d|moller=%d", nPairs,
             (unsigned long long)h, base.precision, base.cell_filter, base.narrow_filter, base.moller);
    return k + buf;
}

bool cache_lookup(const char *path, const std::string &key, tms_params *p, double *ms) {
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[400];
        int fl, bf, tr;
        float cm;
        double t;
        if (sscanf(line, "%399s %d %f %d %d %lf", k, &fl, &cm, &bf, &tr, &t) == 6 && key == k) {
            p->face_level = fl;
            p->cell_mult = cm;
            p->block_faces = bf;
            p->tile_rows = tr;
            *ms = t;
            found = true;   // the last line for a key wins
        }
    }
    fclose(f);
    return found;
}

void cache_store(const char *path, const std::string &key, const tms_params &p, double ms) {
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %.6g %d %d %.6g\n", key.c_str(), p.face_level, (double)p.cell_mult,
            p.block_faces, p.tile_rows, ms);
    fclose(f);
}

}  // namespace

extern "C" tms_status tms_autotune(const tms_mesh *A, const tms_mesh *B, int nPairs,
                                   const tms_params *base, tms_params *best, const char *cache_path,
                                   double *best_ms, void *stream) {
    if (!A || !B || nPairs <= 0 || !best) return TMS_ERR_ARG;
    tms_params p0;
    tms_params_default(&p0);
    if (base) p0 = *base;
    p0.timing = 0;
    const std::string key = tune_key(A, B, nPairs, p0);
    tms_params cached = p0;
    double cms = 0.0;
    if (cache_lookup(cache_path, key, &cached, &cms)) {
        *best = cached;
        if (best_ms) *best_ms = cms;
        return TMS_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // output scratch for the trial runs, sized by a first run
    long long n = 0;
    long long cap = 1 << 16;
    tms_hit *out = nullptr;
    long long *offs = nullptr;
    if (cudaMalloc((void **)&out, cap * sizeof(tms_hit)) != cudaSuccess) return TMS_ERR_CUDA;
    if (cudaMalloc((void **)&offs, (nPairs + 1) * sizeof(long long)) != cudaSuccess) {
        cudaFree(out);
        return TMS_ERR_CUDA;
    }
    auto run = [&](const tms_params &p) -> tms_status {
        if (nPairs == 1) return tms_search(A[0], B[0], &p, out, cap, &n, stream);
        return tms_search_batched(A, B, nPairs, &p, out, cap, offs, &n, stream);
    };
    tms_status s = run(p0);
    if (s == TMS_ERR_CAPACITY && n > cap) {
        cudaFree(out);
        cap = n + 1024;
        if (cudaMalloc((void **)&out, cap * sizeof(tms_hit)) != cudaSuccess) {
            cudaFree(offs);
            return TMS_ERR_CUDA;
        }
        s = run(p0);
    }
    if (s != TMS_OK) {
        cudaFree(out);
        cudaFree(offs);
        return s;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int face_levels[2] = {1, 0};
    const float mults[3] = {1.0625f, 1.5f, 2.5f};
    const int blocks[2] = {128, 64};
    const int rows[2] = {4, 8};
    double bestt = 1e300;
    tms_params bp = p0;
    for (int fl : face_levels)
        for (float cm : mults)
            for (int bf : blocks)
            for (int tr : rows) {
                tms_params p = p0;
                p.face_level = fl;
                p.cell_mult = cm;
                p.block_faces = bf;
                p.tile_rows = tr;
                if (run(p) != TMS_OK) continue;   // warm-up: plan, capture, growth
                std::vector<float> ts;
                for (int r = 0; r < 3; ++r) {
                    cudaEventRecord(e0, st);
                    tms_status rs = run(p);
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    if (rs != TMS_OK) break;
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ts.push_back(ms);
                }
                if (ts.size() < 3) continue;
                std::sort(ts.begin(), ts.end());
                if (ts[1] < bestt) {
                    bestt = ts[1];
                    bp = p;
                }
                tms_release_workspace(stream);   // keep only one trial plan alive
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(offs);
    if (!(bestt < 1e300)) return TMS_ERR_CUDA;
    *best = bp;
    if (best_ms) *best_ms = bestt;
    cache_store(cache_path, key, bp, bestt);
    return TMS_OK;
}

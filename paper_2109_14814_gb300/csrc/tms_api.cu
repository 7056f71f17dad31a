// Host side of the C ABI (include/tms.h): mesh handles, search plans with their
// scratch, the launch sequence of one search (or one batch of searches), CUDA
// graph capture and replay, capacity retries, and the adjoint entry point.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tms_common.cuh"

using namespace tms;

struct tms_mesh_s {
    unsigned magic;
    int device;
    long long id;
    MeshDev dev;       // device pointers, view-offset
    double *d_s;       // owned copy of all M s values
    int N, M, k0, k1;
};

namespace {

constexpr unsigned kMagic = 0x746d7331u;  // "tms1"
std::mutex g_mu;
// tms_search_host: the first n output records copied to host memory right
// after the search on its stream, before the synchronisation that reads the count
struct EarlyCopy {
    tms_hit *host = nullptr;
    long long n = 0;
};
thread_local EarlyCopy g_early;
std::atomic<long long> g_next_id{1};
thread_local std::string g_err;

int ceil_log2(unsigned long long v) {
    int b = 0;
    while ((1ULL << b) < v && b < 63) ++b;
    return b;
}

#define TMS_CK(call)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            g_err = std::string(#call) + ": " + cudaGetErrorString(e_);               \
            return TMS_ERR_CUDA;                                                      \
        }                                                                             \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    return cudaMalloc((void **)p, n * sizeof(T));
}

// the counters and pair 0's grid share one allocation (and one read-back copy)
constexpr size_t kGridOffset = (sizeof(Counters) + 255) / 256 * 256;
constexpr size_t kReadback = kGridOffset + sizeof(Grid);

struct Plan {
    // identity
    std::vector<long long> ids;     // A ids then B ids
    tms_params prm;
    cudaStream_t user = nullptr;
    void *dHits = nullptr;
    long long hitCap = 0;
    long long *dOffsets = nullptr;
    int device = 0;
    int nPairs = 0;
    // mesh tables
    int n_meshes = 0;
    MeshDev *d_meshes = nullptr;
    std::vector<MeshDev> h_meshes;    // host copy of the mesh table
    // patch level: the patch views (one "face" per patch, its box in pbox),
    // which the cell passes and the grid emission read instead of the meshes
    bool patch = false;
    // patch frames (mixed precision with the FP32 filters): the patch-pair
    // test drops pairs that no triangle pair in them can make an FP64 hit
    bool frames = false;
    MeshDev *d_pmeshes = nullptr;
    // per-pair cell multipliers (size classes tuned by tms_autotune), or empty
    std::vector<float> cm_pair;
    float *d_cm_pair = nullptr;
    unsigned char *pbox = nullptr;    // patch boxes of all meshes
    unsigned char *qbox = nullptr;    // their quarter boxes
    float4 *pframe = nullptr;         // their frames (kFrameF4 float4 per patch)
    Cand *ppairs = nullptr;
    Cand *psurv = nullptr;           // patch pairs left by the quarter test
    unsigned long long ppair_cap = 0;
    int2 *d_pairs = nullptr;
    PassEntry *d_pass_all = nullptr, *d_pass_A = nullptr, *d_pass_B = nullptr;
    int n_pass_all = 0, n_pass_A = 0, n_pass_B = 0;
    long long tiles_all = 0, tiles_A = 0, tiles_B = 0;
    long long fslots_all = 0, fslots_A = 0, fslots_B = 0;   // padded face slots per pass
    unsigned long long facesA = 0, facesB = 0;
    int tri_bits = 0, pair_bits = 0;
    // scratch
    Bounds *d_bounds = nullptr;
    Grid *d_grids = nullptr;
    Counters *d_ctr = nullptr;
    Counters *h_ctr = nullptr;
    Grid *h_grid0 = nullptr;
    uint32_t *bmA = nullptr, *bmH = nullptr;
    int bmA_bits = 0, bmH_bits = 0;
    unsigned long long ent_cap = 0, cand_cap = 0, hit_cap = 0;
    uint64_t *ek = nullptr;
    uint32_t *ev = nullptr, *eslot = nullptr, *erank = nullptr, *grouped = nullptr;
    unsigned long long tsize = 0, tsize_min = 0;
    unsigned long long *tkey = nullptr;
    CellRec *crec = nullptr;
    uint2 *tcnt = nullptr;
    uint2 *tstart = nullptr;
    void *sort_scratch = nullptr;
    unsigned long long *partials = nullptr;
    Cand *cand = nullptr, *surv = nullptr;
    uint32_t *qsurv = nullptr;        // candidates left by the quad-level test
    float4 *split = nullptr;          // FP32 split vertex copies of all meshes
    unsigned long long split_total = 0;
    std::vector<unsigned long long> split_off;
    unsigned char *fbox = nullptr;    // face boxes of all meshes
    unsigned long long surv_cap = 0;
    tms_hit *hits = nullptr;
    uint64_t *hk = nullptr, *hk2 = nullptr, *okeys = nullptr;
    uint32_t *hv = nullptr, *hv2 = nullptr, *keep = nullptr, *kscan = nullptr;
    int grid = 304;
    int sort_grid = 608;
    // execution
    cudaStream_t st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraphExec_t exec = nullptr;
    static constexpr int kStages = 15;
    cudaEvent_t tev[kStages + 1] = {};
    float stage_ms[kStages] = {};
    int kernels = 0;
    int retries = 0;
    unsigned long long last_use = 0;

    void free_scratch() {
        void *ptrs[] = {bmA, bmH, ek, ev, eslot, erank, grouped, tkey, crec, tcnt, tstart,
                        sort_scratch, cand, surv, hits, hk, hk2, okeys, hv, hv2,
                        keep, kscan, ppairs, psurv, qsurv};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        ppairs = psurv = nullptr;
        qsurv = nullptr;
        bmA = bmH = nullptr; ek = nullptr; ev = eslot = erank = grouped = nullptr;
        tkey = nullptr; crec = nullptr; tcnt = nullptr; tstart = nullptr;
        sort_scratch = nullptr; cand = surv = nullptr; hits = nullptr; hk = hk2 = okeys = nullptr;
        hv = hv2 = keep = kscan = nullptr;
        if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
    }
    ~Plan() {
        if (st) cudaStreamSynchronize(st);
        free_scratch();
        void *ptrs[] = {d_meshes, d_pairs, d_pass_all, d_pass_A, d_pass_B, d_bounds,
                        d_ctr, partials, split, fbox, d_pmeshes, pbox, qbox, pframe, d_cm_pair};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        if (h_ctr) cudaFreeHost(h_ctr);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        for (auto &e : tev)
            if (e) cudaEventDestroy(e);
        if (st) cudaStreamDestroy(st);
    }

    tms_status alloc_scratch() {
        free_scratch();
        TMS_CK(dalloc(&bmA, (size_t)1 << (bmA_bits)));
        TMS_CK(dalloc(&bmH, (size_t)1 << (bmH_bits)));
        TMS_CK(dalloc(&ek, ent_cap));
        TMS_CK(dalloc(&ev, ent_cap));
        TMS_CK(dalloc(&eslot, ent_cap));
        TMS_CK(dalloc(&erank, ent_cap));
        TMS_CK(dalloc(&grouped, ent_cap));
        // cell table: a power of two, all slots free (zero); distinct cells are
        // far fewer than entries, so it starts at a sixteenth of the entry
        // capacity (L2-resident) and grows when a search finds it over half full
        tsize = 1024;
        const unsigned long long want = (prm.inject & 8u) ? 0 : ent_cap / 16;
        while ((tsize < want || tsize < tsize_min) && tsize < (1ULL << 31)) tsize <<= 1;
        TMS_CK(dalloc(&tkey, tsize));
        TMS_CK(dalloc(&tcnt, tsize));
        TMS_CK(dalloc(&tstart, tsize));
        TMS_CK(cudaMemset(tkey, 0, tsize * sizeof(unsigned long long)));
        TMS_CK(cudaMemset(tcnt, 0, tsize * sizeof(uint2)));
        // per cell: a cell holding both meshes has at least two entries
        TMS_CK(dalloc(&crec, ent_cap / 2 + 1));
        TMS_CK(dalloc(reinterpret_cast<unsigned char **>(&sort_scratch),
                      radix_scratch_size(hit_cap, 2 * tri_bits + pair_bits)));
        TMS_CK(dalloc(&cand, cand_cap));
        TMS_CK(dalloc(&qsurv, cand_cap));
        if (patch) TMS_CK(dalloc(&ppairs, ppair_cap));
        if (patch) TMS_CK(dalloc(&psurv, ppair_cap));
        TMS_CK(dalloc(&surv, surv_cap));
        TMS_CK(dalloc(&hits, hit_cap));
        TMS_CK(dalloc(&hk, hit_cap));
        TMS_CK(dalloc(&hk2, hit_cap));
        TMS_CK(dalloc(&okeys, hit_cap));
        TMS_CK(dalloc(&hv, hit_cap));
        TMS_CK(dalloc(&hv2, hit_cap));
        TMS_CK(dalloc(&keep, hit_cap));
        TMS_CK(dalloc(&kscan, hit_cap));
        return TMS_OK;
    }

    // The whole search as a stream-ordered launch sequence (no host round trip).
    // inside stream capture an event record becomes a graph node only with the
    // external flag
    bool capturing = false;
    void mark(int i, cudaStream_t s) {
        if (!prm.timing) return;
        if (capturing) cudaEventRecordWithFlags(tev[i], s, cudaEventRecordExternal);
        else cudaEventRecord(tev[i], s);
    }

    void enqueue(cudaStream_t s) {
        const tms_params &p = prm;
        const int prec = p.precision, fl = p.face_level;
        const int block = (p.block_faces == 64 || p.block_faces == 256) ? p.block_faces : 128;
        const int sort_passes_h = (2 * tri_bits + pair_bits + kRadixBits - 1) / kRadixBits;
        kernels = 0;
        mark(0, s);
        // the occupancy filter runs at the face level only: patches are few, and
        // nearly every patch-cell incidence lies in a cell both meshes occupy
        const bool filter = p.cell_filter && !patch;
        launch_search_init(d_bounds, n_meshes, d_ctr, filter ? bmA : nullptr,
                           (unsigned long long)1 << bmA_bits, filter ? bmH : nullptr,
                           (unsigned long long)1 << bmH_bits, grid, s);
        GroupArgs ga;
        ga.ent_key = ek; ga.ent_face = ev; ga.d_n = &d_ctr->entries; ga.cap = ent_cap;
        ga.ent_slot = eslot; ga.ent_rank = erank;
        ga.tkey = tkey; ga.tcnt = tcnt; ga.tstart = tstart; ga.tsize = tsize;
        ga.cells = crec; ga.grids = d_grids;
        ga.grouped = grouped; ga.partials = partials; ga.ctr = d_ctr;
        kernels += 1;
        mark(1, s);

        FacePassArgs fa;
        memset(&fa, 0, sizeof(fa));
        fa.meshes = d_meshes;
        fa.tile_rows = p.tile_rows;
        fa.bounds = d_bounds;
        fa.grids = d_grids;
        fa.bmA = bmA;
        fa.bmA_word_bits = bmA_bits;
        fa.bmH = bmH;
        fa.bmH_word_bits = bmH_bits;
        fa.ent_key = ek;
        fa.ent_val = ev;
        fa.ctr = d_ctr;
        fa.ent_cap = ent_cap;

        fa.entries = d_pass_all; fa.n_entries = n_pass_all; fa.total_tiles = tiles_all;
        fa.mode = MODE_BOUNDS;
        fa.patch = patch ? 1 : 0;
        fa.frames = frames ? 1 : 0;
        launch_face_pass(fa, prec, fl, block, s);
        // the cell passes and the grid emission work on the patches (patch level)
        fa.patch = 0;
        fa.frames = 0;
        if (patch) fa.meshes = d_pmeshes;
        mark(2, s);
        launch_grid_params(d_bounds, d_pairs, nPairs, d_grids, p.cell_mult, s, d_cm_pair);
        kernels += 2;
        mark(3, s);

        if (filter) {
            mark(4, s);
            fa.entries = d_pass_A; fa.n_entries = n_pass_A; fa.total_faces = fslots_A;
            fa.mode = MODE_MARK;
            launch_face_pass(fa, prec, fl, block, s);
            mark(5, s);
            fa.entries = d_pass_B; fa.n_entries = n_pass_B; fa.total_faces = fslots_B;
            fa.mode = MODE_PROBE_MARK;
            launch_face_pass(fa, prec, fl, block, s);
            mark(6, s);
            fa.entries = d_pass_A; fa.n_entries = n_pass_A; fa.total_faces = fslots_A;
            fa.mode = MODE_PROBE;
            launch_face_pass(fa, prec, fl, block, s);
            kernels += 3;
        } else {
            mark(4, s);
            mark(5, s);
            mark(6, s);
            fa.entries = d_pass_all; fa.n_entries = n_pass_all; fa.total_faces = fslots_all;
            fa.mode = MODE_EMIT_ALL;
            launch_face_pass(fa, prec, fl, block, s);
            kernels += 1;
        }
        mark(7, s);

        // group the entries by (pair, cell), mesh A's first
        launch_group_count(ga, grid * 2, s);
        mark(8, s);
        launch_group_cells(ga, grid * 2, s);
        kernels += 5;
        mark(9, s);

        EmitArgs ea;
        ea.cells = crec; ea.vals = grouped;
        ea.grids = d_grids; ea.meshes = d_meshes; ea.pairs = d_pairs; ea.ctr = d_ctr;
        ea.ent_cap = ent_cap; ea.cand = cand; ea.cand_cap = cand_cap; ea.moller = p.moller;
        ea.cand_ctr = &d_ctr->cand;
        ea.waves = 0;
        if (patch) {
            // patch pairs with overlapping boxes, each once (owner cell); few
            // tiles (about one per cell), so one wave of blocks
            ea.meshes = d_pmeshes; ea.cand = ppairs; ea.cand_cap = ppair_cap;
            ea.cand_ctr = &d_ctr->ppairs; ea.moller = 0; ea.waves = 1;
        }
        launch_emit(ea, prec, fl, grid / 2, s);
        kernels += 1;
        mark(10, s);
        if (patch) {
            // the quad pairs of the patch pairs
            PatchArgs pa;
            pa.ppairs = ppairs; pa.psurv = psurv; pa.ppair_cap = ppair_cap; pa.meshes = d_meshes;
            pa.pairs = d_pairs;
            pa.ctr = d_ctr; pa.ent_cap = ent_cap; pa.cand = cand; pa.cand_cap = cand_cap;
            pa.moller = p.moller;
            pa.frames = frames ? 1 : 0;
            pa.tau = p.tau;
            launch_patch_quads(pa, prec, grid / 2, s);
            kernels += 2;
        }
        mark(11, s);

        NarrowArgs na;
        na.cand = cand; na.cand_cap = cand_cap; na.surv = surv; na.surv_cap = surv_cap;
        na.qsurv = qsurv;
        na.meshes = d_meshes; na.pairs = d_pairs;
        na.ctr = d_ctr; na.hits = hits; na.hit_key = hk; na.hit_val = hv; na.hit_cap = hit_cap;
        na.tau = p.tau; na.tri_bits = tri_bits; na.fp32_filter = p.narrow_filter;
        launch_narrow(na, fl, grid / 2, grid * 4, s);
        kernels += 2;
        mark(12, s);

        DedupArgs da;
        da.raw = hits;
        da.meshes = d_meshes; da.pairs = d_pairs; da.ctr = d_ctr; da.raw_cap = hit_cap;
        da.keep = keep; da.keep_scan = kscan; da.partials = partials;
        da.out = (tms_hit *)dHits; da.out_cap = (unsigned long long)hitCap; da.out_keys = okeys;
        da.offsets = dOffsets; da.n_pairs = nPairs; da.tri_bits = tri_bits; da.tau = p.tau;
        // the raw hits are few: a small grid keeps the per-pass fixed cost low
        const bool halt = radix_sort(hk, hv, hk2, hv2, sort_scratch, &d_ctr->raw_hits, hit_cap,
                                     2 * tri_bits + pair_bits, sort_grid, &d_ctr->status,
                                     (unsigned long long)p.spin_limit, (p.inject & 16u) ? 1 : 0, s);
        kernels += 2 + sort_passes_h;
        mark(13, s);
        da.keys = halt ? hk2 : hk; da.vals = halt ? hv2 : hv;
        launch_dedup(da, grid, s);
        kernels += 5 + (dOffsets ? 1 : 0);
        mark(14, s);

        cudaMemcpyAsync(h_ctr, d_ctr, kReadback, cudaMemcpyDeviceToHost, s);
        mark(15, s);
    }

    tms_status run() {
        TMS_CK(cudaEventRecord(ev_in, user));
        TMS_CK(cudaStreamWaitEvent(st, ev_in, 0));
        if (prm.use_graph) {
            if (!exec) {
                cudaGraph_t g = nullptr;
                TMS_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                capturing = true;
                enqueue(st);
                capturing = false;
                cudaError_t e = cudaStreamEndCapture(st, &g);
                if (e != cudaSuccess) {
                    g_err = std::string("graph capture: ") + cudaGetErrorString(e);
                    return TMS_ERR_CUDA;
                }
                e = cudaGraphInstantiate(&exec, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) {
                    exec = nullptr;
                    g_err = std::string("graph instantiate: ") + cudaGetErrorString(e);
                    return TMS_ERR_CUDA;
                }
            }
            TMS_CK(cudaGraphLaunch(exec, st));
        } else {
            enqueue(st);
            TMS_CK(cudaGetLastError());
        }
        if (g_early.host && g_early.n > 0 && dHits)
            TMS_CK(cudaMemcpyAsync(g_early.host, dHits, (size_t)g_early.n * sizeof(tms_hit),
                                   cudaMemcpyDeviceToHost, st));
        TMS_CK(cudaEventRecord(ev_out, st));
        TMS_CK(cudaStreamWaitEvent(user, ev_out, 0));
        TMS_CK(cudaEventSynchronize(ev_out));
        if (prm.timing) {
            for (int i = 0; i < kStages; ++i) {
                float ms = 0.0f;
                if (cudaEventElapsedTime(&ms, tev[i], tev[i + 1]) != cudaSuccess) {
                    cudaGetLastError();
                    ms = -1.0f;
                }
                stage_ms[i] = ms;
            }
        }
        return TMS_OK;
    }
};

std::vector<Plan *> g_plans;
unsigned long long g_clock = 0;
std::map<cudaStream_t, tms_stats> g_stats;
std::map<cudaStream_t, std::vector<float>> g_stage_ms;
int g_configured_mask = 0;

bool same_params(const tms_params &a, const tms_params &b) {
    return a.precision == b.precision && a.face_level == b.face_level && a.moller == b.moller &&
           a.cell_filter == b.cell_filter && a.narrow_filter == b.narrow_filter &&
           a.cell_mult == b.cell_mult && a.tau == b.tau && a.entry_capacity == b.entry_capacity &&
           a.cand_capacity == b.cand_capacity && a.hit_capacity == b.hit_capacity &&
           a.use_graph == b.use_graph && a.inject == b.inject && a.block_faces == b.block_faces &&
           a.tile_rows == b.tile_rows && a.timing == b.timing && a.patch == b.patch &&
           a.spin_limit == b.spin_limit;
}

tms_status validate_params(const tms_params &p) {
    if (p.precision != 0 && p.precision != 1) return TMS_ERR_ARG;
    if (p.face_level != 0 && p.face_level != 1) return TMS_ERR_ARG;
    if (!(p.cell_mult >= 1.0f) || !(p.cell_mult < 1e6f)) return TMS_ERR_ARG;
    if (!(p.tau >= 0.0) || !(p.tau < 1.0)) return TMS_ERR_ARG;
    if (p.entry_capacity < 0 || p.cand_capacity < 0 || p.hit_capacity < 0) return TMS_ERR_ARG;
    if (p.patch != 0 && p.patch != 1) return TMS_ERR_ARG;
    if (p.spin_limit < 0) return TMS_ERR_ARG;
    return TMS_OK;
}

tms_status check_mesh(tms_mesh m, int device) {
    if (!m || m->magic != kMagic) return TMS_ERR_STATE;
    if (m->device != device) return TMS_ERR_ARG;
    return TMS_OK;
}

// a mesh in a pass: bounds-pass tiles over its quads; cell-pass slots over its
// faces, or over its patches (patch level)
void fill_pass(std::vector<PassEntry> &v, long long &tiles, long long &fslots, const tms_mesh m,
               int mesh_index, int pair, int role, int block, int rows, int face_level, bool patch) {
    PassEntry e;
    e.mesh = mesh_index;
    e.pair = pair;
    e.role = role;
    e.tiles_i = (m->dev.nqi + block - 1) / block;
    int tiles_k = (m->dev.nqk + rows - 1) / rows;
    e.tile_base = tiles;
    tiles += (long long)e.tiles_i * tiles_k;
    e.face_base = fslots;
    e.faces = patch ? (long long)((m->dev.nqi + kPatchI - 1) / kPatchI) * ((m->dev.nqk + kPatchK - 1) / kPatchK)
                    : (long long)face_slots(m->dev, face_level);
    fslots += (e.faces + 31) / 32 * 32;
    v.push_back(e);
}

tms_status make_plan(const tms_mesh *A, const tms_mesh *B, int nPairs, const tms_params &prm,
                     const std::vector<float> &cm_pair, cudaStream_t user, void *dHits,
                     long long hitCap, long long *dOffsets, int device, Plan **out) {
    Plan *P = new Plan();
    P->prm = prm;
    P->prm.autotune_cache = nullptr;
    P->cm_pair = cm_pair;
    P->user = user;
    P->dHits = dHits;
    P->hitCap = hitCap;
    P->dOffsets = dOffsets;
    P->device = device;
    P->nPairs = nPairs;
    for (int i = 0; i < nPairs; ++i) P->ids.push_back(A[i]->id);
    for (int i = 0; i < nPairs; ++i) P->ids.push_back(B[i]->id);
    const int block = (prm.block_faces == 64 || prm.block_faces == 256) ? prm.block_faces : 128;
    const int rows = prm.tile_rows == 8 ? 8 : 4;
    P->prm.tile_rows = rows;
    P->patch = prm.patch == 1 && prm.face_level == 1;
    const bool patch = P->patch;
    P->frames = patch && prm.precision == 1 && prm.narrow_filter == 1;

    std::vector<MeshDev> meshes;
    std::vector<int2> pairs;
    std::vector<PassEntry> pall, pa, pb;
    unsigned long long max_tri = 1;
    for (int i = 0; i < nPairs; ++i) {
        int ia = (int)meshes.size();
        meshes.push_back(A[i]->dev);
        int ib = (int)meshes.size();
        meshes.push_back(B[i]->dev);
        pairs.push_back(make_int2(ia, ib));
        const unsigned long long fpq = prm.face_level == 0 ? 2 : 1;
        auto cells_of = [&](const MeshDev &d) -> unsigned long long {
            if (patch)
                return (unsigned long long)((d.nqi + kPatchI - 1) / kPatchI) * ((d.nqk + kPatchK - 1) / kPatchK);
            return fpq * (unsigned long long)d.nqi * d.nqk;
        };
        P->facesA += cells_of(A[i]->dev);
        P->facesB += cells_of(B[i]->dev);
        max_tri = std::max(max_tri, 2ULL * A[i]->dev.N * A[i]->dev.nqk);
        max_tri = std::max(max_tri, 2ULL * B[i]->dev.N * B[i]->dev.nqk);
    }
    const int fl = prm.face_level;
    for (int i = 0; i < nPairs; ++i) {
        fill_pass(pall, P->tiles_all, P->fslots_all, A[i], pairs[i].x, i, 0, block, rows, fl, patch);
        fill_pass(pall, P->tiles_all, P->fslots_all, B[i], pairs[i].y, i, 1, block, rows, fl, patch);
        fill_pass(pa, P->tiles_A, P->fslots_A, A[i], pairs[i].x, i, 0, block, rows, fl, patch);
        fill_pass(pb, P->tiles_B, P->fslots_B, B[i], pairs[i].y, i, 1, block, rows, fl, patch);
    }
    // FP32 split vertex copies (32 bytes per view vertex) and face boxes (32 or
    // 64 bytes per face slot), written by the bounds pass
    const unsigned long long box_bytes = prm.precision == 1 ? 32 : 64;
    std::vector<unsigned long long> fbox_off, pbox_off, pframe_off;
    unsigned long long fbox_total = 0, pbox_total = 0, pframe_total = 0;
    for (auto &md : meshes) {
        P->split_off.push_back(P->split_total);
        P->split_total += 2ULL * (unsigned long long)md.N * (unsigned long long)md.M;
        fbox_off.push_back(fbox_total);
        fbox_total += (face_slots(md, fl) * box_bytes + 255) / 256 * 256;
        md.npi = patch ? (md.nqi + kPatchI - 1) / kPatchI : 0;
        md.npk = patch ? (md.nqk + kPatchK - 1) / kPatchK : 0;
        md.pmagic = recip64((unsigned long long)md.npi);
        md.pbox = nullptr;
        md.qbox = nullptr;
        md.pframe = nullptr;
        pbox_off.push_back(pbox_total);
        pbox_total += ((unsigned long long)md.npi * md.npk * box_bytes + 255) / 256 * 256;
        pframe_off.push_back(pframe_total);
        pframe_total += ((unsigned long long)md.npi * md.npk * kFrameF4 + 15) / 16 * 16;
    }
    std::vector<MeshDev> pmeshes;
    {
        cudaError_t se = dalloc(&P->split, P->split_total);
        if (se == cudaSuccess) se = dalloc(&P->fbox, fbox_total);
        if (se == cudaSuccess && patch) se = dalloc(&P->pbox, pbox_total);
        if (se == cudaSuccess && patch) se = dalloc(&P->qbox, 4 * pbox_total);
        if (se == cudaSuccess && P->frames) se = dalloc(&P->pframe, pframe_total);
        if (se != cudaSuccess) { g_err = cudaGetErrorString(se); delete P; return TMS_ERR_CUDA; }
        for (size_t i = 0; i < meshes.size(); ++i) {
            meshes[i].split = P->split + P->split_off[i];
            meshes[i].fbox = P->fbox + fbox_off[i];
            if (patch) {
                meshes[i].pbox = P->pbox + pbox_off[i];
                meshes[i].qbox = P->qbox + 4 * pbox_off[i];
                if (P->frames) meshes[i].pframe = P->pframe + pframe_off[i];
            }
        }
        // a patch view is a mesh of npi x npk quad-like slots, all valid
        for (const MeshDev &md : meshes) {
            MeshDev v = md;
            v.N = md.npi;
            v.M = md.npk + 1;
            v.periodic = 1;
            v.nqi = md.npi;
            v.nqk = md.npk;
            v.fbox = md.pbox;
            v.split = nullptr;
            v.pframe = nullptr;
            pmeshes.push_back(v);
        }
    }
    P->n_meshes = (int)meshes.size();
    P->h_meshes = meshes;
    P->n_pass_all = (int)pall.size();
    P->n_pass_A = (int)pa.size();
    P->n_pass_B = (int)pb.size();
    P->tri_bits = ceil_log2(max_tri);
    P->pair_bits = ceil_log2((unsigned long long)nPairs);
    if (2 * P->tri_bits + P->pair_bits > 64 || P->pair_bits > 31) {
        delete P;
        g_err = "mesh pair too large for 64-bit hit keys";
        return TMS_ERR_ARG;
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    P->grid = std::min(1024, 2 * sms);
    P->sort_grid = 4 * sms;

    cudaError_t e;
#define TMS_PCK(call) do { if ((e = (call)) != cudaSuccess) { g_err = cudaGetErrorString(e); delete P; return TMS_ERR_CUDA; } } while (0)
    TMS_PCK(dalloc(&P->d_meshes, meshes.size()));
    TMS_PCK(dalloc(&P->d_pmeshes, pmeshes.size()));
    if (!cm_pair.empty()) {
        TMS_PCK(dalloc(&P->d_cm_pair, cm_pair.size()));
        TMS_PCK(cudaMemcpy(P->d_cm_pair, cm_pair.data(), cm_pair.size() * sizeof(float),
                           cudaMemcpyHostToDevice));
    }
    TMS_PCK(dalloc(&P->d_pairs, pairs.size()));
    TMS_PCK(dalloc(&P->d_pass_all, pall.size()));
    TMS_PCK(dalloc(&P->d_pass_A, pa.size()));
    TMS_PCK(dalloc(&P->d_pass_B, pb.size()));
    TMS_PCK(dalloc(&P->d_bounds, meshes.size()));
    // counters, then the grids of all pairs (pair 0's right after the counters)
    {
        unsigned char *blk = nullptr;
        TMS_PCK(dalloc(&blk, kGridOffset + pairs.size() * sizeof(Grid)));
        P->d_ctr = reinterpret_cast<Counters *>(blk);
        P->d_grids = reinterpret_cast<Grid *>(blk + kGridOffset);
    }
    TMS_PCK(dalloc(&P->partials, 5 * 1024));
    {
        unsigned char *hb = nullptr;
        TMS_PCK(cudaMallocHost((void **)&hb, kReadback));
        P->h_ctr = reinterpret_cast<Counters *>(hb);
        P->h_grid0 = reinterpret_cast<Grid *>(hb + kGridOffset);
    }
    TMS_PCK(cudaMemcpy(P->d_meshes, meshes.data(), meshes.size() * sizeof(MeshDev), cudaMemcpyHostToDevice));
    TMS_PCK(cudaMemcpy(P->d_pmeshes, pmeshes.data(), pmeshes.size() * sizeof(MeshDev), cudaMemcpyHostToDevice));
    TMS_PCK(cudaMemcpy(P->d_pairs, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice));
    TMS_PCK(cudaMemcpy(P->d_pass_all, pall.data(), pall.size() * sizeof(PassEntry), cudaMemcpyHostToDevice));
    TMS_PCK(cudaMemcpy(P->d_pass_A, pa.data(), pa.size() * sizeof(PassEntry), cudaMemcpyHostToDevice));
    TMS_PCK(cudaMemcpy(P->d_pass_B, pb.data(), pb.size() * sizeof(PassEntry), cudaMemcpyHostToDevice));
    TMS_PCK(cudaStreamCreateWithFlags(&P->st, cudaStreamNonBlocking));
    TMS_PCK(cudaEventCreateWithFlags(&P->ev_in, cudaEventDisableTiming));
    TMS_PCK(cudaEventCreateWithFlags(&P->ev_out, cudaEventDisableTiming));
    if (prm.timing)
        for (auto &evt : P->tev) TMS_PCK(cudaEventCreate(&evt));
#undef TMS_PCK

    const unsigned long long faces = P->facesA + P->facesB;
    unsigned long long ent = prm.entry_capacity > 0 ? (unsigned long long)prm.entry_capacity
                             : patch ? 4 * faces + (1 << 16)
                             : (prm.cell_filter ? std::max<unsigned long long>(1 << 16, faces / 2)
                                                : 4 * faces + (1 << 16));
    if (prm.inject & 1u) ent = 1;
    P->ent_cap = std::min<unsigned long long>(ent, 0x7fffffffULL);
    // patch level: candidates are quad pairs, about one per quad of A
    const unsigned long long quadsA = [&] {
        unsigned long long q = 0;
        for (int i = 0; i < nPairs; ++i) q += (unsigned long long)A[i]->dev.nqi * A[i]->dev.nqk;
        return q;
    }();
    P->cand_cap = prm.cand_capacity > 0 ? (unsigned long long)prm.cand_capacity
                  : patch ? std::max<unsigned long long>(1 << 16, quadsA + quadsA / 4)
                          : std::max<unsigned long long>(1 << 16, 2 * P->ent_cap);
    P->ppair_cap = patch ? std::max<unsigned long long>(1 << 16, 4 * faces) : 0;
    P->hit_cap = prm.hit_capacity > 0 ? (unsigned long long)prm.hit_capacity
                                      : std::max<unsigned long long>(1 << 14, P->cand_cap / 16);
    P->surv_cap = std::max<unsigned long long>(1 << 16, P->cand_cap / 8);
    if (prm.inject & 32u) {
        // test switch: the patch-pair, candidate, survivor and raw-hit buffers
        // start at one record, so that each grows in turn
        P->ppair_cap = patch ? 1 : 0;
        P->cand_cap = P->surv_cap = P->hit_cap = 1;
    }
    P->bmA_bits = std::min(26, std::max(11, ceil_log2(std::max<unsigned long long>(P->facesA, 1) * 8) - 5));
    P->bmH_bits = std::min(25, std::max(11, ceil_log2(P->ent_cap * 8) - 5));
    tms_status s = P->alloc_scratch();
    if (s != TMS_OK) { delete P; return s; }
    *out = P;
    return TMS_OK;
}

Plan *find_plan(const tms_mesh *A, const tms_mesh *B, int nPairs, const tms_params &prm,
                const std::vector<float> &cm_pair, cudaStream_t user, void *dHits, long long hitCap,
                long long *dOffsets, int device) {
    for (Plan *P : g_plans) {
        if (P->device != device || P->user != user || P->dHits != dHits || P->hitCap != hitCap ||
            P->dOffsets != dOffsets || P->nPairs != nPairs || P->cm_pair != cm_pair)
            continue;
        tms_params q = prm;
        q.tile_rows = q.tile_rows == 8 ? 8 : 4;
        if (!same_params(P->prm, q)) continue;
        bool ok = true;
        for (int i = 0; i < nPairs && ok; ++i) ok = P->ids[i] == A[i]->id && P->ids[nPairs + i] == B[i]->id;
        if (ok) return P;
    }
    return nullptr;
}

void drop_plans_if(bool (*pred)(Plan *, void *), void *ctx) {
    std::vector<Plan *> keep;
    for (Plan *P : g_plans) {
        if (pred(P, ctx)) delete P;
        else keep.push_back(P);
    }
    g_plans.swap(keep);
}

tms_status search_core(const tms_mesh *A, const tms_mesh *B, int nPairs, const tms_params &prm,
                       const std::vector<float> &cm_pair, tms_hit *dHits, long long hitCap,
                       long long *dOffsets, long long *nHits, void *stream) {
    if (!nHits || nPairs <= 0 || !A || !B || hitCap < 0 || (hitCap > 0 && !dHits)) return TMS_ERR_ARG;
    tms_status s = validate_params(prm);
    if (s != TMS_OK) return s;
    if (!cm_pair.empty()) {
        if ((int)cm_pair.size() != nPairs) return TMS_ERR_ARG;
        for (float c : cm_pair)
            if (!(c >= 1.0f) || !(c < 1e6f)) return TMS_ERR_ARG;
    }
    int device = 0;
    TMS_CK(cudaGetDevice(&device));
    for (int i = 0; i < nPairs; ++i) {
        if ((s = check_mesh(A[i], device)) != TMS_OK) return s;
        if ((s = check_mesh(B[i], device)) != TMS_OK) return s;
    }
    cudaStream_t user = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!(g_configured_mask & (1 << device))) {
        TMS_CK(configure_face_pass());
        configure_emit();
        configure_patch_quads();
        configure_narrow();
        g_configured_mask |= 1 << device;
    }
    Plan *P = find_plan(A, B, nPairs, prm, cm_pair, user, dHits, hitCap, dOffsets, device);
    if (!P) {
        if (g_plans.size() >= 16) {
            auto it = std::min_element(g_plans.begin(), g_plans.end(),
                                       [](Plan *x, Plan *y) { return x->last_use < y->last_use; });
            delete *it;
            g_plans.erase(it);
        }
        s = make_plan(A, B, nPairs, prm, cm_pair, user, dHits, hitCap, dOffsets, device, &P);
        if (s != TMS_OK) return s;
        g_plans.push_back(P);
    }
    P->last_use = ++g_clock;
    P->retries = 0;
    for (int attempt = 0; attempt < 8; ++attempt) {
        s = P->run();
        if (s != TMS_OK) return s;
        const Counters &c = *P->h_ctr;
        if (c.status & ST_NONFINITE) {
            g_err = "non-finite vertex coordinate";
            return TMS_ERR_ARG;
        }
        if (c.status & ST_PAIR_LIMIT) {
            g_err = "grid proposes too many face pairs (degenerate geometry)";
            return TMS_ERR_ARG;
        }
        if (c.status & ST_TIMEOUT) {
            g_err = "a device-side wait gave up (sort look-back)";
            return TMS_ERR_TIMEOUT;
        }
        bool grow = false;
        if ((c.status & ST_TABLE_FULL) || c.claimed > P->tsize / 2) {
            P->tsize_min = P->tsize * 4;
            grow = true;
        }
        if (!grow && c.entries > P->ent_cap) {
            P->ent_cap = std::min<unsigned long long>(0x7fffffffULL, c.entries + c.entries / 4 + 1024);
            P->bmH_bits = std::min(25, std::max(11, ceil_log2(P->ent_cap * 8) - 5));
            P->cand_cap = std::max(P->cand_cap, 2 * P->ent_cap);
            grow = true;
        }
        if (!grow && P->patch && c.ppairs > P->ppair_cap) {
            P->ppair_cap = c.ppairs + c.ppairs / 4 + 1024;
            grow = true;
        }
        if (!grow && c.cand > P->cand_cap) {
            P->cand_cap = c.cand + c.cand / 4 + 1024;
            grow = true;
        }
        if (!grow && c.fp64 > P->surv_cap) {
            P->surv_cap = c.fp64 + c.fp64 / 4 + 1024;
            grow = true;
        }
        if (!grow && c.raw_hits > P->hit_cap) {
            P->hit_cap = c.raw_hits + c.raw_hits / 4 + 1024;
            grow = true;
        }
        if (!grow) break;
        ++P->retries;
        TMS_CK(cudaStreamSynchronize(P->st));
        s = P->alloc_scratch();
        if (s != TMS_OK) return s;
    }
    const Counters &c = *P->h_ctr;
    if (c.status & ST_TABLE_FULL) {
        g_err = "cell table still full after retries";
        *nHits = (long long)c.out;
        return TMS_ERR_CAPACITY;
    }
    tms_stats st;
    memset(&st, 0, sizeof(st));
    st.entries = (long long)c.entries;
    st.cells = (long long)c.cells;
    st.pair_slots = (long long)c.pair_slots;
    st.candidates = (long long)c.cand;
    st.fp64_solves = (long long)c.fp64;
    st.fp32_solves = (long long)c.fp32;
    st.sat_tests = (long long)c.sat;
    st.quad_tests = (long long)c.quad;
    st.patch_pairs = (long long)c.ppairs;
    st.patch_tests = (long long)c.ptests;
    st.quad_kept = (long long)c.qkeep;
    st.patch_kept = (long long)c.psurv;
    st.raw_hits = (long long)c.raw_hits;
    st.hits = (long long)c.out;
    for (int d = 0; d < 4; ++d) st.grid_n[d] = P->h_grid0->n[d];
    st.empty = P->h_grid0->empty;
    st.retries = P->retries;
    st.kernels = P->kernels;
    g_stats[user] = st;
    if (prm.timing) g_stage_ms[user] = std::vector<float>(P->stage_ms, P->stage_ms + Plan::kStages);
    if (c.entries > P->ent_cap || c.cand > P->cand_cap || c.fp64 > P->surv_cap ||
        c.raw_hits > P->hit_cap || (P->patch && c.ppairs > P->ppair_cap)) {
        g_err = "scratch capacity still exceeded after retries";
        *nHits = (long long)c.out;
        return TMS_ERR_CAPACITY;
    }
    *nHits = (long long)c.out;
    if (prm.inject & 4u) {
        g_err = "injected timeout";
        return TMS_ERR_TIMEOUT;
    }
    if ((long long)c.out > hitCap || (prm.inject & 2u)) {
        g_err = "hit buffer too small";
        return TMS_ERR_CAPACITY;
    }
    return TMS_OK;
}

tms_status search_impl(const tms_mesh *A, const tms_mesh *B, int nPairs, const tms_params *params,
                       tms_hit *dHits, long long hitCap, long long *dOffsets, long long *nHits,
                       void *stream) {
    if (!nHits || nPairs <= 0 || !A || !B) return TMS_ERR_ARG;
    tms_params prm;
    tms_params_default(&prm);
    if (params) prm = *params;
    std::vector<float> cm_pair;
    if (prm.autotune_cache) {
        for (int i = 0; i < nPairs; ++i) {
            MeshDev v;
            int d;
            if (!A[i] || !B[i] || mesh_view(A[i], &v, &d) != TMS_OK || mesh_view(B[i], &v, &d) != TMS_OK)
                return TMS_ERR_STATE;
        }
        tune_lookup(A, B, nPairs, prm.autotune_cache, &prm, &cm_pair);
        prm.autotune_cache = nullptr;
    }
    return search_core(A, B, nPairs, prm, cm_pair, dHits, hitCap, dOffsets, nHits, stream);
}

bool plan_uses(Plan *P, void *ctx) {
    long long id = *(long long *)ctx;
    return std::find(P->ids.begin(), P->ids.end(), id) != P->ids.end();
}
bool plan_on_stream(Plan *P, void *ctx) {
    return ctx == nullptr || P->user == *(cudaStream_t *)ctx;
}

}  // namespace

tms_status tms::search_with_cm(const tms_mesh *A, const tms_mesh *B, int nPairs, const tms_params &params,
                               const std::vector<float> &cm_pair, tms_hit *dHits, long long hitCap,
                               long long *dOffsets, long long *nHits, void *stream) {
    tms_params prm = params;
    prm.autotune_cache = nullptr;
    return search_core(A, B, nPairs, prm, cm_pair, dHits, hitCap, dOffsets, nHits, stream);
}

extern "C" {

void tms_params_default(tms_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->precision = 1;
    p->face_level = 1;
    p->moller = 0;
    p->cell_filter = 1;
    p->narrow_filter = 1;
    p->cell_mult = 1.0625f;
    p->tau = 1e-12;
    p->use_graph = 1;
    p->block_faces = 128;
    p->tile_rows = 4;
    p->patch = 1;
}

const char *tms_status_str(tms_status s) {
    switch (s) {
        case TMS_OK: return "ok";
        case TMS_ERR_ARG: return "invalid argument";
        case TMS_ERR_CAPACITY: return "capacity exceeded";
        case TMS_ERR_TIMEOUT: return "device wait timed out";
        case TMS_ERR_CUDA: return "CUDA error";
        case TMS_ERR_STATE: return "invalid state";
        default: return "unknown status";
    }
}

const char *tms_version(void) { return "tms 0.1.0 (sm_103a)"; }

const char *tms_last_error(void) { return g_err.c_str(); }

tms_status tms_build_mesh(const double *dX, const double *dY, const double *dPx, const double *dPy,
                          int N, int M, int k0, int k1, const double *s, int periodic_theta,
                          void *stream, tms_mesh *out) {
    if (!out) return TMS_ERR_ARG;
    *out = nullptr;
    if (!dX || !dY || !dPx || !dPy || !s) return TMS_ERR_ARG;
    if (M < 2 || k0 < 0 || k1 > M || k1 - k0 < 2) return TMS_ERR_ARG;
    if (periodic_theta ? N < 3 : N < 2) return TMS_ERR_ARG;
    const int nqi = periodic_theta ? N : N - 1;
    if ((unsigned long long)N * (unsigned long long)M >= (1ULL << 31)) return TMS_ERR_ARG;
    int device = 0;
    TMS_CK(cudaGetDevice(&device));
    std::vector<double> hs(M);
    cudaPointerAttributes attr;
    cudaError_t ae = cudaPointerGetAttributes(&attr, s);
    if (ae != cudaSuccess) cudaGetLastError();
    const bool s_dev = ae == cudaSuccess && attr.type == cudaMemoryTypeDevice;
    if (s_dev) TMS_CK(cudaMemcpy(hs.data(), s, M * sizeof(double), cudaMemcpyDeviceToHost));
    else memcpy(hs.data(), s, M * sizeof(double));
    for (int k = 1; k < M; ++k)
        if (!(hs[k] > hs[k - 1])) return TMS_ERR_ARG;
    const double *ptrs[4] = {dX, dY, dPx, dPy};
    for (int c = 0; c < 4; ++c) {
        cudaPointerAttributes pa;
        cudaError_t pe = cudaPointerGetAttributes(&pa, ptrs[c]);
        if (pe != cudaSuccess) { cudaGetLastError(); return TMS_ERR_ARG; }
        if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) return TMS_ERR_ARG;
    }
    tms_mesh m = new tms_mesh_s();
    m->magic = kMagic;
    m->device = device;
    m->id = g_next_id++;
    m->N = N; m->M = M; m->k0 = k0; m->k1 = k1;
    cudaError_t e = cudaMalloc((void **)&m->d_s, M * sizeof(double));
    if (e != cudaSuccess) { delete m; g_err = cudaGetErrorString(e); return TMS_ERR_CUDA; }
    e = cudaMemcpyAsync(m->d_s, hs.data(), M * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) { cudaFree(m->d_s); delete m; g_err = cudaGetErrorString(e); return TMS_ERR_CUDA; }
    const size_t off = (size_t)k0 * N;
    for (int c = 0; c < 4; ++c) m->dev.c[c] = ptrs[c] + off;
    m->dev.s = m->d_s + k0;
    m->dev.N = N;
    m->dev.M = k1 - k0;
    m->dev.periodic = periodic_theta ? 1 : 0;
    m->dev.nqi = nqi;
    m->dev.nqk = k1 - k0 - 1;
    m->dev.pad = 0;
    m->dev.nmagic = recip64((unsigned long long)N);
    *out = m;
    return TMS_OK;
}

}  // extern "C"

void tms::set_last_error(const std::string &msg) { g_err = msg; }

tms_status tms::mesh_view(tms_mesh m, MeshDev *view, int *device) {
    if (!m || m->magic != kMagic) return TMS_ERR_STATE;
    *view = m->dev;
    *device = m->device;
    return TMS_OK;
}

extern "C" {

tms_status tms_destroy_mesh(tms_mesh m) {
    if (!m || m->magic != kMagic) return TMS_ERR_STATE;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        cudaDeviceSynchronize();
        long long id = m->id;
        drop_plans_if(plan_uses, &id);
    }
    cudaFree(m->d_s);
    m->magic = 0;
    delete m;
    return TMS_OK;
}

tms_status tms_search(tms_mesh A, tms_mesh B, const tms_params *params, tms_hit *dHits,
                      long long hitCap, long long *nHits, void *stream) {
    return search_impl(&A, &B, 1, params, dHits, hitCap, nullptr, nHits, stream);
}

namespace {
// the device output of tms_search_host, per device
struct HostOut {
    tms_hit *buf = nullptr;
    long long cap = 0;
    long long last_n = 0;   // the previous call's count: records copied with the count
};
std::mutex g_host_mu;
HostOut g_host_out[64];

// the view rows of a mesh's four coordinate arrays from host memory: one 2D
// copy when the four arrays are equally spaced on both sides (one tensor of
// shape (4, M, N), say), else one copy per coordinate
tms_status upload_view(tms_mesh m, const double *const host[4], cudaStream_t st) {
    for (int c = 0; c < 4; ++c)
        if (!host[c]) return TMS_ERR_ARG;
    const size_t off = (size_t)m->k0 * m->N;
    const size_t bytes = (size_t)(m->k1 - m->k0) * m->N * sizeof(double);
    const ptrdiff_t dp = m->dev.c[1] - m->dev.c[0], hp = host[1] - host[0];
    bool even = dp > 0 && hp > 0 && (size_t)dp * sizeof(double) >= bytes && (size_t)hp * sizeof(double) >= bytes;
    for (int c = 2; c < 4; ++c) even = even && m->dev.c[c] - m->dev.c[c - 1] == dp && host[c] - host[c - 1] == hp;
    if (even) {
        TMS_CK(cudaMemcpy2DAsync(const_cast<double *>(m->dev.c[0]), (size_t)dp * sizeof(double), host[0] + off,
                                 (size_t)hp * sizeof(double), bytes, 4, cudaMemcpyHostToDevice, st));
        return TMS_OK;
    }
    for (int c = 0; c < 4; ++c)
        TMS_CK(cudaMemcpyAsync(const_cast<double *>(m->dev.c[c]), host[c] + off, bytes,
                               cudaMemcpyHostToDevice, st));
    return TMS_OK;
}
}  // namespace

tms_status tms_search_host(tms_mesh A, const double *const hostA[4], tms_mesh B,
                           const double *const hostB[4], const tms_params *params,
                           tms_hit *hostHits, long long hitCap, long long *nHits, void *stream) {
    if (!hostA || !hostB || !nHits || hitCap < 0 || (hitCap > 0 && !hostHits)) return TMS_ERR_ARG;
    int device = 0;
    TMS_CK(cudaGetDevice(&device));
    if (device < 0 || device >= 64) return TMS_ERR_ARG;
    tms_status s;
    if ((s = check_mesh(A, device)) != TMS_OK) return s;
    if ((s = check_mesh(B, device)) != TMS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_view(A, hostA, st)) != TMS_OK) return s;
    if ((s = upload_view(B, hostB, st)) != TMS_OK) return s;
    // one caller at a time per device owns the output buffer for the whole call
    std::lock_guard<std::mutex> lk(g_host_mu);
    HostOut &o = g_host_out[device];
    const long long need = hitCap > 0 ? hitCap : 1;
    if (o.cap < need) {
        if (o.buf) cudaFree(o.buf);
        o.buf = nullptr;
        o.cap = 0;
        TMS_CK(cudaMalloc((void **)&o.buf, (size_t)need * sizeof(tms_hit)));
        o.cap = need;
    }
    // the records are copied back in the same round trip as the count, as many
    // as the previous call found and a margin; the rest, if any, after it
    const long long guess = std::min(hitCap, o.last_n + o.last_n / 8 + 64);
    g_early.host = hostHits;
    g_early.n = guess;
    s = tms_search(A, B, params, o.buf, hitCap, nHits, stream);
    g_early = EarlyCopy();
    if (s != TMS_OK && s != TMS_ERR_CAPACITY) return s;
    const long long n = *nHits < hitCap ? *nHits : hitCap;
    o.last_n = n;
    if (n > guess) {
        TMS_CK(cudaMemcpyAsync(hostHits + guess, o.buf + guess, (size_t)(n - guess) * sizeof(tms_hit),
                               cudaMemcpyDeviceToHost, st));
        TMS_CK(cudaStreamSynchronize(st));
    }
    return s;
}

tms_status tms_search_batched(const tms_mesh *A, const tms_mesh *B, int nPairs,
                              const tms_params *params, tms_hit *dHits, long long hitCap,
                              long long *dOffsets, long long *nHits, void *stream) {
    if (!dOffsets) return TMS_ERR_ARG;
    return search_impl(A, B, nPairs, params, dHits, hitCap, dOffsets, nHits, stream);
}

tms_status tms_backward(tms_mesh A, tms_mesh B, const tms_hit *dHits, long long nHits,
                        const double *dGradP, const double *dGradZ, double *dGradA, double *dGradB,
                        const double *dDvDalphaA, const double *dDvDalphaB, double *dGradAlpha,
                        void *stream) {
    if (nHits < 0 || (nHits > 0 && !dHits)) return TMS_ERR_ARG;
    int device = 0;
    TMS_CK(cudaGetDevice(&device));
    tms_status s;
    if ((s = check_mesh(A, device)) != TMS_OK) return s;
    if ((s = check_mesh(B, device)) != TMS_OK) return s;
    if (nHits == 0) return TMS_OK;
    AdjointArgs a;
    memset(&a, 0, sizeof(a));
    a.hits = dHits;
    a.n = nHits;
    a.A = A->dev;
    a.B = B->dev;
    a.gP = dGradP;
    a.gZ = dGradZ;
    const size_t MNa = (size_t)A->N * A->M, MNb = (size_t)B->N * B->M;
    const size_t offA = (size_t)A->k0 * A->N, offB = (size_t)B->k0 * B->N;
    for (int c = 0; c < 4; ++c) {
        a.gA[c] = dGradA ? dGradA + c * MNa + offA : nullptr;
        a.gB[c] = dGradB ? dGradB + c * MNb + offB : nullptr;
        a.dA[c] = dDvDalphaA ? dDvDalphaA + c * MNa + offA : nullptr;
        a.dB[c] = dDvDalphaB ? dDvDalphaB + c * MNb + offB : nullptr;
    }
    a.galpha = dGradAlpha;
    launch_adjoint(a, (cudaStream_t)stream);
    TMS_CK(cudaGetLastError());
    return TMS_OK;
}

tms_status tms_last_stats(void *stream, tms_stats *out) {
    if (!out) return TMS_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_stats.find((cudaStream_t)stream);
    if (it == g_stats.end()) return TMS_ERR_STATE;
    *out = it->second;
    return TMS_OK;
}

tms_status tms_last_stage_ms(void *stream, float *ms, int cap, int *n) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_stage_ms.find((cudaStream_t)stream);
    if (it == g_stage_ms.end()) return TMS_ERR_STATE;
    if (n) *n = (int)it->second.size();
    for (int i = 0; i < cap && i < (int)it->second.size(); ++i) ms[i] = it->second[i];
    return TMS_OK;
}

tms_status tms_last_patch_frames(void *stream, int side, float *host_out, long long cap,
                                 long long *n_patches, int *npi) {
    if (side != 0 && side != 1) return TMS_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    Plan *P = nullptr;
    for (Plan *Q : g_plans)
        if (Q->user == (cudaStream_t)stream && (!P || Q->last_use > P->last_use)) P = Q;
    if (!P || !P->frames || (int)P->h_meshes.size() < 2) return TMS_ERR_STATE;
    const MeshDev &md = P->h_meshes[side];
    const long long n = (long long)md.npi * md.npk;
    if (n_patches) *n_patches = n;
    if (npi) *npi = md.npi;
    if (cap < 4LL * kFrameF4 * n) return TMS_ERR_CAPACITY;
    if (!host_out && n > 0) return TMS_ERR_ARG;
    TMS_CK(cudaStreamSynchronize(P->user));
    if (n > 0)
        TMS_CK(cudaMemcpy(host_out, md.pframe, (size_t)n * kFrameF4 * sizeof(float4), cudaMemcpyDeviceToHost));
    return TMS_OK;
}

tms_status tms_release_workspace(void *stream) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t s = (cudaStream_t)stream;
    drop_plans_if(plan_on_stream, stream ? (void *)&s : nullptr);
    return TMS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Method of layers (Sec. 5, Sec. 6.2): half-layer column ranges and the sweep
// over the 8 n_max half-layer pairs as one batched search.
// ---------------------------------------------------------------------------

namespace {

constexpr unsigned kLayerMagic = 0x746d736cu;   // "tmsl"

// Shifts view-relative triangle ids to ids of the full meshes the plan was
// built from; shift[p] = (2 N_A (a_k0 - A.k0), 2 N_B (b_k0 - B.k0)).
__global__ void k_layer_ids(tms_hit *hits, long long n, const uint2 *shift, int nPairs) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned p = hits[i].pair;
    if (p >= (unsigned)nPairs) return;
    const uint2 d = shift[p];
    hits[i].triA += d.x;
    hits[i].triB += d.y;
}

// Column holding the boundary value b (within rel_tol |b|), or -1.
int boundary_column(const double *s, int M, double b, double rel_tol) {
    const double *it = std::lower_bound(s, s + M, b);
    int best = -1;
    double bd = 0.0;
    for (const double *q : {it - 1, it}) {
        if (q < s || q >= s + M) continue;
        const double d = std::fabs(*q - b);
        if (d <= rel_tol * std::fabs(b) && (best < 0 || d < bd)) {
            best = (int)(q - s);
            bd = d;
        }
    }
    return best;
}

}  // namespace

struct tms_layer_plan_s {
    unsigned magic;
    int nPairs;
    std::vector<tms_mesh> A, B;       // per pair (shared handles repeat)
    std::vector<tms_mesh> owned;      // distinct sub-view handles
    uint2 *d_shift;
};

extern "C" {

tms_status tms_layer_pairs(const double *sA, int MA, double Du, double lam_u, const double *sB,
                           int MB, double Ds, double lam_s, int n_max, double rel_tol,
                           tms_layer_pair *out, int cap, int *count) {
    if (!count || !sA || !sB || MA < 2 || MB < 2 || n_max < 1 || cap < 0 || (cap > 0 && !out)) {
        g_err = "tms_layer_pairs: bad argument";
        return TMS_ERR_ARG;
    }
    if (!(Du > 0.0) || !(lam_u > 1.0) || !(Ds > 0.0) || !(lam_s > 0.0 && lam_s < 1.0) ||
        !(rel_tol >= 0.0) || !std::isfinite(Du * lam_u) || !std::isfinite(Ds / lam_s)) {
        g_err = "tms_layer_pairs: need D > 0, lam_u > 1, 0 < lam_s < 1, rel_tol >= 0";
        return TMS_ERR_ARG;
    }
    for (int k = 1; k < MA; ++k)
        if (!(sA[k] > sA[k - 1])) { g_err = "tms_layer_pairs: sA not increasing"; return TMS_ERR_ARG; }
    for (int k = 1; k < MB; ++k)
        if (!(sB[k] > sB[k - 1])) { g_err = "tms_layer_pairs: sB not increasing"; return TMS_ERR_ARG; }
    const long long total = 8LL * n_max;
    if (total > 0x7fffffffLL) { g_err = "tms_layer_pairs: n_max too large"; return TMS_ERR_ARG; }
    *count = (int)total;
    // column range [k(lo), k(hi) + 1) of the closed interval between two boundaries
    auto range = [&](const double *s, int M, double v0, double v1, int &k0, int &k1) -> bool {
        const double lo = std::min(v0, v1), hi = std::max(v0, v1);
        const int a = boundary_column(s, M, lo, rel_tol), b = boundary_column(s, M, hi, rel_tol);
        if (a < 0 || b < 0 || b - a < 1) return false;
        k0 = a;
        k1 = b + 1;
        return true;
    };
    int w = 0;
    for (int n = 1; n <= n_max; ++n) {
        for (int su : {1, -1}) {
            int a0, a1;
            if (!range(sA, MA, su * Du * std::pow(lam_u, n - 1), su * Du * std::pow(lam_u, n), a0, a1)) {
                g_err = "tms_layer_pairs: a U half-layer boundary is not a stored s value (layer " +
                        std::to_string(n) + ")";
                return TMS_ERR_ARG;
            }
            for (int m : {n, n - 1}) {
                for (int ss : {1, -1}) {
                    int b0, b1;
                    if (!range(sB, MB, ss * Ds / std::pow(lam_s, m - 1), ss * Ds / std::pow(lam_s, m),
                               b0, b1)) {
                        g_err = "tms_layer_pairs: an S half-layer boundary is not a stored s value "
                                "(layer " + std::to_string(m) + ")";
                        return TMS_ERR_ARG;
                    }
                    if (w < cap) {
                        tms_layer_pair &p = out[w];
                        p.n = n;
                        p.m = m;
                        p.sign_u = su;
                        p.sign_s = ss;
                        p.a_k0 = a0;
                        p.a_k1 = a1;
                        p.b_k0 = b0;
                        p.b_k1 = b1;
                    }
                    ++w;
                }
            }
        }
    }
    if (cap < total) {
        g_err = "tms_layer_pairs: output too small";
        return TMS_ERR_CAPACITY;
    }
    return TMS_OK;
}

tms_status tms_layer_plan_destroy(tms_layer_plan plan) {
    if (!plan || plan->magic != kLayerMagic) return TMS_ERR_STATE;
    for (tms_mesh m : plan->owned) tms_destroy_mesh(m);
    cudaFree(plan->d_shift);
    plan->magic = 0;
    delete plan;
    return TMS_OK;
}

tms_status tms_layer_plan_create(tms_mesh A, tms_mesh B, const tms_layer_pair *pairs, int nPairs,
                                 void *stream, tms_layer_plan *out) {
    if (!out) return TMS_ERR_ARG;
    *out = nullptr;
    if (!A || !B || A->magic != kMagic || B->magic != kMagic) return TMS_ERR_STATE;
    if (!pairs || nPairs < 1) { g_err = "tms_layer_plan_create: no pairs"; return TMS_ERR_ARG; }
    if (2ULL * A->N * (unsigned long long)A->M >= (1ULL << 32) ||
        2ULL * B->N * (unsigned long long)B->M >= (1ULL << 32)) {
        g_err = "tms_layer_plan_create: mesh too large for 32-bit triangle ids";
        return TMS_ERR_ARG;
    }
    for (int p = 0; p < nPairs; ++p) {
        const tms_layer_pair &q = pairs[p];
        if (q.a_k0 < A->k0 || q.a_k1 > A->k1 || q.a_k1 - q.a_k0 < 2 || q.b_k0 < B->k0 ||
            q.b_k1 > B->k1 || q.b_k1 - q.b_k0 < 2) {
            g_err = "tms_layer_plan_create: pair " + std::to_string(p) + " outside the meshes";
            return TMS_ERR_ARG;
        }
    }
    tms_layer_plan P = new tms_layer_plan_s();
    P->magic = kLayerMagic;
    P->nPairs = nPairs;
    P->d_shift = nullptr;
    std::map<std::pair<int, int>, tms_mesh> va, vb;
    auto view = [&](tms_mesh full, std::map<std::pair<int, int>, tms_mesh> &cache, int k0, int k1,
                    tms_mesh *h) -> tms_status {
        auto it = cache.find({k0, k1});
        if (it != cache.end()) { *h = it->second; return TMS_OK; }
        const size_t off = (size_t)full->k0 * full->N;
        tms_status st = tms_build_mesh(full->dev.c[0] - off, full->dev.c[1] - off,
                                       full->dev.c[2] - off, full->dev.c[3] - off, full->N, full->M,
                                       k0, k1, full->d_s, full->dev.periodic, stream, h);
        if (st != TMS_OK) return st;
        cache[{k0, k1}] = *h;
        P->owned.push_back(*h);
        return TMS_OK;
    };
    std::vector<uint2> shift(nPairs);
    for (int p = 0; p < nPairs; ++p) {
        const tms_layer_pair &q = pairs[p];
        tms_mesh ha = nullptr, hb = nullptr;
        tms_status st = view(A, va, q.a_k0, q.a_k1, &ha);
        if (st == TMS_OK) st = view(B, vb, q.b_k0, q.b_k1, &hb);
        if (st != TMS_OK) { tms_layer_plan_destroy(P); return st; }
        P->A.push_back(ha);
        P->B.push_back(hb);
        shift[p] = make_uint2((unsigned)(2LL * A->N * (q.a_k0 - A->k0)),
                              (unsigned)(2LL * B->N * (q.b_k0 - B->k0)));
    }
    cudaError_t e = cudaMalloc((void **)&P->d_shift, nPairs * sizeof(uint2));
    if (e == cudaSuccess)
        e = cudaMemcpy(P->d_shift, shift.data(), nPairs * sizeof(uint2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        g_err = cudaGetErrorString(e);
        tms_layer_plan_destroy(P);
        return TMS_ERR_CUDA;
    }
    *out = P;
    return TMS_OK;
}

tms_status tms_layer_search(tms_layer_plan plan, const tms_params *params, tms_hit *dHits,
                            long long hitCap, long long *dOffsets, long long *nHits, void *stream) {
    if (!plan || plan->magic != kLayerMagic) return TMS_ERR_STATE;
    if (!dOffsets || !nHits) return TMS_ERR_ARG;
    tms_status st = search_impl(plan->A.data(), plan->B.data(), plan->nPairs, params, dHits, hitCap,
                                dOffsets, nHits, stream);
    if (st != TMS_OK && st != TMS_ERR_CAPACITY) return st;
    const long long n = std::min(*nHits, hitCap);
    if (n > 0) {
        k_layer_ids<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
            dHits, n, plan->d_shift, plan->nPairs);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { g_err = cudaGetErrorString(e); return TMS_ERR_CUDA; }
    }
    return st;
}

}  // extern "C"

// tms_search_noalloc: the mesh search for callers that must not allocate.
//
// Some callers cannot call cudaMalloc: flight- or control-loop software that
// fixes its device footprint at start-up and forbids allocation afterwards,
// services whose device memory is entirely held by a pool allocator (a direct
// cudaMalloc would fail or fragment the pool), and embedded hosts that budget
// every device byte when they start.  For them this entry point runs
// the same kernels as tms_search with every scratch buffer carved from one
// file-scope static __device__ array.  That array (kArenaBytes) is part of the
// library image: every GPU that loads the library holds it until the process
// exits.  The caller still owns and passes the inputs (mesh handles) and the
// output buffer.
//
// Limits, fixed by the arena's size: at most kMaxViewVertices vertices per
// mesh view, kEntCap face-cell entries, kCandCap candidates, kSurvCap FP64
// solves and kRawHitCap hits before merging.  A call that needs more returns
// TMS_ERR_ARG (mesh too large) or TMS_ERR_CAPACITY (a stage overflowed) with a
// message in tms_last_error(); it never grows anything.
//
// The broad phase runs on the faces themselves (the patch level of tms_search
// is not used: tms_params.patch is ignored); the hit set and every hit record
// are the same.
//
// Every call shares the one array and leaves its contents behind; each call
// clears what must start at zero (counters, occupancy bitmaps).  Calls whose
// GPU work overlaps -- on two streams, or from two host threads -- race on the
// array: the caller must order them.  The first call on a device looks up the
// array's device address (cudaGetSymbolAddress) with that device current and
// configures the kernels; make that first call before any stream capture.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "tms_common.cuh"

using namespace tms;

namespace {

constexpr size_t kArenaBytes = 72ull << 20;
constexpr unsigned long long kMaxViewVertices = 1ull << 17;
constexpr unsigned long long kEntCap = 1ull << 18;
// cell table slots: twice the entry limit, so that even a call at that limit
// (at most one distinct cell per entry) keeps the table at most half full and
// its linear probes short
constexpr unsigned long long kTableSize = 2 * kEntCap;
constexpr unsigned long long kCandCap = 1ull << 18;
constexpr unsigned long long kSurvCap = 1ull << 16;
constexpr unsigned long long kRawHitCap = 1ull << 14;
constexpr int kBmAWordBits = 17;   // 2^17 words = 4 Mi bits
constexpr int kBmHWordBits = 16;
constexpr int kMaxGrid = 1024;
constexpr int kMaxTriBits = 18;    // triangles of a view: 2 N (M-1) < 2^18

static __device__ __align__(256) unsigned char g_arena[kArenaBytes];

std::mutex g_mu;
unsigned char *g_base[64] = {};
thread_local std::string g_msg;

struct Carve {
    uintptr_t base;      // the arena's address (0 when only the size is wanted)
    size_t off = 0;
    template <typename T>
    T *take(unsigned long long n) {
        off = (off + 255) & ~(size_t)255;
        T *p = reinterpret_cast<T *>(base + off);
        off += (size_t)n * sizeof(T);
        return p;
    }
};

struct Tables {
    MeshDev meshes[2];
    int2 pairs[1];
    PassEntry all[2], pa[1], pb[1];
};

struct Buffers {
    Tables *tables;
    Bounds *bounds;
    Grid *grids;
    Counters *ctr;
    unsigned long long *partials;
    float4 *split[2];
    unsigned char *fbox[2];
    uint32_t *bmA, *bmH;
    uint64_t *ek;
    uint32_t *ev, *eslot, *erank, *grouped;
    unsigned long long *tkey;
    CellRec *crec;
    uint2 *tcnt;
    uint2 *tstart;
    void *sort_scratch;
    Cand *cand, *surv;
    uint32_t *qsurv;
    tms_hit *hits;
    uint64_t *hk, *hk2, *okeys;
    uint32_t *hv, *hv2, *keep, *kscan;
};

// the arena's layout; also used to check, at set-up, that it fits.  Buffers
// live across the whole search (and the cell table, which every call leaves
// with all slots free) come first; then the broad phase's
// buffers, and over the same bytes the narrow phase's and the merge's, which
// are written only after candidate emission, the broad phase's last reader,
// has run on the same stream.  The array starts zeroed: every table slot free.
size_t carve(unsigned char *base, Buffers &b) {
    Carve c{reinterpret_cast<uintptr_t>(base)};
    b.tables = c.take<Tables>(1);
    b.bounds = c.take<Bounds>(2);
    b.grids = c.take<Grid>(1);
    b.ctr = c.take<Counters>(1);
    b.partials = c.take<unsigned long long>(5 * kMaxGrid);
    b.split[0] = c.take<float4>(2 * kMaxViewVertices);
    b.split[1] = c.take<float4>(2 * kMaxViewVertices);
    b.sort_scratch = c.take<unsigned char>(radix_scratch_size(kRawHitCap, 2 * kMaxTriBits));
    b.cand = c.take<Cand>(kCandCap);
    b.tkey = c.take<unsigned long long>(kTableSize);
    b.tcnt = c.take<uint2>(kTableSize);
    const size_t phase = c.off;
    // broad phase: face boxes (two per quad, FP64 at most), bitmaps, entries, cells
    b.fbox[0] = c.take<unsigned char>(2 * kMaxViewVertices * 64);
    b.fbox[1] = c.take<unsigned char>(2 * kMaxViewVertices * 64);
    b.bmA = c.take<uint32_t>(1ull << kBmAWordBits);
    b.bmH = c.take<uint32_t>(1ull << kBmHWordBits);
    b.ek = c.take<uint64_t>(kEntCap);
    b.ev = c.take<uint32_t>(kEntCap);
    b.eslot = c.take<uint32_t>(kEntCap);
    b.erank = c.take<uint32_t>(kEntCap);
    b.grouped = c.take<uint32_t>(kEntCap);
    b.tstart = c.take<uint2>(kTableSize);
    // per cell: a cell holding both meshes has at least two entries
    b.crec = c.take<CellRec>(kEntCap / 2);
    const size_t broad_end = c.off;
    // narrow phase and merge, over the broad phase's bytes
    c.off = phase;
    b.surv = c.take<Cand>(kSurvCap);
    b.qsurv = c.take<uint32_t>(kCandCap);
    b.hits = c.take<tms_hit>(kRawHitCap);
    b.hk = c.take<uint64_t>(kRawHitCap);
    b.hk2 = c.take<uint64_t>(kRawHitCap);
    b.okeys = c.take<uint64_t>(kRawHitCap);
    b.hv = c.take<uint32_t>(kRawHitCap);
    b.hv2 = c.take<uint32_t>(kRawHitCap);
    b.keep = c.take<uint32_t>(kRawHitCap);
    b.kscan = c.take<uint32_t>(kRawHitCap);
    return std::max(broad_end, c.off);
}

int ceil_log2u(unsigned long long v) {
    int b = 0;
    while ((1ULL << b) < v && b < 63) ++b;
    return b;
}

#define NA_CK(call)                                                             \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            g_msg = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return TMS_ERR_CUDA;                                                \
        }                                                                       \
    } while (0)

// once per device, with that device current: the arena's device address
tms_status setup(int device, unsigned char **base) {
    if (device < 0 || device >= 64) {
        g_msg = "device index outside 0..63";
        return TMS_ERR_ARG;
    }
    if (g_base[device]) {
        *base = g_base[device];
        return TMS_OK;
    }
    void *p = nullptr;
    NA_CK(cudaGetSymbolAddress(&p, g_arena));
    NA_CK(configure_face_pass());
    configure_emit();
    configure_narrow();
    Buffers probe;
    if (carve(reinterpret_cast<unsigned char *>(p), probe) > kArenaBytes) {
        g_msg = "scratch layout exceeds the static arena";
        return TMS_ERR_STATE;
    }
    g_base[device] = reinterpret_cast<unsigned char *>(p);
    *base = g_base[device];
    return TMS_OK;
}

}  // namespace

extern "C" const char *tms_noalloc_last_error(void) { return g_msg.c_str(); }

extern "C" tms_status tms_noalloc_footprint(unsigned long long *needed, unsigned long long *reserved) {
    if (!needed || !reserved) return TMS_ERR_ARG;
    Buffers b;
    *needed = (unsigned long long)carve(nullptr, b);
    *reserved = (unsigned long long)kArenaBytes;
    return TMS_OK;
}

extern "C" tms_status tms_search_noalloc(tms_mesh A, tms_mesh B, const tms_params *params,
                                         tms_hit *dHits, long long hitCap, long long *nHits,
                                         void *stream) {
    g_msg.clear();
    if (!nHits || hitCap < 0 || (hitCap > 0 && !dHits)) {
        g_msg = "nHits is NULL, hitCap is negative, or dHits is NULL with hitCap > 0";
        return TMS_ERR_ARG;
    }
    tms_params p;
    tms_params_default(&p);
    if (params) p = *params;
    if ((p.precision != 0 && p.precision != 1) || (p.face_level != 0 && p.face_level != 1) ||
        !(p.cell_mult >= 1.0f) || !(p.tau >= 0.0) || !(p.tau < 1.0) || p.spin_limit < 0) {
        g_msg = "invalid search parameters";
        return TMS_ERR_ARG;
    }
    MeshDev ma, mb;
    int devA = -1, devB = -1, device = 0;
    if (mesh_view(A, &ma, &devA) != TMS_OK || mesh_view(B, &mb, &devB) != TMS_OK) {
        g_msg = "mesh handle invalid (NULL or destroyed)";
        return TMS_ERR_STATE;
    }
    NA_CK(cudaGetDevice(&device));
    if (devA != device || devB != device) {
        g_msg = "mesh is on another device than the current one";
        return TMS_ERR_ARG;
    }
    if ((unsigned long long)ma.N * ma.M > kMaxViewVertices ||
        (unsigned long long)mb.N * mb.M > kMaxViewVertices) {
        g_msg = "mesh view has more than 131072 vertices (the static scratch limit)";
        return TMS_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned char *base = nullptr;
    tms_status st = setup(device, &base);
    if (st != TMS_OK) return st;
    Buffers b;
    carve(base, b);

    // small tables, from host memory on the stack
    const int block = (p.block_faces == 64 || p.block_faces == 256) ? p.block_faces : 128;
    const int rows = p.tile_rows == 8 ? 8 : 4;
    Tables t;
    memset(&t, 0, sizeof(t));
    ma.split = b.split[0];
    mb.split = b.split[1];
    ma.fbox = b.fbox[0];
    mb.fbox = b.fbox[1];
    t.meshes[0] = ma;
    t.meshes[1] = mb;
    t.pairs[0] = make_int2(0, 1);
    long long tiles_all = 0;
    long long fslots_all = 0, fslots_A = 0, fslots_B = 0;
    const MeshDev *mv[2] = {&ma, &mb};
    for (int role = 0; role < 2; ++role) {
        PassEntry e;
        e.mesh = role;
        e.pair = 0;
        e.role = role;
        e.tiles_i = (mv[role]->nqi + block - 1) / block;
        const long long nt = (long long)e.tiles_i * ((mv[role]->nqk + rows - 1) / rows);
        e.faces = (long long)face_slots(*mv[role], p.face_level);
        const long long padded = (e.faces + 31) / 32 * 32;
        e.tile_base = tiles_all;
        e.face_base = fslots_all;
        t.all[role] = e;
        tiles_all += nt;
        fslots_all += padded;
        e.tile_base = 0;
        e.face_base = 0;
        if (role == 0) { t.pa[0] = e; fslots_A = padded; }
        else { t.pb[0] = e; fslots_B = padded; }
    }
    unsigned long long max_tri = std::max(2ULL * ma.N * ma.nqk, 2ULL * mb.N * mb.nqk);
    const int tri_bits = ceil_log2u(max_tri);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int grid = std::min(kMaxGrid, 2 * sms);
    NA_CK(cudaMemcpyAsync(b.tables, &t, sizeof(t), cudaMemcpyHostToDevice, s));

    // the launch sequence of tms_search, on the static buffers
    launch_search_init(b.bounds, 2, b.ctr, p.cell_filter ? b.bmA : nullptr, 1ull << kBmAWordBits,
                       p.cell_filter ? b.bmH : nullptr, 1ull << kBmHWordBits, grid, s);
    GroupArgs ga;
    ga.ent_key = b.ek; ga.ent_face = b.ev; ga.d_n = &b.ctr->entries; ga.cap = kEntCap;
    ga.ent_slot = b.eslot; ga.ent_rank = b.erank;
    ga.tkey = b.tkey; ga.tcnt = b.tcnt; ga.tstart = b.tstart; ga.tsize = kTableSize;
    ga.cells = b.crec; ga.grids = b.grids;
    ga.grouped = b.grouped; ga.partials = b.partials; ga.ctr = b.ctr;
    FacePassArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.meshes = b.tables->meshes;
    fa.tile_rows = rows;
    fa.bounds = b.bounds;
    fa.grids = b.grids;
    fa.bmA = b.bmA;
    fa.bmA_word_bits = kBmAWordBits;
    fa.bmH = b.bmH;
    fa.bmH_word_bits = kBmHWordBits;
    fa.ent_key = b.ek;
    fa.ent_val = b.ev;
    fa.ctr = b.ctr;
    fa.ent_cap = kEntCap;
    fa.entries = b.tables->all; fa.n_entries = 2; fa.total_tiles = tiles_all;
    fa.mode = MODE_BOUNDS;
    launch_face_pass(fa, p.precision, p.face_level, block, s);
    launch_grid_params(b.bounds, b.tables->pairs, 1, b.grids, p.cell_mult, s);
    if (p.cell_filter) {
        fa.entries = b.tables->pa; fa.n_entries = 1; fa.total_faces = fslots_A;
        fa.mode = MODE_MARK;
        launch_face_pass(fa, p.precision, p.face_level, block, s);
        fa.entries = b.tables->pb; fa.total_faces = fslots_B;
        fa.mode = MODE_PROBE_MARK;
        launch_face_pass(fa, p.precision, p.face_level, block, s);
        fa.entries = b.tables->pa; fa.total_faces = fslots_A;
        fa.mode = MODE_PROBE;
        launch_face_pass(fa, p.precision, p.face_level, block, s);
    } else {
        fa.entries = b.tables->all; fa.n_entries = 2; fa.total_faces = fslots_all;
        fa.mode = MODE_EMIT_ALL;
        launch_face_pass(fa, p.precision, p.face_level, block, s);
    }
    launch_group_count(ga, grid, s);
    launch_group_cells(ga, grid, s);
    EmitArgs ea;
    ea.cells = b.crec; ea.vals = b.grouped;
    ea.grids = b.grids; ea.meshes = b.tables->meshes; ea.pairs = b.tables->pairs; ea.ctr = b.ctr;
    ea.ent_cap = kEntCap; ea.cand = b.cand; ea.cand_cap = kCandCap; ea.moller = p.moller;
    ea.cand_ctr = &b.ctr->cand;
    ea.waves = 0;
    launch_emit(ea, p.precision, p.face_level, grid / 2, s);
    NarrowArgs na;
    na.cand = b.cand; na.cand_cap = kCandCap; na.surv = b.surv; na.surv_cap = kSurvCap;
    na.qsurv = b.qsurv;
    na.meshes = b.tables->meshes; na.pairs = b.tables->pairs; na.ctr = b.ctr; na.hits = b.hits;
    na.hit_key = b.hk; na.hit_val = b.hv; na.hit_cap = kRawHitCap; na.tau = p.tau;
    na.tri_bits = tri_bits; na.fp32_filter = p.narrow_filter;
    launch_narrow(na, p.face_level, grid / 2, grid * 4, s);
    const bool halt = radix_sort(b.hk, b.hv, b.hk2, b.hv2, b.sort_scratch, &b.ctr->raw_hits, kRawHitCap,
                                 2 * tri_bits, 2 * grid, &b.ctr->status,
                                 (unsigned long long)p.spin_limit, (p.inject & 16u) ? 1 : 0, s);
    DedupArgs da;
    da.keys = halt ? b.hk2 : b.hk; da.vals = halt ? b.hv2 : b.hv; da.raw = b.hits;
    da.meshes = b.tables->meshes; da.pairs = b.tables->pairs; da.ctr = b.ctr; da.raw_cap = kRawHitCap;
    da.keep = b.keep; da.keep_scan = b.kscan; da.partials = b.partials;
    da.out = dHits; da.out_cap = (unsigned long long)hitCap; da.out_keys = b.okeys;
    da.offsets = nullptr; da.n_pairs = 1; da.tri_bits = tri_bits; da.tau = p.tau;
    launch_dedup(da, grid, s);
    NA_CK(cudaGetLastError());

    Counters c;
    NA_CK(cudaMemcpyAsync(&c, b.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (c.status & ST_NONFINITE) {
        g_msg = "non-finite vertex coordinate";
        return TMS_ERR_ARG;
    }
    if (c.status & ST_PAIR_LIMIT) {
        g_msg = "grid proposes too many face pairs (degenerate geometry)";
        return TMS_ERR_ARG;
    }
    if (c.status & ST_TIMEOUT) {
        g_msg = "a device-side wait gave up (sort look-back)";
        return TMS_ERR_TIMEOUT;
    }
    if (c.status & ST_TABLE_FULL) {
        g_msg = "cell table full";
        return TMS_ERR_STATE;
    }
    if (c.entries > kEntCap || c.cand > kCandCap || c.fp64 > kSurvCap || c.raw_hits > kRawHitCap) {
        g_msg = "a search stage exceeded the static scratch limits";
        *nHits = -1;
        return TMS_ERR_CAPACITY;
    }
    *nHits = (long long)c.out;
    if ((long long)c.out > hitCap) {
        g_msg = "hit buffer too small";
        return TMS_ERR_CAPACITY;
    }
    return TMS_OK;
}

// Candidate-pair emission of the broad phase.
//
// Input: the face ids grouped by cell, mesh A's first (tms_group.cu), with per
// cell its key, the start of its A and B lists and the exclusive scan of its
// 32 x 32 tiles.  nA * nB is the number of face pairs a cell proposes; its
// exclusive scan is the paper's box_gid_idxs array (Sec. 6.3, Algorithm 1).
//
// Emission re-designed for GB300: the nA x nB pair matrix of a cell is cut
// into 32 x 32 tiles and one warp tests one tile -- each lane holds one A box
// in registers, the tile's B boxes sit in shared memory and are read by
// broadcast, so a proposed pair costs a few compares and no memory traffic.
// (Algorithm 1 gives every proposed pair its own work item that locates its
// box with a linear walk and fetches vertices.)  Per pair: the bounding-box
// test of Sec. 6.2.2, then the owner-cell rule -- the pair is kept only in the
// cell that is the componentwise max of the two faces' lowest cells, so a pair
// sharing several cells is emitted exactly once -- then optionally the Moller
// quick test of Sec. 6.2.3.  Each lane collects the tile's overlaps as a bit
// mask over the rows (no vote per row: at about 3% overlapping pairs most
// groups of rows hold one somewhere in the warp); the owner rule is applied
// per tile from four ballots of the rows' owned coordinates; one warp scan
// places the survivors in a per-warp stage that is appended at one atomic per
// 64 or more.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tms_common.cuh"

namespace tms {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kTile = 32;
constexpr int kEmitWarps = 8;
constexpr unsigned kCandFlush = 64;    // the stage is appended once it holds this many
constexpr unsigned kStageCap = 192;    // staged candidates per warp

// ---------------------------------------------------------------------------
// emission
// ---------------------------------------------------------------------------
// a face's box from its mesh's face-box array (written by the bounds pass)
template <int PREC>
struct EBox;
template <>
struct __align__(16) EBox<1> {
    typedef float4 Half;
    float lo[4], hi[4];
    __device__ void store_halves(Half &l, Half &h) const {
        l = make_float4(lo[0], lo[1], lo[2], lo[3]);
        h = make_float4(hi[0], hi[1], hi[2], hi[3]);
    }
    // closed overlap of two boxes given by halves (touching is overlap)
    static __device__ __forceinline__ bool halves_overlap(const Half &xl, const Half &xh, const Half &yl,
                                                          const Half &yh) {
        const float4 a = xl, b = xh, c = yl, d = yh;
        return !(b.x < c.x) & !(d.x < a.x) & !(b.y < c.y) & !(d.y < a.y) & !(b.z < c.z) & !(d.z < a.z) &
               !(b.w < c.w) & !(d.w < a.w);
    }
    __device__ void load(const void *fbox, uint32_t face) {
        const float4 *p = reinterpret_cast<const float4 *>(fbox) + 2 * (size_t)face;
        const float4 l = __ldg(p), h = __ldg(p + 1);
        lo[0] = l.x; lo[1] = l.y; lo[2] = l.z; lo[3] = l.w;
        hi[0] = h.x; hi[1] = h.y; hi[2] = h.z; hi[3] = h.w;
    }
    // a box that overlaps nothing
    __device__ void set_empty() {
#pragma unroll
        for (int d = 0; d < 4; ++d) { lo[d] = __int_as_float(0x7f800000); hi[d] = -lo[d]; }
    }
    // the face's lowest cell, as the cell passes compute it, 4 x u16
    __device__ uint2 low_cell(const Grid &g) const {
        int c[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) c[d] = cell_of(lo[d], g.o32[d], g.inv32[d], g.n[d]);
        return make_uint2((uint32_t)c[0] | ((uint32_t)c[1] << 16), (uint32_t)c[2] | ((uint32_t)c[3] << 16));
    }
};
template <>
struct __align__(16) EBox<0> {
    struct __align__(16) Half { double v[4]; };
    double lo[4], hi[4];
    __device__ void store_halves(Half &l, Half &h) const {
#pragma unroll
        for (int d = 0; d < 4; ++d) { l.v[d] = lo[d]; h.v[d] = hi[d]; }
    }
    static __device__ __forceinline__ bool halves_overlap(const Half &xl, const Half &xh, const Half &yl,
                                                          const Half &yh) {
        bool ov = true;
#pragma unroll
        for (int d = 0; d < 4; ++d) ov &= !(xh.v[d] < yl.v[d]) & !(yh.v[d] < xl.v[d]);
        return ov;
    }
    __device__ void load(const void *fbox, uint32_t face) {
        const double2 *p = reinterpret_cast<const double2 *>(fbox) + 4 * (size_t)face;
        const double2 x0 = __ldg(p), x1 = __ldg(p + 1), x2 = __ldg(p + 2), x3 = __ldg(p + 3);
        lo[0] = x0.x; lo[1] = x0.y; lo[2] = x1.x; lo[3] = x1.y;
        hi[0] = x2.x; hi[1] = x2.y; hi[2] = x3.x; hi[3] = x3.y;
    }
    __device__ void set_empty() {
#pragma unroll
        for (int d = 0; d < 4; ++d) { lo[d] = __longlong_as_double(0x7ff0000000000000LL); hi[d] = -lo[d]; }
    }
    __device__ uint2 low_cell(const Grid &g) const {
        int c[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) c[d] = cell_of(lo[d], g.o64[d], g.inv64[d], g.n[d]);
        return make_uint2((uint32_t)c[0] | ((uint32_t)c[1] << 16), (uint32_t)c[2] | ((uint32_t)c[3] << 16));
    }
};


// Moller quick test (Sec. 6.2.3) on the (x, y, px) projection.  The plane of a
// triangle (x1, x2, x3) has normal (x1 - x2) x (x3 - x2); a point set lies
// strictly on one side when f = n . (X - x2) has one strict sign at all points.
// A rounding guard makes the test conservative: a value counts as signed only
// beyond a bound on its rounding error.
__device__ __forceinline__ bool same_side(const double x1[4], const double x2[4], const double x3[4],
                                          const double (*P)[4], int np) {
    double u[3], v[3];
    for (int c = 0; c < 3; ++c) { u[c] = x1[c] - x2[c]; v[c] = x3[c] - x2[c]; }
    double nrm[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    double un = fabs(u[0]) + fabs(u[1]) + fabs(u[2]);
    double vn = fabs(v[0]) + fabs(v[1]) + fabs(v[2]);
    int pos = 0, neg = 0;
    for (int j = 0; j < np; ++j) {
        double w[3];
        for (int c = 0; c < 3; ++c) w[c] = P[j][c] - x2[c];
        double f = nrm[0] * w[0] + nrm[1] * w[1] + nrm[2] * w[2];
        double wn = fabs(w[0]) + fabs(w[1]) + fabs(w[2]);
        double guard = 32.0 * 1.1102230246251565e-16 * un * vn * wn;
        if (f > guard) ++pos;
        else if (f < -guard) ++neg;
    }
    return pos == np || neg == np;
}

__device__ __forceinline__ void face_vertices(const MeshDev &m, uint32_t face, int face_level,
                                              double V[4][4], int &nv) {
    if (face_level == 0) {
        int ii[3], kk[3];
        tri_ij(m, face, ii, kk);
        for (int j = 0; j < 3; ++j) load_vertex(m, ii[j], kk[j], V[j]);
        nv = 3;
    } else {
        int i = (int)(face % (uint32_t)m.N), k = (int)(face / (uint32_t)m.N);
        int ip = (i + 1 == m.N) ? 0 : i + 1;
        load_vertex(m, i, k, V[0]);        // (i, k)
        load_vertex(m, ip, k, V[1]);       // (i+1, k)
        load_vertex(m, i, k + 1, V[2]);    // (i, k+1)
        load_vertex(m, ip, k + 1, V[3]);   // (i+1, k+1)
        nv = 4;
    }
}

// true when the Moller test proves the two faces disjoint
__device__ bool moller_reject(const MeshDev &ma, uint32_t fa, const MeshDev &mb, uint32_t fb,
                              int face_level) {
    double VA[4][4], VB[4][4];
    int na, nb;
    face_vertices(ma, fa, face_level, VA, na);
    face_vertices(mb, fb, face_level, VB, nb);
    if (face_level == 0) {
        if (same_side(VA[0], VA[1], VA[2], VB, 3)) return true;
        return same_side(VB[0], VB[1], VB[2], VA, 3);
    }
    // quads: all four vertices of one quad on one side of the planes of both
    // triangles of the other (T1 = (i+1,k),(i,k),(i,k+1); T2 = (i,k+1),(i+1,k+1),(i+1,k))
    if (same_side(VA[1], VA[0], VA[2], VB, 4) && same_side(VA[2], VA[3], VA[1], VB, 4)) return true;
    return same_side(VB[1], VB[0], VB[2], VA, 4) && same_side(VB[2], VB[3], VB[1], VA, 4);
}

// the coordinates in which a face's lowest cell is this cell: bit d set when
// lo_d == cur_d (both packed 4 x u16); a face in the cell has lo_d <= cur_d
__device__ __forceinline__ uint32_t own_mask(uint2 lo, uint2 cur) {
    const uint32_t ex = __vcmpeq2(lo.x, cur.x), ey = __vcmpeq2(lo.y, cur.y);
    return (ex & 1u) | ((ex >> 15) & 2u) | ((ey & 1u) << 2) | ((ey >> 13) & 8u);
}

template <int PREC>
__device__ __forceinline__ bool boxes_overlap(const EBox<PREC> &x, const EBox<PREC> &y) {
    bool ov = true;
#pragma unroll
    for (int d = 0; d < 4; ++d) ov &= !(x.hi[d] < y.lo[d]) & !(y.hi[d] < x.lo[d]);
    return ov;
}

template <int PREC, bool MOLLER>
__global__ void __launch_bounds__(32 * kEmitWarps, (PREC == 1 && !MOLLER) ? 5 : 2) k_emit(EmitArgs a, int face_level) {
    // the tile's B side: boxes (read by broadcast in the hot loop) and face ids
    __shared__ EBox<PREC> sBox[kEmitWarps][kTile];
    __shared__ uint32_t sFace[kEmitWarps][kTile];
    __shared__ Cand sOut[kEmitWarps][kStageCap];   // staged candidates
    // nothing to do after an entry overflow (the host retries with more room),
    // and a bounded amount of work in any case
    if (a.ctr->entries > a.ent_cap) return;
    if (a.ctr->pair_slots > kMaxPairSlots) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctr->status, ST_PAIR_LIMIT);
        return;
    }
    const unsigned long long total_tiles = a.ctr->tiles;
    const unsigned long long ncell = clamp_count(&a.ctr->cells, a.ent_cap);
    const unsigned long long nent = clamp_count(&a.ctr->grouped, a.ent_cap);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long gw = blockIdx.x * (unsigned long long)kEmitWarps + warp;
    const unsigned long long nw = (unsigned long long)gridDim.x * kEmitWarps;
    // each warp owns a contiguous range of tiles: one search for its first
    // tile's cell, then a forward walk over the cells
    const unsigned long long per = (total_tiles + nw - 1) / nw;
    const unsigned long long t_begin = gw * per;
    const unsigned long long t_end = min(t_begin + per, total_tiles);
    Cand *stage = sOut[warp];
    unsigned staged = 0;                       // warp-uniform
    const unsigned long long cap = a.cand_cap;
    Cand *cand_out = a.cand;
    // the whole stage to one atomically reserved range of the candidate array
    auto flush = [&]() {
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.cand_ctr, (unsigned long long)staged);
        base = __shfl_sync(FULL, base, 0);
        for (unsigned k = lane; k < staged; k += 32)
            if (base + k < cap) cand_out[base + k] = stage[k];
        __syncwarp();
        staged = 0;
    };
    // the last cell whose first tile is at or before t_begin (cell 0 starts at
    // tile 0; tile offsets increase strictly): a 32-way search, each step one
    // probe per lane and one vote, about four dependent steps for 10^5 cells
    unsigned long long c = 0;
    if (t_begin < t_end) {
        unsigned long long lo = 0, hi = ncell - 1;
        while (lo < hi) {
            const unsigned long long span = hi - lo;
            // probe k at lo + (k + 1) * span / 32 (k < span when span < 32); the
            // probes rise with k, so the lanes at or before t_begin are a prefix
            const unsigned long long q = lo + ((unsigned long long)(lane + 1) * span) / 32;
            const bool probe = span >= 32 || (unsigned long long)lane < span;
            const unsigned long long qq = span >= 32 ? q : lo + 1 + lane;
            const bool le = probe && a.cells[qq].tile_off <= t_begin;
            const int n_le = __popc(__ballot_sync(FULL, le));
            const int n_probe = span >= 32 ? 32 : (int)span;
            const unsigned long long q_le = n_le ? __shfl_sync(FULL, qq, n_le - 1) : lo;
            const unsigned long long q_gt = __shfl_sync(FULL, qq, n_le < n_probe ? n_le : 0);
            lo = q_le;
            hi = n_le < n_probe ? q_gt - 1 : hi;
        }
        c = lo;
    }
    // the lanes' face, kept across tiles of one A row: its box and the
    // coordinates in which it is not in its lowest cell (its partner must be)
    EBox<PREC> abox;
    abox.set_empty();
    uint32_t aneed = 0, aface = 0;
    uint32_t prev_a0 = 0xFFFFFFFFu;
    unsigned long long prev_c = ~0ULL;
    bool prev_swap = true;
    // the pair's face-box arrays, looked up again only when the pair changes
    uint32_t cached_pair = 0xFFFFFFFFu;
    const void *fbA = nullptr, *fbB = nullptr;
    int2 pr = make_int2(0, 0);
    for (unsigned long long t = t_begin; t < t_end; ++t) {
        while (c + 1 < ncell && a.cells[c + 1].tile_off <= t) ++c;
        const CellRec cr = a.cells[c];
        const uint32_t s = cr.start;
        const uint32_t bstart = cr.bstart;
        const uint32_t e = (c + 1 < ncell) ? a.cells[c + 1].start : (uint32_t)nent;
        const uint32_t nBc = e - bstart;
        const uint32_t tB = (nBc + kTile - 1) / kTile;
        const uint32_t local = (uint32_t)(t - cr.tile_off);
        // B-fastest order: consecutive tiles of a cell share their A row
        const uint32_t a0 = s + (local / tB) * kTile, b0 = bstart + (local % tB) * kTile;
        const int nAt0 = (int)min((uint32_t)kTile, bstart - a0);
        const int nBt0 = (int)min((uint32_t)kTile, e - b0);
        // lanes take the larger side of the tile, the loop the smaller one
        const bool swapAB = nBt0 > nAt0;
        const uint32_t l0 = swapAB ? b0 : a0, m0 = swapAB ? a0 : b0;
        const int nAt = swapAB ? nBt0 : nAt0, nBt = swapAB ? nAt0 : nBt0;
        const uint32_t pair = cr.pair;
        const uint2 cur = cr.xy;
        const Grid &gr = a.grids[pair];
        if (pair != cached_pair) {
            pr = a.pairs[pair];
            fbA = a.meshes[pr.x].fbox;
            fbB = a.meshes[pr.y].fbox;
            cached_pair = pair;
        }
        // own entry (the lanes' side) in registers, the other side in shared memory
        const void *fbL = swapAB ? fbB : fbA, *fbM = swapAB ? fbA : fbB;
        // the lanes keep their face when the previous tile had the same A row on
        // the lanes' side (a full A row always does: only a partial one swaps)
        const bool reuse = !swapAB && !prev_swap && a0 == prev_a0 && c == prev_c;
        prev_swap = swapAB;
        prev_a0 = a0;
        prev_c = c;
        if (!reuse) {
            abox.set_empty();
            if (lane < nAt) {
                aface = a.vals[l0 + lane];
                abox.load(fbL, aface);
                aneed = ~own_mask(abox.low_cell(gr), cur) & 0xFu;
            }
        }
        // every row of the B side is written; rows past nBt hold an empty box
        EBox<PREC> bb;
        bb.set_empty();
        uint32_t bown = 0;
        __syncwarp();                          // the previous tile's rows are read
        if (lane < nBt) {
            const uint32_t bface = a.vals[m0 + lane];
            bb.load(fbM, bface);
            bown = own_mask(bb.low_cell(gr), cur);
            sFace[warp][lane] = bface;
        }
        sBox[warp][lane] = bb;
        // owner cell: the componentwise max of the two faces' lowest cells is this
        // cell iff every coordinate is owned by one of them, so a lane's face may
        // pair only with rows owning every coordinate it does not own
        uint32_t rows = ~0u;
        {
            const uint32_t w0 = __ballot_sync(FULL, bown & 1u), w1 = __ballot_sync(FULL, bown & 2u);
            const uint32_t w2 = __ballot_sync(FULL, bown & 4u), w3 = __ballot_sync(FULL, bown & 8u);
            if (aneed & 1u) rows &= w0;
            if (aneed & 2u) rows &= w1;
            if (aneed & 4u) rows &= w2;
            if (aneed & 8u) rows &= w3;
        }
        __syncwarp();
        // the box test against every row, four rows per step
        uint32_t K = 0;
        const int nB4 = (nBt + 3) & ~3;
        for (int j = 0; j < nB4; j += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                K |= (boxes_overlap(abox, sBox[warp][j + u]) ? 1u : 0u) << (j + u);
        }
        K &= rows;
        if (MOLLER) {
            for (uint32_t k = K; k; k &= k - 1) {
                const int j = __ffs(k) - 1;
                const uint32_t bface = sFace[warp][j];
                const uint32_t fa = swapAB ? bface : aface, fb = swapAB ? aface : bface;
                if (moller_reject(a.meshes[pr.x], fa, a.meshes[pr.y], fb, face_level)) K &= ~(1u << j);
            }
        }
        // the survivors' places: a warp scan of the per-lane counts
        const uint32_t cnt = __popc(K);
        uint32_t incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += y;
        }
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        if (total == 0) continue;
        auto cand_of = [&](int j) {
            const uint32_t bface = sFace[warp][j];
            Cand cd;
            cd.faceA = swapAB ? bface : aface;
            cd.faceB = swapAB ? aface : bface;
            cd.pair = pair;
            cd.pad = 0;
            return cd;
        };
        if (staged + total > kStageCap && staged) flush();
        if (total > kStageCap) {
            // a dense tile: its candidates straight to one reserved range
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(a.cand_ctr, (unsigned long long)total);
            base = __shfl_sync(FULL, base, 0);
            unsigned long long pos = base + incl - cnt;
            for (uint32_t k = K; k; k &= k - 1, ++pos)
                if (pos < cap) cand_out[pos] = cand_of(__ffs(k) - 1);
        } else {
            unsigned pos = staged + incl - cnt;
            for (uint32_t k = K; k; k &= k - 1) stage[pos++] = cand_of(__ffs(k) - 1);
            staged += total;
            if (staged >= kCandFlush) flush();
        }
    }
    if (staged) flush();
}

// Whole waves of resident blocks: every warp owns the same number of tiles, so
// a partial last wave would leave SMs idle at the end; several waves let the
// block scheduler even out tiles of unequal cost (dense cells).  Resident
// blocks per SM of each kernel variant, the same on every GB300; looked up by
// configure_emit (outside stream capture) or at the first launch.
constexpr int kEmitWaves = 4;
int g_emit_resident[2][2] = {};

template <int PREC, bool MOLLER>
int emit_resident() {
    int &r = g_emit_resident[PREC][MOLLER ? 1 : 0];
    if (r == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_emit<PREC, MOLLER>, 32 * kEmitWarps, 0) !=
                cudaSuccess || nb < 1)
            nb = 1;
        r = nb;
    }
    return r;
}

template <int PREC, bool MOLLER>
void emit_waves(const EmitArgs &a, int face_level, int sms, cudaStream_t st) {
    const int waves = a.waves > 0 ? a.waves : kEmitWaves;
    k_emit<PREC, MOLLER><<<sms * emit_resident<PREC, MOLLER>() * waves, 32 * kEmitWarps, 0, st>>>(
        a, face_level);
}

// ---------------------------------------------------------------------------
// quad pairs of the patch pairs (patch level)
// ---------------------------------------------------------------------------
constexpr int kPatchWarps = 8;
constexpr unsigned kPatchFlush = 64;   // staged candidates per atomic
constexpr int kQuarterBlock = 128;     // stage 1: one lane per patch pair

// Each patch carries four quarter boxes (2 x 2 blocks of 4 x 2 quads).
// Stage 1 (k_patch_quarters), one lane per patch pair: its 16 quarter pairs; a
// patch pair none of whose quarter pairs overlap holds no overlapping quad pair
// and is dropped before any quad box is read; the others are listed with their
// 16-bit mask (bit 4 i + j: A quarter i meets B quarter j).
// Stage 2 (k_patch_quads), one warp per listed pair, grid-stride: the pair's
// quarter boxes and quad boxes are loaded together (neither waits for the
// other).  Lane l holds quad (row l / kPatchI, column l % kPatchI) of each
// patch; a quad that meets none of the other patch's quarter boxes cannot
// overlap any of its quads (they all lie in those boxes), so each side is cut
// to its quads that meet one.  The survivors' pairs take the box test of
// Sec. 6.2.2 (optionally the Moller test of Sec. 6.2.3) and are appended
// through a per-warp stage: the smaller side's survivors stay in registers, one
// per lane and repeated in G = 32 / n groups of lanes, while each round reads G
// of the other side's survivors from shared memory (close to a broadcast), so a
// round costs two short shared-memory reads and no division.
// patch id -> (patch row, patch column): the quotient by npi from a 64-bit
// reciprocal (exact for 32-bit ids, npi >= 2)
__device__ __forceinline__ void patch_rc(uint32_t patch, uint32_t npi, unsigned long long magic,
                                         uint32_t &pk, uint32_t &pi) {
    pk = npi == 1 ? patch : (uint32_t)__umul64hi((unsigned long long)patch, magic);
    pi = patch - pk * npi;
}

// Patch frames (the record at kFrameF4).  For a direction w the points of a
// patch lie within S(w) of w . c along w, where S(e_m) = h_m along the patch's
// own axis e_m and S(w) = sum_k |fl(w . e_k)| h_k + |w|_1 rho for any other w.
// A triangle of the patch has its vertices among the patch's, so its
// projection lies in that interval, and widened to weights >= -tau' it lies in
// (1 + 6 tau') S(w) of w . c (its length is at most 2 S(w); see widen3).  Two
// patches X, Y are dropped when along some w
//   |w . (c_X - c_Y)| > (1 + 6 tau') (S_X(w) + S_Y(w)) + |w|_1 reach,
// reach the FP64 solve's backward error (fp64_reach) for any triangle pair of
// the two patches: every entry of the system is an edge, |A_ij| <= 2 max(L_X,
// L_Y), and |r| <= L_X + L_Y, so reach <= 1.011e-12 (1 + 2 tau') (L_X + L_Y).  Then no
// triangle pair of the patch pair is an FP64 hit, as in the triangle-level
// separating-axis test.  The left side is computed as
// fl(w . fl(c_X - c_Y)), within 5.001 u sum_i |w_i||fl(c_X - c_Y)_i| of the
// exact value; every bound on the right is rounded up (factor 1.0001).
// Directions: the two completing axes (approximate normals) of each patch,
// then the four directions orthogonal to one patch's parameter directions and
// one of the other's.
struct PFrame {
    float c[4], e[4][4], h[4];
    float rho, L, n2, n3;
};
__device__ __forceinline__ void load_frame(const float4 *f, uint32_t patch, PFrame &F) {
    const float4 *q = f + (size_t)patch * kFrameF4;
    const float4 x0 = __ldg(q), x1 = __ldg(q + 1), x2 = __ldg(q + 2), x3 = __ldg(q + 3);
    const float4 x4 = __ldg(q + 4), x5 = __ldg(q + 5), x6 = __ldg(q + 6);
    F.c[0] = x0.x; F.c[1] = x0.y; F.c[2] = x0.z; F.c[3] = x0.w;
    F.e[0][0] = x1.x; F.e[0][1] = x1.y; F.e[0][2] = x1.z; F.e[0][3] = x1.w;
    F.e[1][0] = x2.x; F.e[1][1] = x2.y; F.e[1][2] = x2.z; F.e[1][3] = x2.w;
    F.e[2][0] = x3.x; F.e[2][1] = x3.y; F.e[2][2] = x3.z; F.e[2][3] = x3.w;
    F.e[3][0] = x4.x; F.e[3][1] = x4.y; F.e[3][2] = x4.z; F.e[3][3] = x4.w;
    F.h[0] = x5.x; F.h[1] = x5.y; F.h[2] = x5.z; F.h[3] = x5.w;
    F.rho = x6.x; F.L = x6.y; F.n2 = x6.z; F.n3 = x6.w;
}
__device__ __forceinline__ float fdot4(const float a[4], const float b[4]) {
    return fmaf(a[3], b[3], fmaf(a[2], b[2], fmaf(a[1], b[1], a[0] * b[0])));
}
// the gap test along w (|w|_1 <= nw) for a patch whose own axis it is (half
// width hx) against patch Y, given pw[k] = fl(w . e_k^Y)
__device__ __forceinline__ bool frame_gap(const float w[4], float nw, float hx, const PFrame &Y,
                                          const float pw[4], const float dc[4], float tw, float reach) {
    const float g = fabsf(fdot4(w, dc));
    const float q = fmaf(fabsf(w[3]), fabsf(dc[3]),
                         fmaf(fabsf(w[2]), fabsf(dc[2]), fmaf(fabsf(w[1]), fabsf(dc[1]), fabsf(w[0]) * fabsf(dc[0]))));
    float sy = nw * Y.rho;
#pragma unroll
    for (int k = 0; k < 4; ++k) sy = fmaf(fabsf(pw[k]), Y.h[k], sy);
    const float need = fmaf(tw, hx + sy, nw * reach);
    return g > fmaf(3.0e-7f, q, need) * 1.0001f;
}
// the vector orthogonal to a, b and c in R^4 (cofactor expansion of the 4 x 4
// determinant with rows (x, a, b, c))
__device__ __forceinline__ float det3f(float a0, float a1, float a2, float b0, float b1, float b2,
                                       float c0, float c1, float c2) {
    return a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0);
}
__device__ __forceinline__ void cross4f(const float a[4], const float b[4], const float c[4], float x[4]) {
    x[0] = det3f(a[1], a[2], a[3], b[1], b[2], b[3], c[1], c[2], c[3]);
    x[1] = -det3f(a[0], a[2], a[3], b[0], b[2], b[3], c[0], c[2], c[3]);
    x[2] = det3f(a[0], a[1], a[3], b[0], b[1], b[3], c[0], c[1], c[3]);
    x[3] = -det3f(a[0], a[1], a[2], b[0], b[1], b[2], c[0], c[1], c[2]);
}
// the gap test along any w: both patches through their frames,
// S(w) = sum_k |fl(w . e_k)| h_k + |w|_1 rho
__device__ __forceinline__ bool frame_gap_any(const float w[4], const PFrame &X, const PFrame &Y,
                                              const float dc[4], float tw, float reach) {
    const float nw = (fabsf(w[0]) + fabsf(w[1]) + fabsf(w[2]) + fabsf(w[3])) * 1.0001f;
    float sx = nw * X.rho, sy = nw * Y.rho;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        sx = fmaf(fabsf(fdot4(w, X.e[k])), X.h[k], sx);
        sy = fmaf(fabsf(fdot4(w, Y.e[k])), Y.h[k], sy);
    }
    const float g = fabsf(fdot4(w, dc));
    const float q = fmaf(fabsf(w[3]), fabsf(dc[3]),
                         fmaf(fabsf(w[2]), fabsf(dc[2]), fmaf(fabsf(w[1]), fabsf(dc[1]), fabsf(w[0]) * fabsf(dc[0]))));
    const float need = fmaf(tw, sx + sy, nw * reach);
    return g > fmaf(3.0e-7f, q, need) * 1.0001f;
}
// true when the frames prove that no triangle pair of the two patches is an
// FP64 hit; tw = 1 + 6 tau' rounded up
__device__ __forceinline__ bool frames_separated(const PFrame &X, const PFrame &Y, float tw) {
    float dc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) dc[i] = X.c[i] - Y.c[i];
    // fp64_reach with max|A| <= 2 (L_X + L_Y) and |r| <= L_X + L_Y; tw = 1 + 6 tau'
    // bounds 1 + 2 tau'
    const float reach = 1.03e-12f * tw * (X.L + Y.L) + 1e-37f;
    // p[m][k] = fl(e_m^X . e_k^Y) for X's normals; q[m][k] = fl(e_m^Y . e_k^X)
    // for Y's normals (its k = 2, 3 entries are p's)
    float p2[4], p3[4], q2[4], q3[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        p2[k] = fdot4(X.e[2], Y.e[k]);
        p3[k] = fdot4(X.e[3], Y.e[k]);
    }
    q2[0] = fdot4(Y.e[2], X.e[0]); q2[1] = fdot4(Y.e[2], X.e[1]); q2[2] = p2[2]; q2[3] = p3[2];
    q3[0] = fdot4(Y.e[3], X.e[0]); q3[1] = fdot4(Y.e[3], X.e[1]); q3[2] = p2[3]; q3[3] = p3[3];
    if (frame_gap(X.e[2], X.n2, X.h[2], Y, p2, dc, tw, reach) ||
        frame_gap(X.e[3], X.n3, X.h[3], Y, p3, dc, tw, reach) ||
        frame_gap(Y.e[2], Y.n2, Y.h[2], X, q2, dc, tw, reach) ||
        frame_gap(Y.e[3], Y.n3, Y.h[3], X, q3, dc, tw, reach))
        return true;
    // mixed directions: orthogonal to one patch's two parameter directions and
    // one of the other's (both patches thin along it when their tangent planes
    // share a direction); any w serves, so w is not normalised
    float w[4];
    cross4f(X.e[0], X.e[1], Y.e[0], w);
    if (frame_gap_any(w, X, Y, dc, tw, reach)) return true;
    cross4f(X.e[0], X.e[1], Y.e[1], w);
    if (frame_gap_any(w, X, Y, dc, tw, reach)) return true;
    cross4f(Y.e[0], Y.e[1], X.e[0], w);
    if (frame_gap_any(w, X, Y, dc, tw, reach)) return true;
    cross4f(Y.e[0], Y.e[1], X.e[1], w);
    return frame_gap_any(w, X, Y, dc, tw, reach);
}

template <int PREC>
__global__ void __launch_bounds__(kQuarterBlock) k_patch_quarters(PatchArgs a) {
    // nothing to do after an overflow of the patch-level grid (the host retries)
    if (a.ctr->entries > a.ent_cap || a.ctr->pair_slots > kMaxPairSlots) return;
    const unsigned long long n = clamp_count(&a.ctr->ppairs, a.ppair_cap);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    uint32_t cached_pair = 0xFFFFFFFFu;
    const void *qbA = nullptr, *qbB = nullptr;
    const float4 *pfA = nullptr, *pfB = nullptr;
    // 1 + 6 tau', tau' = tau + 1e-15 (the margin's rounding), rounded up
    const float tw = 1.0f + 2.0f * widen3(__double2float_ru(a.tau));
    for (unsigned long long j0 = blockIdx.x * (unsigned long long)blockDim.x + (threadIdx.x & ~31u);
         j0 < n; j0 += stride) {
        const unsigned long long j = j0 + (threadIdx.x & 31);
        uint32_t mask = 0;
        Cand pp = {0u, 0u, 0u, 0u};
        if (j < n) {
            pp = a.ppairs[j];
            if (pp.pair != cached_pair) {
                const int2 pr = a.pairs[pp.pair];
                qbA = a.meshes[pr.x].qbox;
                qbB = a.meshes[pr.y].qbox;
                pfA = a.meshes[pr.x].pframe;
                pfB = a.meshes[pr.y].pframe;
                cached_pair = pp.pair;
            }
            EBox<PREC> xa[4], xb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                xa[q].load(qbA, 4 * pp.faceA + q);
                xb[q].load(qbB, 4 * pp.faceB + q);
            }
#pragma unroll
            for (int qa = 0; qa < 4; ++qa)
#pragma unroll
                for (int qb = 0; qb < 4; ++qb)
                    mask |= (uint32_t)boxes_overlap(xa[qa], xb[qb]) << (4 * qa + qb);
            if (a.frames && mask != 0u) {
                PFrame X, Y;
                load_frame(pfA, pp.faceA, X);
                load_frame(pfB, pp.faceB, Y);
                if (frames_separated(X, Y, tw)) mask = 0u;
            }
        }
        pp.pad = mask;
        const unsigned long long pos = warp_append(&a.ctr->psurv, mask != 0u, FULL);
        if (mask != 0u) a.psurv[pos] = pp;
    }
}

template <int PREC, bool MOLLER>
__global__ void __launch_bounds__(32 * kPatchWarps, (PREC == 1 && !MOLLER) ? 3 : 2) k_patch_quads(PatchArgs a) {
    // survivors' boxes as separate low and high halves (16-byte rows for FP32)
    __shared__ typename EBox<PREC>::Half sLo[kPatchWarps][2][32], sHi[kPatchWarps][2][32];
    __shared__ uint32_t sQ[kPatchWarps][2][32];     // survivors' quad ids, [0] A, [1] B
    __shared__ EBox<PREC> sQuart[kPatchWarps][8];   // the pair's quarter boxes, A's then B's
    __shared__ Cand sOut[kPatchWarps][kPatchFlush + 32];
    // nothing to do after an overflow of the patch-level grid (the host retries)
    if (a.ctr->entries > a.ent_cap || a.ctr->pair_slots > kMaxPairSlots) return;
    const unsigned long long n = clamp_count(&a.ctr->psurv, a.ppair_cap);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    const unsigned long long gw = blockIdx.x * (unsigned long long)kPatchWarps + warp;
    const unsigned long long nw = (unsigned long long)gridDim.x * kPatchWarps;
    const int r = lane / kPatchI, c = lane % kPatchI;
    Cand *stage = sOut[warp];
    unsigned staged = 0;
    unsigned long long tests = 0;
    Cand *const cand_out = a.cand;
    const unsigned long long cap = a.cand_cap;
    auto store = [cand_out, cap](unsigned long long pos, const Cand &rec) {
        if (pos < cap) cand_out[pos] = rec;
    };
    uint32_t cached_pair = 0xFFFFFFFFu;
    const void *fbA = nullptr, *fbB = nullptr, *qbA = nullptr, *qbB = nullptr;
    int NA = 1, nqiA = 0, nqkA = 0, NB = 1, nqiB = 0, nqkB = 0;
    uint32_t npiA = 1, npiB = 1;
    unsigned long long mgA = 0, mgB = 0;
    int2 pr = make_int2(0, 0);
    for (unsigned long long j = gw; j < n; j += nw) {
        const Cand pp = a.psurv[j];
        if (pp.pair != cached_pair) {
            pr = a.pairs[pp.pair];
            const MeshDev &ma = a.meshes[pr.x];
            const MeshDev &mb = a.meshes[pr.y];
            fbA = ma.fbox; qbA = ma.qbox; NA = ma.N; nqiA = ma.nqi; nqkA = ma.nqk; npiA = ma.npi;
            fbB = mb.fbox; qbB = mb.qbox; NB = mb.N; nqiB = mb.nqi; nqkB = mb.nqk; npiB = mb.npi;
            mgA = ma.pmagic;
            mgB = mb.pmagic;
            cached_pair = pp.pair;
        }
        // lanes 0..7 load the quarter boxes (A's then B's) while every lane loads
        // its two quad boxes below
        EBox<PREC> xq;
        if (lane < 8) xq.load(lane < 4 ? qbA : qbB, 4 * (lane < 4 ? pp.faceA : pp.faceB) + (lane & 3));
        uint32_t pka, pia, pkb, pib;
        patch_rc(pp.faceA, npiA, mgA, pka, pia);
        patch_rc(pp.faceB, npiB, mgB, pkb, pib);
        const int kqa = (int)pka * kPatchK + r, iqa = (int)pia * kPatchI + c;
        const int kqb = (int)pkb * kPatchK + r, iqb = (int)pib * kPatchI + c;
        const bool va = kqa < nqkA && iqa < nqiA, vb = kqb < nqkB && iqb < nqiB;
        const uint32_t qa = (uint32_t)kqa * (uint32_t)NA + (uint32_t)iqa;
        const uint32_t qb = (uint32_t)kqb * (uint32_t)NB + (uint32_t)iqb;
        EBox<PREC> ba, bb;
        ba.set_empty();
        bb.set_empty();
        if (va) ba.load(fbA, qa);
        if (vb) bb.load(fbB, qb);
        __syncwarp();                          // the previous pair's quarter boxes are read
        if (lane < 8) sQuart[warp][lane] = xq;
        __syncwarp();
        // survivors: quads meeting some quarter of the other patch
        bool sa = false, sb = false;
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            sa |= boxes_overlap(ba, sQuart[warp][4 + k]);
            sb |= boxes_overlap(bb, sQuart[warp][k]);
        }
        sa &= va;
        sb &= vb;
        const uint32_t mA = __ballot_sync(FULL, sa), mB = __ballot_sync(FULL, sb);
        if (!mA || !mB) continue;
        const uint32_t nA = __popc(mA), nB = __popc(mB);
        __syncwarp();                          // the previous pair's survivors are read
        if (sa) {
            const int k = __popc(mA & lt);
            ba.store_halves(sLo[warp][0][k], sHi[warp][0][k]);
            sQ[warp][0][k] = qa;
        }
        if (sb) {
            const int k = __popc(mB & lt);
            bb.store_halves(sLo[warp][1][k], sHi[warp][1][k]);
            sQ[warp][1][k] = qb;
        }
        __syncwarp();
        tests += nA * nB;
        // the smaller side in registers: lane = (group g, member m), m < nR
        const int R = nB <= nA ? 1 : 0, I = 1 - R;
        const uint32_t nR = R ? nB : nA, nI = R ? nA : nB;
        // lane / nR and 32 / nR from FP32 reciprocals: (x + 1/2) / nR lies at
        // least 1/64 from an integer for x <= 32, far above the reciprocal's error
        const float rR = __fdividef(1.0f, (float)nR);
        const uint32_t g = (uint32_t)(((float)lane + 0.5f) * rR);
        const uint32_t G = (uint32_t)(32.5f * rR);
        const uint32_t m = (uint32_t)lane - g * nR;
        const bool member = g < G;
        const typename EBox<PREC>::Half rlo = sLo[warp][R][member ? m : 0], rhi = sHi[warp][R][member ? m : 0];
        const uint32_t rq = sQ[warp][R][member ? m : 0];
        for (uint32_t base = 0; base < nI; base += G) {
            const uint32_t ii = base + g;
            const bool act = member && ii < nI;
            bool ov = false;
            uint32_t iq = 0;
            if (act) {
                ov = EBox<PREC>::halves_overlap(sLo[warp][I][ii], sHi[warp][I][ii], rlo, rhi);
                iq = sQ[warp][I][ii];
                if (MOLLER && ov) {
                    const uint32_t fa = R ? iq : rq, fb = R ? rq : iq;
                    ov = !moller_reject(a.meshes[pr.x], fa, a.meshes[pr.y], fb, 1);
                }
            }
            Cand cd;
            cd.faceA = R ? iq : rq;
            cd.faceB = R ? rq : iq;
            cd.pair = pp.pair;
            cd.pad = 0;
            stage_push<kPatchFlush>(stage, staged, ov, cd, &a.ctr->cand, store);
        }
    }
    __syncwarp();
    stage_flush<kPatchFlush>(stage, staged, &a.ctr->cand, store);
    // every lane counted the same tests (warp-uniform): one lane adds them
    if (lane == 0 && tests) atomicAdd(&a.ctr->ptests, tests);
}

int g_patch_resident[2][2] = {};

template <int PREC, bool MOLLER>
int patch_resident() {
    int &res = g_patch_resident[PREC][MOLLER ? 1 : 0];
    if (res == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_patch_quads<PREC, MOLLER>, 32 * kPatchWarps,
                                                          0) != cudaSuccess || nb < 1)
            nb = 1;
        res = nb;
    }
    return res;
}

int g_quarter_resident[2] = {};

template <int PREC>
int quarter_resident() {
    int &res = g_quarter_resident[PREC];
    if (res == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_patch_quarters<PREC>, kQuarterBlock, 0) !=
                cudaSuccess || nb < 1)
            nb = 1;
        res = nb;
    }
    return res;
}

template <int PREC, bool MOLLER>
void patch_waves(const PatchArgs &a, int sms, cudaStream_t st) {
    k_patch_quarters<PREC><<<sms * quarter_resident<PREC>(), kQuarterBlock, 0, st>>>(a);
    k_patch_quads<PREC, MOLLER><<<sms * patch_resident<PREC, MOLLER>(), 32 * kPatchWarps, 0, st>>>(a);
}

}  // namespace

void configure_patch_quads() {
    quarter_resident<0>();
    quarter_resident<1>();
    patch_resident<0, false>();
    patch_resident<0, true>();
    patch_resident<1, false>();
    patch_resident<1, true>();
}

void launch_patch_quads(const PatchArgs &a, int precision, int sms, cudaStream_t st) {
    if (precision == 1) {
        if (a.moller) patch_waves<1, true>(a, sms, st);
        else patch_waves<1, false>(a, sms, st);
    } else {
        if (a.moller) patch_waves<0, true>(a, sms, st);
        else patch_waves<0, false>(a, sms, st);
    }
}

// Looks up the emission's resident blocks per SM once, outside stream capture
// (a failed lookup leaves one block per SM).
void configure_emit() {
    emit_resident<0, false>();
    emit_resident<0, true>();
    emit_resident<1, false>();
    emit_resident<1, true>();
}

void launch_emit(const EmitArgs &a, int precision, int face_level, int sms, cudaStream_t st) {
    if (precision == 1) {
        if (a.moller) emit_waves<1, true>(a, face_level, sms, st);
        else emit_waves<1, false>(a, face_level, sms, st);
    } else {
        if (a.moller) emit_waves<0, true>(a, face_level, sms, st);
        else emit_waves<0, false>(a, face_level, sms, st);
    }
}

}  // namespace tms

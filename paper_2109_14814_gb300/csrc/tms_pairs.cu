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
// quick test of Sec. 6.2.3; survivors are staged per warp and appended 32 at a
// time.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tms_common.cuh"

namespace tms {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kTile = 32;
constexpr int kEmitWarps = 8;
constexpr unsigned kCandFlush = 64;    // candidates per atomic on the candidate counter

// ---------------------------------------------------------------------------
// emission
// ---------------------------------------------------------------------------
// a face's box from its mesh's face-box array (written by the bounds pass)
template <int PREC>
struct EBox;
template <>
struct __align__(16) EBox<1> {
    float lo[4], hi[4];
    __device__ void load(const void *fbox, uint32_t face) {
        const float4 *p = reinterpret_cast<const float4 *>(fbox) + 2 * (size_t)face;
        const float4 l = __ldg(p), h = __ldg(p + 1);
        lo[0] = l.x; lo[1] = l.y; lo[2] = l.z; lo[3] = l.w;
        hi[0] = h.x; hi[1] = h.y; hi[2] = h.z; hi[3] = h.w;
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
    double lo[4], hi[4];
    __device__ void load(const void *fbox, uint32_t face) {
        const double2 *p = reinterpret_cast<const double2 *>(fbox) + 4 * (size_t)face;
        const double2 x0 = __ldg(p), x1 = __ldg(p + 1), x2 = __ldg(p + 2), x3 = __ldg(p + 3);
        lo[0] = x0.x; lo[1] = x0.y; lo[2] = x1.x; lo[3] = x1.y;
        hi[0] = x2.x; hi[1] = x2.y; hi[2] = x3.x; hi[3] = x3.y;
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
__global__ void __launch_bounds__(32 * kEmitWarps) k_emit(EmitArgs a, int face_level) {
    // the tile's B side, structure of arrays: the hot loop reads only the boxes
    __shared__ EBox<PREC> sBox[kEmitWarps][kTile];
    __shared__ uint32_t sMask[kEmitWarps][kTile];
    __shared__ uint32_t sFace[kEmitWarps][kTile];
    __shared__ Cand sOut[kEmitWarps][kCandFlush + 32];   // staged candidates
    // nothing to do after an entry overflow (the host retries with more room),
    // and a bounded amount of work in any case
    if (a.ctr->entries > a.ent_cap) return;
    if (a.ctr->pair_slots > kMaxPairSlots) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&a.ctr->status, ST_PAIR_LIMIT);
        return;
    }
    const unsigned long long total = a.ctr->tiles;
    const unsigned long long ncell = clamp_count(&a.ctr->cells, a.ent_cap);
    const unsigned long long nent = clamp_count(&a.ctr->grouped, a.ent_cap);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long gw = blockIdx.x * (unsigned long long)kEmitWarps + warp;
    const unsigned long long nw = (unsigned long long)gridDim.x * kEmitWarps;
    // each warp owns a contiguous range of tiles: one binary search for its first
    // tile's cell, then a forward walk over the cells
    const unsigned long long per = (total + nw - 1) / nw;
    const unsigned long long t_begin = gw * per;
    const unsigned long long t_end = min(t_begin + per, total);
    Cand *stage = sOut[warp];
    unsigned staged = 0;
    const unsigned long long cap = a.cand_cap;
    Cand *cand_out = a.cand;
    auto store = [cand_out, cap](unsigned long long pos, const Cand &cd) {
        if (pos < cap) cand_out[pos] = cd;
    };
    unsigned long long c = 0;
    if (t_begin < t_end) {
        unsigned long long lo = 0, hi = ncell - 1;
        while (lo < hi) {
            unsigned long long mid = (lo + hi + 1) >> 1;
            if (a.cells[mid].tile_off <= t_begin) lo = mid; else hi = mid - 1;
        }
        c = lo;
    }
    // the lanes' face, kept across tiles of one A row
    EBox<PREC> abox;
    uint32_t amask = 0, aface = 0;
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
        const bool hasA = lane < nAt;
        if (hasA && !reuse) {
            aface = a.vals[l0 + lane];
            abox.load(fbL, aface);
            amask = own_mask(abox.low_cell(gr), cur);
        }
        if (lane < nBt) {
            const uint32_t bface = a.vals[m0 + lane];
            EBox<PREC> bb;
            bb.load(fbM, bface);
            sBox[warp][lane] = bb;
            sMask[warp][lane] = own_mask(bb.low_cell(gr), cur);
            sFace[warp][lane] = bface;
        }
        __syncwarp();
        // the append of the pairs with box j that survive (and, optionally, Moller)
        auto emit_j = [&](int j, bool keep) {
            const uint32_t bface = sFace[warp][j];
            if (MOLLER && keep) {
                const uint32_t fa = swapAB ? bface : aface, fb = swapAB ? aface : bface;
                keep = !moller_reject(a.meshes[pr.x], fa, a.meshes[pr.y], fb, face_level);
            }
            Cand cd;
            cd.faceA = swapAB ? bface : aface;
            cd.faceB = swapAB ? aface : bface;
            cd.pair = pair;
            cd.pad = 0;
            stage_push<kCandFlush>(stage, staged, keep, cd, &a.ctr->cand, store);
        };
        // owner cell: the componentwise max of the two faces' lowest cells is this
        // cell iff every coordinate is owned by one of them (masks OR to 0xF);
        // two B boxes per step, one vote, the append only when a lane keeps a pair
        int j = 0;
        for (; j + 1 < nBt; j += 2) {
            const EBox<PREC> b0x = sBox[warp][j], b1x = sBox[warp][j + 1];
            const bool k0 = hasA & ((amask | sMask[warp][j]) == 0xFu) & boxes_overlap(abox, b0x);
            const bool k1 = hasA & ((amask | sMask[warp][j + 1]) == 0xFu) & boxes_overlap(abox, b1x);
            if (__ballot_sync(FULL, k0 | k1) == 0u) continue;
            emit_j(j, k0);
            emit_j(j + 1, k1);
        }
        if (j < nBt) {
            const bool k0 = hasA & ((amask | sMask[warp][j]) == 0xFu) & boxes_overlap(abox, sBox[warp][j]);
            if (__ballot_sync(FULL, k0) != 0u) emit_j(j, k0);
        }
        __syncwarp();
    }
    __syncwarp();
    stage_flush<kCandFlush>(stage, staged, &a.ctr->cand, store);
}

}  // namespace

void launch_emit(const EmitArgs &a, int precision, int face_level, int grid, cudaStream_t st) {
    const dim3 b(32 * kEmitWarps);
    if (precision == 1) {
        if (a.moller) k_emit<1, true><<<grid, b, 0, st>>>(a, face_level);
        else k_emit<1, false><<<grid, b, 0, st>>>(a, face_level);
    } else {
        if (a.moller) k_emit<0, true><<<grid, b, 0, st>>>(a, face_level);
        else k_emit<0, false><<<grid, b, 0, st>>>(a, face_level);
    }
}

}  // namespace tms

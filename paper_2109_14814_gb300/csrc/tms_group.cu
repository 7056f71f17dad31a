// Grouping of the broad phase's face-cell entries by grid cell.
//
// The paper's GPU broad phase keeps, per grid box, the list of quads of each
// mesh that touch it, and proposes every (A quad, B quad) pair of a box
// (Sec. 6.2.1, Sec. 6.3 and Algorithm 1, whose box_gid_idxs array is the
// exclusive scan of nA * nB over the boxes).  Re-designed for GB300 without a
// sort: the entries need only be grouped by (pair, cell), with mesh A's faces
// first, so
//   k_group_count    finds or claims each entry's (pair, cell) key in an
//                    open-addressing table (linear probing), and one atomic per
//                    group of equal keys in a warp gives every entry its rank
//                    within (cell, role) and the cell its A and B counts;
//   k_cells_*        scan the whole table (three launches: per-block sums, one
//                    block over the sums, per-slot offsets): cells holding
//                    faces of both meshes get consecutive indices, their
//                    entries' start, their first B entry and their 32 x 32 tile
//                    offset; the totals go to the counters; every slot read is
//                    returned to the free state;
//   k_group_scatter  writes every entry's face id to its cell's A or B list.
// The order of a cell's entries is left to the atomics; the search's output
// does not depend on it.  The table is sized from the entry capacity (an
// sixteenth of it, so that it stays in L2 and a scan of all of it is cheap); a
// search that finds it over half full, or full, is run again with a table four
// times larger.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tms_common.cuh"

namespace tms {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kGroupBlock = 256;
constexpr int kCellScanBlock = 512;
constexpr int kTileEdge = 32;

// the table slot of stored key k (never kHashEmpty), claimed if new
__device__ __forceinline__ uint32_t table_slot(const GroupArgs &a, unsigned long long k) {
    const unsigned long long mask = a.tsize - 1;
    unsigned long long h = mix64(k) & mask;
    for (unsigned long long probe = 0; probe < a.tsize; ++probe) {
        unsigned long long cur = __ldcg(a.tkey + h);
        if (cur == k) return (uint32_t)h;
        if (cur == kHashEmpty) {
            cur = atomicCAS(a.tkey + h, kHashEmpty, k);
            if (cur == kHashEmpty || cur == k) return (uint32_t)h;
        }
        h = (h + 1) & mask;
    }
    // every slot taken: the host grows the table and runs the search again
    atomicOr(&a.ctr->status, ST_TABLE_FULL);
    return 0;
}

__global__ void __launch_bounds__(kGroupBlock) k_group_count(GroupArgs a) {
    if (a.ctr->entries > a.cap) return;   // the host retries with more room
    const unsigned long long n = a.ctr->entries;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x - lane;
         i0 < n; i0 += stride) {
        const unsigned long long i = i0 + lane;
        const bool ok = i < n;
        const uint64_t key = ok ? a.ent_key[i] : ~0ULL;
        // lanes with the same (pair, cell, role) share one table lookup and one atomic
        const uint32_t peers = __match_any_sync(FULL, key);
        const int leader = __ffs(peers) - 1;
        uint32_t slot = 0, base = 0;
        if (ok && lane == leader) {
            slot = table_slot(a, (key >> 1) + 1);
            uint32_t *cnt = (key & 1) ? &a.tcnt[slot].y : &a.tcnt[slot].x;
            base = atomicAdd(cnt, (uint32_t)__popc(peers));
        }
        slot = __shfl_sync(FULL, slot, leader);
        base = __shfl_sync(FULL, base, leader);
        if (ok) {
            // the role rides in the slot's top bit (slots are below 2^31)
            a.ent_slot[i] = slot | ((uint32_t)(key & 1) << 31);
            a.ent_rank[i] = base + __popc(peers & lt);
        }
    }
}

struct CellVals {
    unsigned long long both, size, tiles, pairs, claimed;
};

__device__ __forceinline__ CellVals cell_vals(const GroupArgs &a, unsigned long long slot) {
    const uint2 c = a.tcnt[slot];
    CellVals v;
    v.claimed = (c.x | c.y) ? 1 : 0;
    const bool both = c.x > 0 && c.y > 0;
    v.both = both ? 1 : 0;
    v.size = both ? (unsigned long long)c.x + c.y : 0;
    v.tiles = both ? (unsigned long long)((c.x + kTileEdge - 1) / kTileEdge) * ((c.y + kTileEdge - 1) / kTileEdge) : 0;
    v.pairs = both ? (unsigned long long)c.x * c.y : 0;
    return v;
}

__device__ __forceinline__ void slot_chunk(unsigned long long n, unsigned long long &b,
                                          unsigned long long &e) {
    unsigned long long per = (n + gridDim.x - 1) / gridDim.x;
    per = (per + 31) & ~31ULL;
    b = per * blockIdx.x;
    e = b + per;
    if (b > n) b = n;
    if (e > n) e = n;
}

__global__ void __launch_bounds__(kCellScanBlock) k_cells_reduce(GroupArgs a) {
    __shared__ unsigned long long red[5][kCellScanBlock / 32];
    if (a.ctr->entries > a.cap) return;
    unsigned long long b, e;
    slot_chunk(a.tsize, b, e);
    unsigned long long s[5] = {0, 0, 0, 0, 0};
    for (unsigned long long j = b + threadIdx.x; j < e; j += blockDim.x) {
        const CellVals v = cell_vals(a, j);
        s[0] += v.both; s[1] += v.size; s[2] += v.tiles; s[3] += v.pairs; s[4] += v.claimed;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        for (int off = 16; off > 0; off >>= 1) s[k] += __shfl_xor_sync(FULL, s[k], off);
        if (lane == 0) red[k][warp] = s[k];
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
        a.partials[threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

// exclusive scan of the per-block sums (one block of 1024 threads, g <= 1024):
// the five quantities at once, each by a warp scan and a scan of the 32 warp sums
__global__ void __launch_bounds__(1024) k_cells_partials(GroupArgs a, int g) {
    __shared__ unsigned long long wsum[5][32];
    if (a.ctr->entries > a.cap) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned long long x[5], incl[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        x[k] = t < g ? a.partials[k * g + t] : 0;
        incl[k] = x[k];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL, incl[k], off);
            if (lane >= off) incl[k] += y;
        }
        if (lane == 31) wsum[k][warp] = incl[k];
    }
    __syncthreads();
    if (warp < 5) {
        const unsigned long long w = wsum[warp][lane];
        unsigned long long wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL, wi, off);
            if (lane >= off) wi += y;
        }
        wsum[warp][lane] = wi - w;
        if (lane == 31) {
            // totals: the counters the emission and the host read
            if (warp == 0) a.ctr->cells = wi;
            else if (warp == 1) a.ctr->grouped = wi;
            else if (warp == 2) a.ctr->tiles = wi;
            else if (warp == 3) a.ctr->pair_slots = wi;
            else a.ctr->claimed = wi;   // the host grows a crowded table
        }
    }
    __syncthreads();
    if (t < g) {
#pragma unroll
        for (int k = 0; k < 5; ++k) a.partials[k * g + t] = wsum[k][warp] + incl[k] - x[k];
    }
}

__global__ void __launch_bounds__(kCellScanBlock) k_cells_down(GroupArgs a) {
    __shared__ unsigned long long wsum[3][kCellScanBlock / 32];
    __shared__ unsigned long long carry[3];
    if (a.ctr->entries > a.cap) return;
    unsigned long long b, e;
    slot_chunk(a.tsize, b, e);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 3) carry[threadIdx.x] = a.partials[threadIdx.x * gridDim.x + blockIdx.x];
    __syncthreads();
    for (unsigned long long base = b; base < e; base += blockDim.x) {
        const unsigned long long j = base + threadIdx.x;
        const unsigned long long slot = j;
        CellVals v = {0, 0, 0, 0, 0};
        if (j < e) v = cell_vals(a, slot);
        unsigned long long x[3] = {v.both, v.size, v.tiles}, incl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            incl[k] = x[k];
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned long long y = __shfl_up_sync(FULL, incl[k], off);
                if (lane >= off) incl[k] += y;
            }
            if (lane == 31) wsum[k][warp] = incl[k];
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const unsigned long long w = lane < (int)(blockDim.x >> 5) ? wsum[k][lane] : 0;
                unsigned long long wi = w;
                for (int off = 1; off < 32; off <<= 1) {
                    const unsigned long long y = __shfl_up_sync(FULL, wi, off);
                    if (lane >= off) wi += y;
                }
                if (lane < (int)(blockDim.x >> 5)) wsum[k][lane] = wi - w;
            }
        }
        __syncthreads();
        unsigned long long ex[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) ex[k] = carry[k] + wsum[k][warp] + incl[k] - x[k];
        if (j < e && v.claimed) {
            if (v.both) {
                const unsigned long long c = ex[0];
                const uint2 cnt = a.tcnt[slot];
                const unsigned long long key = a.tkey[slot] - 1;
                CellRec rec;
                rec.pair = (uint32_t)(key >> 31);
                // the cell's coordinates (the emission's owner test needs them per tile)
                const Grid &g = a.grids[rec.pair];
                uint32_t cell = (uint32_t)(key & 0x7FFFFFFFu), cc[4];
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    cc[d] = cell % (uint32_t)g.n[d];
                    cell /= (uint32_t)g.n[d];
                }
                rec.xy = make_uint2(cc[0] | (cc[1] << 16), cc[2] | (cc[3] << 16));
                rec.start = (uint32_t)ex[1];
                rec.bstart = (uint32_t)ex[1] + cnt.x;
                rec.tile_off = ex[2];
                rec.pad = 0;
                a.cells[c] = rec;
                // the scatter's one gather: both list starts of the slot
                a.tstart[slot] = make_uint2((uint32_t)ex[1], (uint32_t)ex[1] + cnt.x);
            } else {
                a.tstart[slot] = make_uint2(kNoCell, kNoCell);
            }
            // the slot is free again for the next search (the scatter reads tstart only)
            a.tkey[slot] = kHashEmpty;
            a.tcnt[slot] = make_uint2(0u, 0u);
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
#pragma unroll
            for (int k = 0; k < 3; ++k) carry[k] = ex[k] + x[k];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kGroupBlock) k_group_scatter(GroupArgs a) {
    if (a.ctr->entries > a.cap) return;
    const unsigned long long n = a.ctr->entries;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += stride) {
        const uint32_t sr = a.ent_slot[i];
        const uint2 st = a.tstart[sr & 0x7FFFFFFFu];
        if (st.x == kNoCell) continue;
        const uint32_t start = (sr >> 31) ? st.y : st.x;
        const unsigned long long pos = (unsigned long long)start + a.ent_rank[i];
        if (pos < a.cap) a.grouped[pos] = a.ent_face[i];
    }
}

}  // namespace

// one lane per entry slot: no warp walks a chain of dependent table lookups
static int entry_grid(const GroupArgs &a) {
    const unsigned long long b = (a.cap + kGroupBlock - 1) / kGroupBlock;
    return (int)(b < 1 ? 1 : (b > (1ULL << 30) ? (1ULL << 30) : b));
}

void launch_group_count(const GroupArgs &a, int grid, cudaStream_t st) {
    (void)grid;
    k_group_count<<<entry_grid(a), kGroupBlock, 0, st>>>(a);
}

void launch_group_cells(const GroupArgs &a, int grid, cudaStream_t st) {
    const int g = grid < 1024 ? grid : 1024;
    k_cells_reduce<<<g, kCellScanBlock, 0, st>>>(a);
    k_cells_partials<<<1, 1024, 0, st>>>(a, g);
    k_cells_down<<<g, kCellScanBlock, 0, st>>>(a);
    k_group_scatter<<<entry_grid(a), kGroupBlock, 0, st>>>(a);
}

}  // namespace tms

// Internal device structures and helpers of the GB300 mesh-intersection search.
// Not part of the public ABI (include/tms.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/tms.h"

namespace tms {

// ---------------------------------------------------------------------------
// tunables
// ---------------------------------------------------------------------------
constexpr int kRadixBits = 9;            // five passes for the 44-bit hit keys of 4M-triangle meshes
constexpr int kRadixBins = 1 << kRadixBits;
constexpr int kSortBlock = 512;          // threads per radix block (16 warps, one per digit)
constexpr int kSortItems = 4;            // keys per thread per tile
constexpr int kSortTile = kSortBlock * kSortItems;
constexpr int kScanBlock = 512;
constexpr int kCellBits = 31;            // a pair's grid has < 2^31 cells
constexpr int kMaxCellsPerDim = 65535;
constexpr unsigned long long kMaxPairSlots = 1ULL << 36;  // bound on proposed pairs per call

// Face-pass modes
enum FaceMode : int {
    MODE_BOUNDS = 0,      // per-mesh world bounds, widest face extent, finiteness
    MODE_MARK = 1,        // set occupancy bits of mesh-A cells
    MODE_PROBE_MARK = 2,  // mesh B: emit entries in A-occupied cells, mark them hot
    MODE_PROBE = 3,       // mesh A: emit entries in hot cells
    MODE_EMIT_ALL = 4     // emit every face-cell incidence (no occupancy filter)
};

// status bits written by kernels into Counters::status
enum StatusBits : unsigned int {
    ST_NONFINITE = 1u << 0,
    ST_TIMEOUT = 1u << 1,
    ST_PAIR_LIMIT = 1u << 2,
    ST_TABLE_FULL = 1u << 3,
};

// ---------------------------------------------------------------------------
// device-side descriptors
// ---------------------------------------------------------------------------
struct MeshDev {
    const double *c[4];   // x, y, px, py, offset to the first view column
    const double *s;      // s values of the view (M entries), device
    float4 *split;        // plan scratch: the FP32 split of every view vertex
                          // (k*N + i): hi = RN32(x) at [k*N + i], lo = RN32(x - hi)
                          // at [N*M + k*N + i] (hi and lo in separate halves, so a
                          // gather of the hi parts alone reads dense 16-byte rows),
                          // written by the bounds pass, gathered by the narrow filters
    void *fbox;           // plan scratch: per face slot its box, written by the
                          // bounds pass (mixed precision: float4 lo, float4 hi,
                          // rounded outward; plain: 8 doubles lo[4], hi[4]);
                          // slot = face id (quad k*N + i, or triangle 2(k*N + i) + t)
    int N;                // theta samples
    int M;                // vertex rows in the view
    int periodic;
    int nqi;              // quads per row (N or N-1)
    int nqk;              // quad rows (M-1)
    int pad;
    void *pbox;           // plan scratch (patch level): per patch of kPatchI x
                          // kPatchK quads the union of their boxes, in the
                          // format of fbox, written by the bounds pass; slot =
                          // patch row * npi + patch column
    void *qbox;           // plan scratch (patch level): per patch its four
                          // quarter boxes -- quad rows (0-1, 2-3) x columns
                          // (0-3, 4-7), slot 4 p + 2 row half + column half;
                          // a quarter without quads holds an empty box
    int npi;              // patches per quad row, ceil(nqi / kPatchI) (0: none)
    int npk;              // patch rows, ceil(nqk / kPatchK)
    unsigned long long pmagic;  // ceil(2^64 / npi) for npi >= 2: a patch id's row
                                // is __umul64hi(id, pmagic) (exact for 32-bit ids)
    unsigned long long nmagic;  // ceil(2^64 / N): a quad id's row is
                                // __umul64hi(q, nmagic) (N >= 2, exact for 32-bit ids)
    float4 *pframe;       // plan scratch (patch level, mixed precision, FP32
                          // filters on): per patch its frame, kFrameF4 float4
                          // at slot * kFrameF4 (layout at kFrameF4); else NULL
};

// (i, k) of quad q = k N + i, by the reciprocal of N (no integer division)
__host__ __device__ inline unsigned long long recip64(unsigned long long d) {
    return d >= 2 ? ~0ULL / d + 1 : 0;
}

// Patch level of the broad phase: quads grouped into patches of kPatchI quads
// along theta by kPatchK quad rows -- 32 quads, one per lane of a warp.
constexpr int kPatchI = 8;
constexpr int kPatchK = 4;

// A patch frame, written by the bounds pass and read by the patch-pair test:
// an FP32 point c, four FP32 axes e_0..e_3 (e_0, e_1 along the patch's two
// parameter directions, e_2, e_3 completing them) and bounds rigorous for the
// patch's FP64 vertices V:
//   h_k >= max_V |e_k . (V - c)|,
//   rho >= max_V max_i |r_i| + 4.0001 u max|e| sum_k h_k,
//   r = (V - c) - sum_k (e_k . (V - c)) e_k
// (r is what the frame does not reproduce: rounding-small when the axes are
// orthonormal, and no such assumption is made), L >= max |V_i|, and n_k >=
// |e_k|_1 for the two completing axes.  For any direction w then
//   |w . (V - c)| <= sum_k |w . e_k| h_k + |w|_1 rho
// with w . e_k rounded in FP32 (the second term of rho covers that rounding),
// and |e_k . (V - c)| <= h_k.  Layout: c, e_0, e_1, e_2, e_3, (h_0..h_3),
// (rho, L, n_2, n_3).
constexpr int kFrameF4 = 7;

struct PassEntry {        // one mesh processed by a face pass
    int mesh;             // index into the mesh table
    int pair;             // mesh-pair index
    int role;             // 0 = mesh A, 1 = mesh B of the pair
    int tiles_i;          // tiles along theta (bounds pass)
    long long tile_base;  // first global tile of this mesh (bounds pass)
    long long face_base;  // first global face slot of this mesh (cell passes),
                          // a multiple of 32 so that no warp spans two meshes
    long long faces;      // face slots of this mesh
};

// face slots of a mesh view: quads k*N + i (i < N, k < nqk; slot i = N-1 of an
// open mesh is unused), or two triangles per quad
__host__ __device__ inline unsigned long long face_slots(const MeshDev &m, int face_level) {
    return (face_level == 0 ? 2ULL : 1ULL) * (unsigned long long)m.N * (unsigned long long)m.nqk;
}

struct Bounds {           // per mesh, order-preserving uint64 encodings of doubles
    unsigned long long lo[4];
    unsigned long long hi[4];
    unsigned long long w[4];
    unsigned int flags;
    unsigned int faces;   // nonzero once any face was seen
};

struct Grid {             // per pair: trimmed world and uniform grid
    double o64[4], e64[4], inv64[4];
    float o32[4], e32[4], inv32[4];
    int n[4];
    int empty;
    int pad[3];
};

struct Counters {
    unsigned long long entries;
    unsigned long long cells;      // cells holding faces of both meshes
    unsigned long long grouped;    // entries of those cells
    unsigned long long pair_slots;
    unsigned long long tiles;
    unsigned long long cand;
    unsigned long long fp64;
    unsigned long long fp32;       // triangle pairs through the verified FP32 solve
    unsigned long long sat;        // triangle pairs through the separating-axis prefilter
    unsigned long long quad;       // quad candidates through the quad-level prefilter
    unsigned long long qkeep;      // quad candidates it could not clear
    unsigned long long claimed;    // cell-table slots claimed by this search
    unsigned long long ppairs;     // patch pairs with overlapping boxes (patch level)
    unsigned long long ptests;     // quad-pair box tests inside those patch pairs
    unsigned long long psurv;      // patch pairs with an overlapping quarter pair
    unsigned long long raw_hits;
    unsigned long long out;
    unsigned int status;
    unsigned int pad;
};

constexpr unsigned long long kHashEmpty = 0;   // free slot of the cell table (keys are stored + 1)
constexpr uint32_t kNoCell = 0xFFFFFFFFu;

struct Cand {             // candidate face pair
    uint32_t faceA, faceB, pair, pad;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline unsigned long long ord_enc(double v) {
#ifdef __CUDA_ARCH__
    long long b = __double_as_longlong(v);
#else
    long long b;
    memcpy(&b, &v, 8);
#endif
    return (b >= 0) ? ((unsigned long long)b | 0x8000000000000000ULL) : ~(unsigned long long)b;
}

__host__ __device__ inline double ord_dec(unsigned long long u) {
    long long b = (u & 0x8000000000000000ULL) ? (long long)(u & 0x7FFFFFFFFFFFFFFFULL)
                                              : (long long)(~u);
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double v;
    memcpy(&v, &b, 8);
    return v;
#endif
}

// How far apart two triangles can be and still make an FP64 hit.  The FP64
// solve (Gaussian elimination with partial pivoting, reciprocal pivots, on the
// 4 x 4 system of Eq. (precise)) returns z with (A + E) z = r + e, where
// |E_ij| <= gamma_30 (|L||U|)_ij + u64 |A_ij| <= 1.1e-13 max|A| (multipliers <= 1,
// growth <= 2^3, the rounding of A's entries from the vertices included) and
// |e| <= u64 |r|.  A hit has weights >= -tau' (tau' = tau plus the rounding of the
// margin, 1e-15 at most), so |z| <= 1 + 2 tau' and the points x2 + a e1 + b e2
// and y2 + c f1 + d f2 of the two triangles, widened to weights >= -tau', differ
// by A z - r = e - E z: |E z| <= 1.1e-13 max|A| sum_j |z_j| <= 4.4e-13 (1 + 2 tau')
// max|A| and |e| <= 1.12e-16 |r|, at most fp64_reach(max|A|, |r|, tau) in every
// coordinate.  A separating-axis test that proves the widened triangles further
// apart than that therefore proves that the FP64 solve reports no hit --
// whatever the system's condition.
__device__ __forceinline__ float fp64_reach(float amax, float rmax, float tau) {
    return (5e-13f * (1.0f + 2.0f * tau) * amax + 1.2e-16f * rmax) * 1.01f + 1e-37f;
}

// along w, a triangle's projection widened to weights >= -tau' grows by at most
// 3 tau' times its length on each side; tp = 3 tau' from tau (FP32, rounded up)
__device__ __forceinline__ float widen3(float tau) { return 3.0f * tau * 1.001f + 3e-15f; }

// 64-bit mixer (MurmurHash3 finaliser) for hashing (pair, cell) into a bitmap.
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

// Two bits inside one 32-bit word: word index from the top bits, bit positions
// from the low bits (a blocked Bloom filter with k = 2).
__device__ __forceinline__ void bloom_slot(uint64_t h, int word_bits, uint32_t &word,
                                           uint32_t &mask) {
    word = (uint32_t)(h >> (64 - word_bits));
    mask = (1u << (h & 31)) | (1u << ((h >> 5) & 31));
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long clamp_count(const unsigned long long *p,
                                                          unsigned long long cap) {
    unsigned long long n = *p;
    return n < cap ? n : cap;
}

// Warp-aggregated append: every lane of `mask` calls this; lanes with pred
// receive a unique slot.  One atomic per warp.
__device__ __forceinline__ unsigned long long warp_append(unsigned long long *counter, bool pred,
                                                          unsigned int mask) {
    unsigned int want = __ballot_sync(mask, pred);
    unsigned long long base = 0;
    if (want) {
        int leader = __ffs(want) - 1;
        int lane = threadIdx.x & 31;
        if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(want));
        base = __shfl_sync(mask, base, leader);
    }
    return base + __popc(want & lanemask_lt());
}

// Warp-staged append for high-volume outputs: lanes with pred place one record
// each in the warp's shared-memory stage (FLUSH + 32 records); every FLUSH
// records go out with one atomic on the global counter and coalesced stores,
// so the counter sees one atomic per FLUSH records (a single global counter
// serialises its atomics).  All 32 lanes call it together with the same n;
// store(pos, rec) writes record rec at global position pos (the caller checks
// pos against its capacity).
// the records left in the stage (fewer than FLUSH) at the end of a kernel
template <unsigned FLUSH, typename Rec, typename Store>
__device__ __forceinline__ void stage_flush(Rec *stage, unsigned cnt, unsigned long long *counter,
                                            const Store &store) {
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0 && cnt) base = atomicAdd(counter, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
    for (unsigned k = 0; k < FLUSH; k += 32)
        if (k + lane < cnt) store(base + k + lane, stage[k + lane]);
    __syncwarp();
}

template <unsigned FLUSH, typename Rec, typename Store>
__device__ __forceinline__ void stage_push(Rec *stage, unsigned &n, bool pred, const Rec &rec,
                                           unsigned long long *counter, const Store &store) {
    static_assert(FLUSH % 32 == 0, "flush whole warps");
    const unsigned want = __ballot_sync(0xffffffffu, pred);
    if (!want) return;
    const int lane = threadIdx.x & 31;
    if (pred) stage[n + __popc(want & lanemask_lt())] = rec;
    n += __popc(want);
    if (n >= FLUSH) {
        __syncwarp();
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(counter, (unsigned long long)FLUSH);
        base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
        for (unsigned k = 0; k < FLUSH; k += 32) store(base + k + lane, stage[k + lane]);
        __syncwarp();
        // move the remainder (fewer than 32) to the front
        const unsigned rem = n - FLUSH;
        Rec r;
        if ((unsigned)lane < rem) r = stage[FLUSH + lane];
        __syncwarp();
        if ((unsigned)lane < rem) stage[lane] = r;
        __syncwarp();
        n = rem;
    }
}

// FP64 -> FP32 conversions from the IEEE-754 encodings, with integer operations
// only (the FP64 pipe, which also carries FP64 conversions, is scarce on GB300).
// Normal-range results equal round-down / round-up / round-to-nearest-even of
// the value.  Outside the FP32 normal range the results are still valid bounds:
// |x| < 2^-126 rounds outward to 0 or +-2^-126 (nearest: to +-0), |x| >= 2^128
// to +-FLT_MAX or +-inf, NaN stays NaN.
__device__ __forceinline__ unsigned f32_bits_trunc(unsigned long long b, int e32) {
    return ((unsigned)(b >> 63) << 31) | ((unsigned)e32 << 23) |
           (unsigned)((b & 0xFFFFFFFFFFFFFULL) >> 29);
}
__device__ __forceinline__ float f32_special(unsigned long long b, int e32, int dir) {
    // dir: -1 down, +1 up, 0 nearest
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const bool is_nan = ((b >> 52) & 0x7ff) == 0x7ff && (b & 0xFFFFFFFFFFFFFULL) != 0;
    if (is_nan) return __uint_as_float(0x7fc00000u);
    if (e32 >= 255) {                       // |x| >= 2^128 or inf
        const bool neg = sign != 0;
        if (dir == 0) return __uint_as_float(sign | 0x7f800000u);
        if (dir < 0) return __uint_as_float(neg ? 0xff800000u : 0x7f7fffffu);
        return __uint_as_float(neg ? 0xff7fffffu : 0x7f800000u);
    }
    // |x| < 2^-126
    const bool nonzero = (b & 0x7FFFFFFFFFFFFFFFULL) != 0;
    if (dir == 0 || !nonzero) return __uint_as_float(sign);
    const bool neg = sign != 0;
    if (dir < 0) return neg ? -1.17549435e-38f : 0.0f;
    return neg ? -0.0f : 1.17549435e-38f;
}
__device__ __forceinline__ float f32_rd(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e32 = (int)((b >> 52) & 0x7ff) - 896;
    if (e32 <= 0 || e32 >= 255) return f32_special(b, e32, -1);
    unsigned f = f32_bits_trunc(b, e32);
    f += (unsigned)(b >> 63) & (unsigned)((b & 0x1FFFFFFFULL) != 0);   // negative, inexact
    return __uint_as_float(f);
}
__device__ __forceinline__ float f32_ru(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e32 = (int)((b >> 52) & 0x7ff) - 896;
    if (e32 <= 0 || e32 >= 255) return f32_special(b, e32, +1);
    unsigned f = f32_bits_trunc(b, e32);
    f += ((unsigned)(b >> 63) ^ 1u) & (unsigned)((b & 0x1FFFFFFFULL) != 0);  // positive, inexact
    return __uint_as_float(f);
}
__device__ __forceinline__ float f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e32 = (int)((b >> 52) & 0x7ff) - 896;
    if (e32 <= 0 || e32 >= 255) return f32_special(b, e32, 0);
    unsigned f = f32_bits_trunc(b, e32) & 0x7fffffffu;
    const unsigned rem = (unsigned)(b & 0x1FFFFFFFULL);
    f += (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & (f & 1u));
    return __uint_as_float(f | ((unsigned)(b >> 63) << 31));
}
// finiteness from the exponent bits (no FP64 compare)
__device__ __forceinline__ bool finite64(double x) {
    return (((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// cell index along one coordinate: monotone non-decreasing in v, clamped
__device__ __forceinline__ int cell_of(float v, float o, float inv, int n) {
    float t = (v - o) * inv;
    t = fminf(fmaxf(t, 0.0f), (float)(n - 1));
    return (int)t;
}
__device__ __forceinline__ int cell_of(double v, double o, double inv, int n) {
    double t = (v - o) * inv;
    t = fmin(fmax(t, 0.0), (double)(n - 1));
    return (int)t;
}

// Triangle vertex grid indices, Sec. 6.2.4 orderings.
// T1 (tau 0): x1 = (i+1, k), x2 = (i, k), x3 = (i, k+1)
// T2 (tau 1): x1 = (i, k+1), x2 = (i+1, k+1), x3 = (i+1, k)
__device__ __forceinline__ void tri_ij(const MeshDev &m, uint32_t t, int ii[3], int kk[3]) {
    uint32_t q = t >> 1;
    int tau = t & 1;
    const uint32_t kq = (uint32_t)__umul64hi((unsigned long long)q, m.nmagic);   // q / N
    int i = (int)(q - kq * (uint32_t)m.N), k = (int)kq;
    int ip = (i + 1 == m.N) ? 0 : i + 1;
    if (tau == 0) {
        ii[0] = ip; kk[0] = k;
        ii[1] = i;  kk[1] = k;
        ii[2] = i;  kk[2] = k + 1;
    } else {
        ii[0] = i;  kk[0] = k + 1;
        ii[1] = ip; kk[1] = k + 1;
        ii[2] = ip; kk[2] = k;
    }
}

__device__ __forceinline__ void load_vertex(const MeshDev &m, int i, int k, double v[4]) {
    size_t off = (size_t)k * m.N + i;
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = __ldg(m.c[c] + off);
}

// ---------------------------------------------------------------------------
// launch helpers implemented in the .cu files
// ---------------------------------------------------------------------------
struct FacePassArgs {
    const PassEntry *entries;
    int n_entries;
    long long total_tiles;         // bounds pass: tiles of all entries
    long long total_faces;         // cell passes: face slots of all entries (padded)
    const MeshDev *meshes;
    int mode;
    int tile_rows;
    Bounds *bounds;                // indexed by mesh
    const Grid *grids;             // indexed by pair
    uint32_t *bmA;
    int bmA_word_bits;
    uint32_t *bmH;
    int bmH_word_bits;
    uint64_t *ent_key;             // pair << 32 | cell << 1 | role
    uint32_t *ent_val;             // face id
    Counters *ctr;
    unsigned long long ent_cap;
    int patch;                     // bounds pass: also the patch boxes, and the
                                   // widest patch (not face) extent for the grid
    int frames;                    // bounds pass, patch level, mixed precision:
                                   // also the patch frames (MeshDev::pframe)
};

void launch_face_pass(const FacePassArgs &a, int precision, int face_level, int block,
                      cudaStream_t st);
cudaError_t configure_face_pass();
// counters zeroed, bounds reset, bitmaps cleared (NULL: not cleared); word
// counts are multiples of four
void launch_search_init(Bounds *b, int n, Counters *ctr, uint32_t *bmA, unsigned long long n32a,
                        uint32_t *bmH, unsigned long long n32h, int grid, cudaStream_t st);
// cm_pair: per-pair cell multipliers (device, n_pairs), or NULL for cell_mult
void launch_grid_params(const Bounds *b, const int2 *pairs, int n_pairs, Grid *g,
                        float cell_mult, cudaStream_t st, const float *cm_pair = nullptr);

// polls of one device-side wait when tms_params.spin_limit is 0
constexpr unsigned long long kDefaultSpinLimit = 1ULL << 22;

// radix sort of (u64 key, u32 value) with a device-side count (at most cap);
// scratch holds radix_scratch_size(cap, key_bits) bytes; returns true when the
// sorted data ends in the alternate buffers.  A look-back wait gives up after
// spin_limit polls (0: kDefaultSpinLimit) and sets ST_TIMEOUT in *status;
// unpublished != 0 (a test switch) makes every wait run out.
bool radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                void *scratch, const unsigned long long *d_n, unsigned long long cap,
                int key_bits, int grid, unsigned int *status, unsigned long long spin_limit,
                int unpublished, cudaStream_t st);
size_t radix_scratch_size(unsigned long long cap, int key_bits);

// exclusive scans with a device-side count; total written to *d_total
void scan_u32(const uint32_t *in, uint32_t *out, const unsigned long long *d_n,
              unsigned long long cap, unsigned long long *partials, unsigned long long *d_total,
              int grid, cudaStream_t st);
void scan_u64(const unsigned long long *in, unsigned long long *out,
              const unsigned long long *d_n, unsigned long long cap,
              unsigned long long *partials, unsigned long long *d_total, int grid,
              cudaStream_t st);

// One cell holding faces of both meshes, as the emission reads it (32 bytes).
struct CellRec {
    uint32_t start;                // first A entry in `grouped`
    uint32_t bstart;               // first B entry
    unsigned long long tile_off;   // exclusive scan of the 32 x 32 tiles of nA x nB
    uint2 xy;                      // the cell's coordinates, 4 x u16
    uint32_t pair;
    uint32_t pad;
};

// Grouping of the face-cell entries by (pair, cell), mesh A's faces first:
// an open-addressing table of the (pair, cell) keys counts each cell's A and B
// entries and ranks every entry within its (cell, role); the cells holding
// faces of both meshes are compacted, and the face ids are scattered into one
// array, cell by cell (the paper's per-grid-box quad lists, Sec. 6.3).
struct GroupArgs {
    const uint64_t *ent_key;       // pair << 32 | cell << 1 | role
    const uint32_t *ent_face;
    const unsigned long long *d_n; // entry count
    unsigned long long cap;        // entry capacity
    uint32_t *ent_slot;            // [cap] table slot of each entry | role << 31
    uint32_t *ent_rank;            // [cap] rank within (cell, role)
    unsigned long long *tkey;      // [tsize] (pair << 31 | cell) + 1, or kHashEmpty
    uint2 *tcnt;                   // [tsize] A and B entry counts
    uint2 *tstart;                 // [tsize] the slot's A and B list starts (kNoCell: no cell)
    unsigned long long tsize;      // power of two; grown by the host when over half full
    // per compacted cell, [cap / 2]
    CellRec *cells;
    const Grid *grids;             // per pair (cells per coordinate)
    uint32_t *grouped;             // [cap] face ids by cell, A then B
    unsigned long long *partials;  // [5 * 1024]
    Counters *ctr;
};
// table counts and ranks (1 launch), then the cells and the scatter (4 launches);
// the table is left with every slot free
void launch_group_count(const GroupArgs &a, int grid, cudaStream_t st);
void launch_group_cells(const GroupArgs &a, int grid, cudaStream_t st);

struct EmitArgs {
    const CellRec *cells;          // the cells holding faces of both meshes
    const uint32_t *vals;          // face ids grouped by cell
    const Grid *grids;
    const MeshDev *meshes;
    const int2 *pairs;
    Counters *ctr;
    unsigned long long ent_cap;
    Cand *cand;
    unsigned long long cand_cap;
    unsigned long long *cand_ctr;  // the output's counter (candidates, or patch pairs)
    int moller;
    int waves;                     // waves of resident blocks (0: the default, 4)
};
// whole waves of resident blocks on `sms` SMs
void launch_emit(const EmitArgs &a, int precision, int face_level, int sms, cudaStream_t st);
void configure_emit();

// Quad pairs of the patch pairs (patch level): one warp per patch pair, one
// lane per quad of each patch; each side's quads are first tested against the
// other patch's box, then every surviving pair, and the box-overlapping quad
// pairs are appended as candidates.  A quad pair lies in exactly one patch
// pair, so each is emitted once.
struct PatchArgs {
    const Cand *ppairs;            // patch pairs (faceA, faceB = patch ids)
    Cand *psurv;                   // those with an overlapping quarter pair (pad = mask)
    unsigned long long ppair_cap;
    const MeshDev *meshes;         // the meshes (quad and patch boxes)
    const int2 *pairs;
    Counters *ctr;
    unsigned long long ent_cap;
    Cand *cand;
    unsigned long long cand_cap;
    int moller;
    int frames;                    // 1: patch pairs whose frames prove that no
                                   // triangle pair in them is an FP64 hit are dropped
    double tau;                    // the hit test's margin tolerance
};
void launch_patch_quads(const PatchArgs &a, int precision, int sms, cudaStream_t st);

void configure_patch_quads();

struct NarrowArgs {
    const Cand *cand;
    unsigned long long cand_cap;
    uint32_t *qsurv;               // [cand_cap] candidates the quad-level test left
    Cand *surv;                    // triangle pairs left for the FP64 solve
    unsigned long long surv_cap;
    const MeshDev *meshes;
    const int2 *pairs;
    Counters *ctr;
    tms_hit *hits;
    uint64_t *hit_key;
    uint32_t *hit_val;
    unsigned long long hit_cap;
    double tau;
    int tri_bits;
    int fp32_filter;
};
// the quad-level test over all candidates (quad faces), then the filter on what it
// left as one wave of resident blocks on `sms` SMs, the FP64 solve on `grid` blocks
void launch_narrow(const NarrowArgs &a, int face_level, int sms, int grid, cudaStream_t st);
void configure_narrow();

// FP32 split of a double: hi = RN32(x), lo = RN32(x - hi), integer operations
// only in the normal range
__device__ __forceinline__ void split_f32(double x, float &hi, float &lo) {
    hi = f32_rn(x);
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    const int e32 = e - 896;
    // x = sign * (2^52 + m) * 2^(e - 1075); the low 29 bits of m were rounded away
    const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
    const int rem = (int)(m & 0x1FFFFFFFULL);
    const unsigned hb = __float_as_uint(hi) & 0x7fffffffu;
    const unsigned trunc = ((unsigned)e32 << 23) | (unsigned)(m >> 29);
    // rounded up (|hi| > |x|): x - hi = -(2^29 - rem) ulp, else +rem ulp (ulp = 2^(e-1075))
    const int r = (hb != trunc) ? rem - (1 << 29) : rem;
    const int ex = e - 1075 + 127;   // 2^(e - 1075) as an FP32 power of two
    float l = 0.0f;
    if (e32 > 0 && e32 < 255 && ex >= 1) l = __int2float_rn(r) * __uint_as_float((unsigned)ex << 23);
    // outside that range lo is 0 and the caller's error bound carries an absolute
    // term for coordinates below 2^-74
    lo = (b >> 63) ? -l : l;
}

// All four FP32 roundings the bounds pass needs from one decomposition of x:
// rd / ru the FP32 numbers just below and above x (outward box bounds) and the
// split hi = RN32(x), lo = RN32(x - hi); identical to f32_rd, f32_ru and
// split_f32, which take the special cases (zero, subnormal, huge, NaN).
__device__ __forceinline__ void f32_all(double x, float &rd, float &ru, float &hi, float &lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    const int e32 = e - 896;
    if (e32 <= 0 || e32 >= 255) {
        rd = f32_rd(x);
        ru = f32_ru(x);
        split_f32(x, hi, lo);
        return;
    }
    const unsigned long long m = b & 0xFFFFFFFFFFFFFULL;
    const unsigned mag = ((unsigned)e32 << 23) | (unsigned)(m >> 29);   // truncated |x|
    const unsigned rem = (unsigned)(m & 0x1FFFFFFFULL);               // the 29 bits dropped
    const unsigned neg = (unsigned)(b >> 63);
    const unsigned sgn = neg << 31;
    const unsigned inexact = rem != 0u;
    rd = __uint_as_float(sgn | (mag + (neg & inexact)));
    ru = __uint_as_float(sgn | (mag + ((neg ^ 1u) & inexact)));
    const unsigned up = (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & (mag & 1u));
    hi = __uint_as_float(sgn | (mag + up));
    // x - hi = (rem - up 2^29) ulp, ulp = 2^(e - 1075)
    const int r = up ? (int)rem - (1 << 29) : (int)rem;
    const int ex = e - 1075 + 127;
    float l = 0.0f;
    if (ex >= 1) l = __int2float_rn(r) * __uint_as_float((unsigned)ex << 23);
    lo = neg ? -l : l;
}

struct DedupArgs {
    const uint64_t *keys;          // sorted hit keys
    const uint32_t *vals;          // sorted raw-hit indices
    const tms_hit *raw;
    const MeshDev *meshes;
    const int2 *pairs;
    Counters *ctr;
    unsigned long long raw_cap;
    uint32_t *keep;
    uint32_t *keep_scan;
    unsigned long long *partials;
    tms_hit *out;
    unsigned long long out_cap;
    uint64_t *out_keys;            // [raw_cap], scratch for offsets
    long long *offsets;            // nPairs + 1 (may be null)
    int n_pairs;
    int tri_bits;
    double tau;
};
void launch_dedup(const DedupArgs &a, int grid, cudaStream_t st);


struct AdjointArgs {
    const tms_hit *hits;
    long long n;
    MeshDev A, B;
    const double *gP, *gZ;
    double *gA[4];
    double *gB[4];
    const double *dA[4];
    const double *dB[4];
    double *galpha;
};
void launch_adjoint(const AdjointArgs &a, cudaStream_t st);

// device view of a mesh handle (TMS_ERR_STATE for an invalid handle)
tms_status mesh_view(tms_mesh m, MeshDev *view, int *device);

// The search with per-pair cell multipliers (empty: params->cell_mult for all);
// tms_search and tms_search_batched after resolving params->autotune_cache.
tms_status search_with_cm(const tms_mesh *A, const tms_mesh *B, int nPairs, const tms_params &params,
                          const std::vector<float> &cm_pair, tms_hit *dHits, long long hitCap,
                          long long *dOffsets, long long *nHits, void *stream);

// Tuned settings for these meshes from an autotune cache file: overrides the
// face level, patch level, bounds-pass tile and cell multiplier in *p and sets
// per-pair multipliers (empty when no size class has its own); false when the
// file holds nothing for them.  Each file is read once per batch and process.
bool tune_lookup(const tms_mesh *A, const tms_mesh *B, int nPairs, const char *path, tms_params *p,
                 std::vector<float> *cm_pair);

// Message returned by tms_last_error() on the calling thread.
void set_last_error(const std::string &msg);

}  // namespace tms

// Face passes of the broad phase.
//
// Broad phase of arXiv 2109.14814, Sec. 6.2.1-6.2.2, re-designed for GB300:
//   bounds pass      (one read of every vertex) per-mesh world bounds, widest
//                    face extent per coordinate (the grid rule of Sec. 6.2.1:
//                    cell edge > widest face), a finiteness check of every
//                    vertex, the box of every face (Sec. 6.2.2) and the FP32
//                    split copy of the vertices for the narrow filter;
//   cell passes      (one read of every face box) the cells each face covers:
//     MODE_MARK        occupancy bits of the cells covered by mesh A's faces;
//     MODE_PROBE_MARK  mesh B: one entry per face-cell incidence in a cell that
//                      mesh A occupies, and those cells marked "hot";
//     MODE_PROBE       mesh A: one entry per face-cell incidence in a hot cell;
//     MODE_EMIT_ALL    one entry per face-cell incidence (no filter).
// Cells that do not hold faces of both meshes are dropped, as the paper drops
// grid boxes whose quad list is empty on either side (Sec. 6.3); the occupancy
// bitmaps only decide this before any list is built.  A bitmap is a blocked
// Bloom filter over hash(pair, cell): a false positive only adds entries, never
// removes one, so every face pair sharing a cell still meets in the sort.
//
// Bounds pass tiling: a block owns a tile of TI quads along theta x TK quad
// rows.  All (TI+1) x (TK+1) vertices of the tile are loaded once, coalesced
// along theta, into shared memory (converted to FP32 lower/upper bounds in the
// mixed precision mode), then each thread builds the boxes of its quads' faces.
//
// Cell passes: one thread per face slot; a warp expands its 32 faces' cell
// ranges into one list of (face, cell) items and works through it 32 items at
// a time, so its loop runs ceil(sum of cells / 32) times instead of 32 x the
// largest count.  An entry is (key = pair << 32 | cell << 1 | role, face id).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "tms_common.cuh"

namespace tms {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <int PREC>
struct Vtx;

// mixed precision: a vertex as FP32 lower and upper bounds of its coordinates
template <>
struct Vtx<1> {
    float lo[4], hi[4];
};

// plain FP64
template <>
struct Vtx<0> {
    double v[4];
};

template <int PREC>
struct BoxT;
template <>
struct BoxT<1> {
    float lo[4], hi[4];
};
template <>
struct BoxT<0> {
    double lo[4], hi[4];
};

__device__ __forceinline__ void box_init(BoxT<1> &b, const Vtx<1> &v) {
#pragma unroll
    for (int d = 0; d < 4; ++d) { b.lo[d] = v.lo[d]; b.hi[d] = v.hi[d]; }
}
__device__ __forceinline__ void box_add(BoxT<1> &b, const Vtx<1> &v) {
#pragma unroll
    for (int d = 0; d < 4; ++d) { b.lo[d] = fminf(b.lo[d], v.lo[d]); b.hi[d] = fmaxf(b.hi[d], v.hi[d]); }
}
__device__ __forceinline__ void box_init(BoxT<0> &b, const Vtx<0> &v) {
#pragma unroll
    for (int d = 0; d < 4; ++d) { b.lo[d] = v.v[d]; b.hi[d] = v.v[d]; }
}
__device__ __forceinline__ void box_add(BoxT<0> &b, const Vtx<0> &v) {
#pragma unroll
    for (int d = 0; d < 4; ++d) { b.lo[d] = fmin(b.lo[d], v.v[d]); b.hi[d] = fmax(b.hi[d], v.v[d]); }
}

__device__ __forceinline__ void to_vtx(const double x[4], Vtx<1> &v) {
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        v.lo[d] = f32_rd(x[d]);
        v.hi[d] = f32_ru(x[d]);
    }
}
__device__ __forceinline__ void to_vtx(const double x[4], Vtx<0> &v) {
#pragma unroll
    for (int d = 0; d < 4; ++d) v.v[d] = x[d];
}

// FP32 split copy of a vertex (hi and lo float4), gathered later by the FP32
// narrow filter: one 32-byte record per vertex instead of four 8-byte loads
__device__ __forceinline__ void write_split(const MeshDev &m, size_t idx, const double x[4]) {
    float4 hi, lo;
    split_f32(x[0], hi.x, lo.x);
    split_f32(x[1], hi.y, lo.y);
    split_f32(x[2], hi.z, lo.z);
    split_f32(x[3], hi.w, lo.w);
    m.split[idx] = hi;
    m.split[(size_t)m.N * m.M + idx] = lo;
}

// The tile's own vertex: its FP32 bounds for the boxes and its split copy,
// from one decomposition per coordinate in the mixed mode.
template <int PREC>
__device__ __forceinline__ void vtx_and_split(const double x[4], Vtx<PREC> &out, const MeshDev &m,
                                              size_t idx);
template <>
__device__ __forceinline__ void vtx_and_split<1>(const double x[4], Vtx<1> &out, const MeshDev &m,
                                                 size_t idx) {
    Vtx<1> v;
    float4 hi, lo;
    f32_all(x[0], v.lo[0], v.hi[0], hi.x, lo.x);
    f32_all(x[1], v.lo[1], v.hi[1], hi.y, lo.y);
    f32_all(x[2], v.lo[2], v.hi[2], hi.z, lo.z);
    f32_all(x[3], v.lo[3], v.hi[3], hi.w, lo.w);
    out = v;
    m.split[idx] = hi;
    m.split[(size_t)m.N * m.M + idx] = lo;
}
template <>
__device__ __forceinline__ void vtx_and_split<0>(const double x[4], Vtx<0> &out, const MeshDev &m,
                                                 size_t idx) {
    to_vtx(x, out);
    write_split(m, idx, x);
}

template <int PREC>
struct GridView;
template <>
struct GridView<1> {
    float o[4], e[4], inv[4];
    int n[4];
    __device__ void load(const Grid &g) {
#pragma unroll
        for (int d = 0; d < 4; ++d) { o[d] = g.o32[d]; e[d] = g.e32[d]; inv[d] = g.inv32[d]; n[d] = g.n[d]; }
    }
};
template <>
struct GridView<0> {
    double o[4], e[4], inv[4];
    int n[4];
    __device__ void load(const Grid &g) {
#pragma unroll
        for (int d = 0; d < 4; ++d) { o[d] = g.o64[d]; e[d] = g.e64[d]; inv[d] = g.inv64[d]; n[d] = g.n[d]; }
    }
};

// the box of a face (or patch) into slot `face` of a box array
template <int PREC>
__device__ __forceinline__ void write_box(void *arr, uint32_t face, const BoxT<PREC> &b);
template <>
__device__ __forceinline__ void write_box<1>(void *arr, uint32_t face, const BoxT<1> &b) {
    float4 *p = reinterpret_cast<float4 *>(arr) + 2 * (size_t)face;
    p[0] = make_float4(b.lo[0], b.lo[1], b.lo[2], b.lo[3]);
    p[1] = make_float4(b.hi[0], b.hi[1], b.hi[2], b.hi[3]);
}
template <>
__device__ __forceinline__ void write_box<0>(void *arr, uint32_t face, const BoxT<0> &b) {
    double2 *p = reinterpret_cast<double2 *>(arr) + 4 * (size_t)face;
    p[0] = make_double2(b.lo[0], b.lo[1]);
    p[1] = make_double2(b.lo[2], b.lo[3]);
    p[2] = make_double2(b.hi[0], b.hi[1]);
    p[3] = make_double2(b.hi[2], b.hi[3]);
}
template <int PREC>
__device__ __forceinline__ void write_fbox(const MeshDev &m, uint32_t face, const BoxT<PREC> &b) {
    write_box<PREC>(m.fbox, face, b);
}

// a box that contains nothing (identity of the union)
__device__ __forceinline__ void box_empty(BoxT<1> &b) {
#pragma unroll
    for (int d = 0; d < 4; ++d) { b.lo[d] = __int_as_float(0x7f800000); b.hi[d] = -b.lo[d]; }
}
__device__ __forceinline__ void box_empty(BoxT<0> &b) {
#pragma unroll
    for (int d = 0; d < 4; ++d) { b.lo[d] = __longlong_as_double(0x7ff0000000000000LL); b.hi[d] = -b.lo[d]; }
}
template <int PREC>
__device__ __forceinline__ void box_union(BoxT<PREC> &b, const BoxT<PREC> &x) {
#pragma unroll
    for (int d = 0; d < 4; ++d) { b.lo[d] = min(b.lo[d], x.lo[d]); b.hi[d] = max(b.hi[d], x.hi[d]); }
}
// union over aligned groups of `lanes` lanes (a quarter's 4 columns, a patch's 8)
template <int PREC>
__device__ __forceinline__ void box_reduce_lanes(BoxT<PREC> &b, int from, int lanes) {
#pragma unroll
    for (int off = from; off < lanes; off <<= 1) {
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            b.lo[d] = min(b.lo[d], __shfl_xor_sync(0xffffffffu, b.lo[d], off));
            b.hi[d] = max(b.hi[d], __shfl_xor_sync(0xffffffffu, b.hi[d], off));
        }
    }
}

template <int PREC>
__device__ __forceinline__ void read_fbox(const MeshDev &m, uint32_t face, BoxT<PREC> &b);
template <>
__device__ __forceinline__ void read_fbox<1>(const MeshDev &m, uint32_t face, BoxT<1> &b) {
    const float4 *p = reinterpret_cast<const float4 *>(m.fbox) + 2 * (size_t)face;
    const float4 l = __ldg(p), h = __ldg(p + 1);
    b.lo[0] = l.x; b.lo[1] = l.y; b.lo[2] = l.z; b.lo[3] = l.w;
    b.hi[0] = h.x; b.hi[1] = h.y; b.hi[2] = h.z; b.hi[3] = h.w;
}
template <>
__device__ __forceinline__ void read_fbox<0>(const MeshDev &m, uint32_t face, BoxT<0> &b) {
    const double2 *p = reinterpret_cast<const double2 *>(m.fbox) + 4 * (size_t)face;
    const double2 x0 = __ldg(p), x1 = __ldg(p + 1), x2 = __ldg(p + 2), x3 = __ldg(p + 3);
    b.lo[0] = x0.x; b.lo[1] = x0.y; b.lo[2] = x1.x; b.lo[3] = x1.y;
    b.hi[0] = x2.x; b.hi[1] = x2.y; b.hi[2] = x3.x; b.hi[3] = x3.y;
}

// Per-thread accumulators of the bounds pass, in the box precision (FP32
// min/max in the mixed mode: FP64 arithmetic is a scarce pipe on GB300)
template <int PREC>
struct BoundAcc;
template <>
struct BoundAcc<1> {
    float lo[4], hi[4], w[4];
    unsigned seen;
    __device__ void init() {
#pragma unroll
        for (int d = 0; d < 4; ++d) { lo[d] = __int_as_float(0x7f800000); hi[d] = -lo[d]; w[d] = 0.0f; }
        seen = 0;
    }
    __device__ void add(const BoxT<1> &b) {
        add_bounds(b);
        add_width(b);
    }
    __device__ void add_bounds(const BoxT<1> &b) {
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            lo[d] = fminf(lo[d], b.lo[d]);
            hi[d] = fmaxf(hi[d], b.hi[d]);
        }
        seen = 1;
    }
    __device__ void add_width(const BoxT<1> &b) {
#pragma unroll
        for (int d = 0; d < 4; ++d) w[d] = fmaxf(w[d], b.hi[d] - b.lo[d]);
    }
    __device__ double get_lo(int d) const { return (double)lo[d]; }
    __device__ double get_hi(int d) const { return (double)hi[d]; }
    __device__ double get_w(int d) const { return (double)w[d]; }
};
template <>
struct BoundAcc<0> {
    double lo[4], hi[4], w[4];
    unsigned seen;
    __device__ void init() {
#pragma unroll
        for (int d = 0; d < 4; ++d) { lo[d] = __longlong_as_double(0x7ff0000000000000LL); hi[d] = -lo[d]; w[d] = 0.0; }
        seen = 0;
    }
    __device__ void add(const BoxT<0> &b) {
        add_bounds(b);
        add_width(b);
    }
    __device__ void add_bounds(const BoxT<0> &b) {
#pragma unroll
        for (int d = 0; d < 4; ++d) {
            lo[d] = fmin(lo[d], b.lo[d]);
            hi[d] = fmax(hi[d], b.hi[d]);
        }
        seen = 1;
    }
    __device__ void add_width(const BoxT<0> &b) {
#pragma unroll
        for (int d = 0; d < 4; ++d) w[d] = fmax(w[d], b.hi[d] - b.lo[d]);
    }
    __device__ double get_lo(int d) const { return lo[d]; }
    __device__ double get_hi(int d) const { return hi[d]; }
    __device__ double get_w(int d) const { return w[d]; }
};

// ord_enc of the value as a double: FP64 values directly; FP32 values through the
// exact float -> double conversion done on the bits (integer operations only)
__device__ __forceinline__ unsigned long long ord_enc_any(double v) { return ord_enc(v); }
__device__ __forceinline__ unsigned long long ord_enc_any(float v) {
    const unsigned b = __float_as_uint(v);
    const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
    const unsigned e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    unsigned long long db;
    if (e == 255u) {
        db = sgn | (0x7ffULL << 52) | ((unsigned long long)m << 29);          // inf, NaN
    } else if (e == 0u) {
        if (m == 0u) {
            db = sgn;                                                         // +-0
        } else {
            // subnormal m 2^-149 = 1.f 2^(p - 149), p the top bit of m
            const int p = 31 - __clz(m);
            const unsigned long long frac = ((unsigned long long)m << (52 - p)) & 0xFFFFFFFFFFFFFULL;
            db = sgn | ((unsigned long long)(p - 149 + 1023) << 52) | frac;
        }
    } else {
        db = sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
    }
    const long long bb = (long long)db;
    return (bb >= 0) ? (db | 0x8000000000000000ULL) : ~db;
}

// the pass entry (mesh of a pass) holding global index x, by binary search
__device__ __forceinline__ int find_entry(const FacePassArgs &a, long long x, bool by_face) {
    int lo = 0, hi = a.n_entries - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const long long b = by_face ? a.entries[mid].face_base : a.entries[mid].tile_base;
        if (b <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// patch frames (mixed precision; the record and its bounds are described at
// kFrameF4).  The axes need not be orthonormal for the bounds to hold: the
// remainder r absorbs whatever the rounded axes fail to reproduce, and is
// bounded through the axes' Gram matrix.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dot4f(const float a[4], const float b[4]) {
    return fmaf(a[3], b[3], fmaf(a[2], b[2], fmaf(a[1], b[1], a[0] * b[0])));
}
__device__ __forceinline__ float det3(float a0, float a1, float a2, float b0, float b1, float b2,
                                      float c0, float c1, float c2) {
    return a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0);
}
// the vector orthogonal to a, b and c in R^4 (cofactor expansion of the
// 4 x 4 determinant with rows (x, a, b, c))
__device__ __forceinline__ void cross4(const float a[4], const float b[4], const float c[4], float x[4]) {
    x[0] = det3(a[1], a[2], a[3], b[1], b[2], b[3], c[1], c[2], c[3]);
    x[1] = -det3(a[0], a[2], a[3], b[0], b[2], b[3], c[0], c[2], c[3]);
    x[2] = det3(a[0], a[1], a[3], b[0], b[1], b[3], c[0], c[1], c[3]);
    x[3] = -det3(a[0], a[1], a[2], b[0], b[1], b[2], c[0], c[1], c[2]);
}
// non-negative floats (and NaN, above +inf) compare as their bit patterns:
// an integer maximum of |x| keeps a NaN, which fmaxf would drop
__device__ __forceinline__ unsigned abs_bits(float x) { return __float_as_uint(x) & 0x7fffffffu; }

// The frame of a patch, computed by its kPatchI lanes at the close of its patch
// row and written as kFrameF4 float4 by its first lane.  Every lane of the
// warp calls it (the shuffles are uniform).  pr0: the patch's first vertex
// row in the tile's vertex array sv; rq: its quad rows; pb: its box (held by
// every lane of the patch).
// Axes: e_0, e_1 from the patch's two parameter directions (sums of opposite
// edges, one Gram-Schmidt step), e_2 orthogonal to e_0, e_1 and the coordinate
// axis farthest from their span, e_3 orthogonal to e_0, e_1, e_2.  A patch
// whose parameter directions are zero or unbounded gets a frame that
// separates nothing.
// Bounds, with u = 2^-24, the exact vertex V in its FP32 bounds [lo, hi] and
// d = V - c:
//   |d|_inf <= D = max_i max(pb.hi_i - c_i, c_i - pb.lo_i)   (all V in pb)
//   hi_i - lo_i <= 2^-23 L + 2^-149                           (adjacent floats)
//   d~ = fl(hi - c): |d_i - d~_i| <= (hi_i - lo_i) + u |d~_i|, |d~_i| <= D (1 + u)
//   a~_k = fl(e_k . d~) (4 FMAs, error <= gamma_4 sum_i |e_ki||d~_i|, gamma_4 <
//   4.0001 u), so |e_k . d - a~_k| <= n_k nu, nu = 2^-23 L + 5.001 u D (+ 2^-149)
//   and h_k = max |a~_k| + n_k nu (n_k >= |e_k|_1);
//   r = (I - E^T E) d, so |r|_inf <= g D with g >= ||I - E^T E||_inf, from
//   G~_ij = fl(delta_ij - sum_k e_ki e_kj) (4 FMAs, error <= gamma_4 (1 + 4 e_max^2)).
// Sums and products of non-negative terms are rounded up by a factor 1.0001
// (a handful of roundings of 2^-24 each); absolute terms cover underflow.
__device__ __forceinline__ void patch_frame(const Vtx<1> *sv, int W, int t, int cols_q, int pr0, int rq,
                                            const BoxT<1> &pb, float4 *out, uint32_t p, bool patch_lane) {
    const float u = 5.9604645e-08f;
    const float inf = __int_as_float(0x7f800000);
    const int p0 = t & ~(kPatchI - 1), l = t - p0;
    const int cq = patch_lane ? min(kPatchI, cols_q - p0) : 0;    // the patch's quad columns
    const int pr1 = pr0 + rq;
    float c[4], L = 0.0f, D = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        c[i] = 0.5f * (pb.lo[i] + pb.hi[i]);
        L = fmaxf(L, fmaxf(fabsf(pb.lo[i]), fabsf(pb.hi[i])));
        D = fmaxf(D, fmaxf(pb.hi[i] - c[i], c[i] - pb.lo[i]));
    }
    D *= 1.0001f;
    float t1[4] = {0.0f, 0.0f, 0.0f, 0.0f}, t2[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (patch_lane) {
        const float4 v00 = *reinterpret_cast<const float4 *>(sv[pr0 * W + p0].hi);
        const float4 v01 = *reinterpret_cast<const float4 *>(sv[pr0 * W + p0 + cq].hi);
        const float4 v10 = *reinterpret_cast<const float4 *>(sv[pr1 * W + p0].hi);
        const float4 v11 = *reinterpret_cast<const float4 *>(sv[pr1 * W + p0 + cq].hi);
        t1[0] = (v01.x - v00.x) + (v11.x - v10.x); t2[0] = (v10.x - v00.x) + (v11.x - v01.x);
        t1[1] = (v01.y - v00.y) + (v11.y - v10.y); t2[1] = (v10.y - v00.y) + (v11.y - v01.y);
        t1[2] = (v01.z - v00.z) + (v11.z - v10.z); t2[2] = (v10.z - v00.z) + (v11.z - v01.z);
        t1[3] = (v01.w - v00.w) + (v11.w - v10.w); t2[3] = (v10.w - v00.w) + (v11.w - v01.w);
    }
    float E[4][4];
    const float n1 = dot4f(t1, t1);
    const float s1 = rsqrtf(n1);
#pragma unroll
    for (int i = 0; i < 4; ++i) E[0][i] = t1[i] * s1;
    const float pj = dot4f(t2, E[0]);
#pragma unroll
    for (int i = 0; i < 4; ++i) t2[i] = fmaf(-pj, E[0][i], t2[i]);
    const float n2 = dot4f(t2, t2);
    const float s2 = rsqrtf(n2);
#pragma unroll
    for (int i = 0; i < 4; ++i) E[1][i] = t2[i] * s2;
    // zero or unbounded parameter directions: no frame
    bool bad = !(n1 > 1e-30f && n1 < 1e30f && n2 > 1e-30f && n2 < 1e30f);
    {
        // e_2 from the coordinate axis k farthest from span(e_0, e_1): the one
        // with the least e_0k^2 + e_1k^2 (|cross4(e_0, e_1, axis_k)|^2 is one minus
        // that for orthonormal e_0, e_1)
        int kb = 0;
        float best = __int_as_float(0x7f800000);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float sk = fmaf(E[0][k], E[0][k], E[1][k] * E[1][k]);
            if (sk < best) { best = sk; kb = k; }
        }
        float ax[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) ax[i] = i == kb ? 1.0f : 0.0f;
        float x[4];
        cross4(E[0], E[1], ax, x);
        const float s3 = rsqrtf(dot4f(x, x));
#pragma unroll
        for (int i = 0; i < 4; ++i) E[2][i] = x[i] * s3;
        cross4(E[0], E[1], E[2], x);
        const float s4 = rsqrtf(dot4f(x, x));
#pragma unroll
        for (int i = 0; i < 4; ++i) E[3][i] = x[i] * s4;
    }
    // the vertices: lane l takes column p0 + l of the patch (rows pr0..pr1), and
    // lanes 0..rq the closing column p0 + cq, one vertex each; the integer
    // maximum keeps NaN
    unsigned am[4] = {0u, 0u, 0u, 0u};
    auto vertex = [&](const Vtx<1> &v) {
        const float4 hv = *reinterpret_cast<const float4 *>(v.hi);
        const float d[4] = {hv.x - c[0], hv.y - c[1], hv.z - c[2], hv.w - c[3]};
#pragma unroll
        for (int k = 0; k < 4; ++k) am[k] = max(am[k], abs_bits(dot4f(E[k], d)));
    };
    if (l < cq)
        for (int rr = pr0; rr <= pr1; ++rr) vertex(sv[rr * W + t]);
    if (cq > 0 && l <= rq) vertex(sv[(pr0 + l) * W + p0 + cq]);
#pragma unroll
    for (int off = 1; off < kPatchI; off <<= 1)
#pragma unroll
        for (int k = 0; k < 4; ++k) am[k] = max(am[k], __shfl_xor_sync(0xffffffffu, am[k], off));
    // per-patch terms (every lane alike)
    float nk[4], emax = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        nk[k] = (fabsf(E[k][0]) + fabsf(E[k][1]) + fabsf(E[k][2]) + fabsf(E[k][3])) * 1.0001f;
        emax = fmaxf(emax, fmaxf(fmaxf(fabsf(E[k][0]), fabsf(E[k][1])), fmaxf(fabsf(E[k][2]), fabsf(E[k][3]))));
    }
    // |I - E^T E| (symmetric: ten entries)
    float G[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i; j < 4; ++j) {
            float gij = i == j ? 1.0f : 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) gij = fmaf(-E[k][i], E[k][j], gij);
            G[i][j] = G[j][i] = fabsf(gij);
        }
    float g = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) g = fmaxf(g, (G[i][0] + G[i][1]) + (G[i][2] + G[i][3]));
    g = fmaf((4.0f * 4.0001f) * u, fmaf(4.0f * emax, emax, 1.0f), g) * 1.0001f;
    const float nu = fmaf(5.001f * u, D, 1.1921e-7f * L) * 1.0001f + 1e-30f;
    float h[4], hs = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h[k] = fmaf(nk[k], nu, __uint_as_float(am[k])) * 1.0001f + 1e-36f;
        hs += h[k];
        bad |= !(h[k] < inf);
    }
    // plus the rounding of fl(w . e_k) in the pair test: gamma_4 |w|_1 e_max
    // per unit of h_k
    float rho = fmaf((4.0001f * u) * emax, hs * 1.0001f, g * D * 1.0001f) * 1.0001f + 1e-36f;
    bad |= !(rho < inf) || !(fabsf(E[2][0] + E[2][1] + E[2][2] + E[2][3] + E[3][0] + E[3][1] + E[3][2] + E[3][3]) < inf);
    if (bad) {
        h[0] = h[1] = h[2] = h[3] = inf;
        rho = inf;
    }
    if (patch_lane && l == 0) {
        float4 *o = out + (size_t)p * kFrameF4;
        o[0] = make_float4(c[0], c[1], c[2], c[3]);
        o[1] = make_float4(E[0][0], E[0][1], E[0][2], E[0][3]);
        o[2] = make_float4(E[1][0], E[1][1], E[1][2], E[1][3]);
        o[3] = make_float4(E[2][0], E[2][1], E[2][2], E[2][3]);
        o[4] = make_float4(E[3][0], E[3][1], E[3][2], E[3][3]);
        o[5] = make_float4(h[0], h[1], h[2], h[3]);
        o[6] = make_float4(rho, L, nk[2], nk[3]);
    }
}

// ---------------------------------------------------------------------------
// bounds pass
// ---------------------------------------------------------------------------
template <int PREC, int FACE, int TK>
__global__ void __launch_bounds__(256) k_bounds_pass(FacePassArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Vtx<PREC> *sv = reinterpret_cast<Vtx<PREC> *>(smem_raw);
    const int TI = blockDim.x;
    const int W = TI + 1;
    const long long tile = blockIdx.x;

    const PassEntry pe = a.entries[find_entry(a, tile, false)];
    const MeshDev m = a.meshes[pe.mesh];
    const long long lt = tile - pe.tile_base;
    const int ti = (int)(lt % pe.tiles_i), tk = (int)(lt / pe.tiles_i);
    const int i0 = ti * TI, kq0 = tk * TK;
    const int cols_q = min(TI, m.nqi - i0);
    const int rows_q = min(TK, m.nqk - kq0);

    // ---- load the tile's vertices: rows kq0..kq0+rows_q, columns i0..i0+cols_q
    unsigned nonfinite = 0;
    {
        const int t = threadIdx.x;
        double x[TK + 1][4];
        const bool col_ok = t < cols_q;
        const int vi = i0 + t;
#pragma unroll
        for (int r = 0; r <= TK; ++r) {
            if (col_ok && r <= rows_q) {
                size_t off = (size_t)(kq0 + r) * m.N + vi;
#pragma unroll
                for (int c = 0; c < 4; ++c) x[r][c] = __ldg(m.c[c] + off);
            }
        }
        // a vertex's split copy is written by the tile that owns it: rows below the
        // tile's last (the next tile's first) and the mesh's last row
        const bool last_rows = kq0 + rows_q == m.nqk;
#pragma unroll
        for (int r = 0; r <= TK; ++r) {
            if (col_ok && r <= rows_q) {
#pragma unroll
                for (int c = 0; c < 4; ++c) nonfinite |= !finite64(x[r][c]);
                if (r < rows_q || last_rows)
                    vtx_and_split<PREC>(x[r], sv[r * W + t], m, (size_t)(kq0 + r) * m.N + vi);
                else
                    to_vtx(x[r], sv[r * W + t]);
            }
        }
        // the last vertex column of the tile (wraps to column 0 on a periodic mesh);
        // it belongs to the next tile, except an open mesh's last column
        if (t <= rows_q) {
            int vj = i0 + cols_q;
            if (vj == m.N) vj = 0;
            size_t off = (size_t)(kq0 + t) * m.N + vj;
            double y[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                y[c] = __ldg(m.c[c] + off);
                nonfinite |= !finite64(y[c]);
            }
            const bool own_col = !m.periodic && vj == m.N - 1 && (t < rows_q || last_rows);
            if (own_col) vtx_and_split<PREC>(y, sv[t * W + cols_q], m, off);
            else to_vtx(y, sv[t * W + cols_q]);
        }
    }
    __syncthreads();

    BoundAcc<PREC> acc;
    acc.init();

    const int t = threadIdx.x;
    const bool col_valid = t < cols_q;
    const int i = i0 + t;
    if (FACE == 1 && a.patch) {
        // quad faces with patches: as below, and each column's box over the
        // patch row (kPatchK quad rows; tiles are whole patch rows) united across
        // the kPatchI lanes of the patch (every lane of the block takes part:
        // the row loop and its shuffles are uniform).  The widest extent the
        // grid needs is then the widest patch's.
        // this column's boxes over the upper and lower halves of the patch row
        BoxT<PREC> prev, ptop, pbot, pb0, pb1;   // pb0, pb1: the boxes of the tile's patch rows
        box_empty(prev);
        box_empty(ptop);
        box_empty(pbot);
        box_empty(pb0);
        box_empty(pb1);
        // the patch exists when its first column is in the tile
        const bool patch_lane = (t & ~(kPatchI - 1)) < cols_q;
        if (col_valid) {
            box_init(prev, sv[t]);
            box_add(prev, sv[t + 1]);
        }
        for (int r = 0; r < rows_q; ++r) {
            if (col_valid) {
                BoxT<PREC> next;
                box_init(next, sv[(r + 1) * W + t]);
                box_add(next, sv[(r + 1) * W + t + 1]);
                BoxT<PREC> bq;
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    bq.lo[d] = min(prev.lo[d], next.lo[d]);
                    bq.hi[d] = max(prev.hi[d], next.hi[d]);
                }
                const uint32_t q = (uint32_t)(kq0 + r) * (uint32_t)m.N + (uint32_t)i;
                acc.add_bounds(bq);
                write_fbox<PREC>(m, q, bq);
                if ((r % kPatchK) < kPatchK / 2) box_union<PREC>(ptop, bq);
                else box_union<PREC>(pbot, bq);
                prev = next;
            }
            if ((r % kPatchK) == kPatchK - 1 || r == rows_q - 1) {
                // quarters over 4 columns, then the patch over both column halves
                box_reduce_lanes<PREC>(ptop, 1, kPatchI / 2);
                box_reduce_lanes<PREC>(pbot, 1, kPatchI / 2);
                BoxT<PREC> pb = ptop;
                box_union<PREC>(pb, pbot);
                box_reduce_lanes<PREC>(pb, kPatchI / 2, kPatchI);
                const uint32_t p = (uint32_t)((kq0 + r) / kPatchK) * (uint32_t)m.npi +
                                   (uint32_t)(i / kPatchI);
                if (patch_lane && (t % (kPatchI / 2)) == 0) {
                    const uint32_t half = (uint32_t)((t % kPatchI) / (kPatchI / 2));
                    write_box<PREC>(m.qbox, 4 * p + half, ptop);
                    write_box<PREC>(m.qbox, 4 * p + 2 + half, pbot);
                }
                if (patch_lane && (t % kPatchI) == 0) {
                    write_box<PREC>(m.pbox, p, pb);
                    acc.add_width(pb);
                }
                if (r < kPatchK) pb0 = pb;
                else pb1 = pb;
                box_empty(ptop);
                box_empty(pbot);
            }
        }
        // the frames of the tile's patches, after its rows (fewer registers live
        // than at the close of each patch row)
        if constexpr (PREC == 1) {
            if (a.frames) {
                for (int pr = 0; pr * kPatchK < rows_q; ++pr) {
                    const BoxT<1> pbx = pr == 0 ? pb0 : pb1;
                    const uint32_t p = (uint32_t)(kq0 / kPatchK + pr) * (uint32_t)m.npi + (uint32_t)(i / kPatchI);
                    patch_frame(sv, W, t, cols_q, pr * kPatchK, min(kPatchK, rows_q - pr * kPatchK), pbx,
                                m.pframe, p, patch_lane);
                }
            }
        }
    } else if (FACE == 1 && col_valid) {
        // quad faces: the extremes of the two vertex columns of each row once, each
        // quad box from two consecutive rows (exact: min and max only)
        BoxT<PREC> prev;
        box_init(prev, sv[t]);
        box_add(prev, sv[t + 1]);
        for (int r = 0; r < rows_q; ++r) {
            BoxT<PREC> next;
            box_init(next, sv[(r + 1) * W + t]);
            box_add(next, sv[(r + 1) * W + t + 1]);
            BoxT<PREC> bq;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                bq.lo[d] = min(prev.lo[d], next.lo[d]);
                bq.hi[d] = max(prev.hi[d], next.hi[d]);
            }
            const uint32_t q = (uint32_t)(kq0 + r) * (uint32_t)m.N + (uint32_t)i;
            acc.add(bq);
            write_fbox<PREC>(m, q, bq);
            prev = next;
        }
    } else if (FACE == 0 && col_valid) {
        for (int r = 0; r < rows_q; ++r) {
            const int k = kq0 + r;
            const Vtx<PREC> va = sv[r * W + t];             // (i, k)
            const Vtx<PREC> vb = sv[r * W + t + 1];         // (i+1, k)
            const Vtx<PREC> vc = sv[(r + 1) * W + t];       // (i, k+1)
            const Vtx<PREC> vd = sv[(r + 1) * W + t + 1];   // (i+1, k+1)
            const uint32_t q = (uint32_t)k * (uint32_t)m.N + (uint32_t)i;
            if (FACE == 0) {
                BoxT<PREC> b1, b2;
                box_init(b1, vb); box_add(b1, va); box_add(b1, vc);   // T1: x1=(i+1,k) x2=(i,k) x3=(i,k+1)
                box_init(b2, vc); box_add(b2, vd); box_add(b2, vb);   // T2: x1=(i,k+1) x2=(i+1,k+1) x3=(i+1,k)
                acc.add(b1);
                acc.add(b2);
                write_fbox<PREC>(m, 2 * q, b1);
                write_fbox<PREC>(m, 2 * q + 1, b2);
            } else {
                BoxT<PREC> bq;
                box_init(bq, va); box_add(bq, vb); box_add(bq, vc); box_add(bq, vd);
                acc.add(bq);
                write_fbox<PREC>(m, q, bq);
            }
        }
    }

    // block reduction, then one set of atomics per block
    // in the accumulators' own type: FP32 in the mixed mode (no FP64 instruction
    // in this kernel: GB300's FP64 pipe is narrow), FP64 in the plain mode
    typedef typename std::remove_reference<decltype(acc.lo[0])>::type AccT;
    __shared__ AccT red[8][12];
    __shared__ unsigned redf[8][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        for (int off = 16; off > 0; off >>= 1) {
            acc.lo[d] = min(acc.lo[d], __shfl_xor_sync(FULL, acc.lo[d], off));
            acc.hi[d] = max(acc.hi[d], __shfl_xor_sync(FULL, acc.hi[d], off));
            acc.w[d] = max(acc.w[d], __shfl_xor_sync(FULL, acc.w[d], off));
        }
    }
    unsigned fl = __reduce_or_sync(FULL, nonfinite);
    unsigned seen = __reduce_or_sync(FULL, acc.seen);
    if (lane == 0) {
#pragma unroll
        for (int d = 0; d < 4; ++d) { red[warp][d] = acc.lo[d]; red[warp][4 + d] = acc.hi[d]; red[warp][8 + d] = acc.w[d]; }
        redf[warp][0] = fl;
        redf[warp][1] = seen;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        Bounds *B = a.bounds + pe.mesh;
        unsigned f = 0, s = 0;
        for (int w = 0; w < nw; ++w) { f |= redf[w][0]; s |= redf[w][1]; }
        if (s) {
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                AccT l = red[0][d], h = red[0][4 + d], ww = red[0][8 + d];
                for (int w = 1; w < nw; ++w) {
                    l = min(l, red[w][d]);
                    h = max(h, red[w][4 + d]);
                    ww = max(ww, red[w][8 + d]);
                }
                atomicMin(&B->lo[d], ord_enc_any(l));
                atomicMax(&B->hi[d], ord_enc_any(h));
                atomicMax(&B->w[d], ord_enc_any(ww));
            }
            atomicOr(&B->faces, 1u);
        }
        if (f) {
            atomicOr(&B->flags, ST_NONFINITE);
            atomicOr(&a.ctr->status, ST_NONFINITE);
        }
    }
}

// ---------------------------------------------------------------------------
// cell passes
// ---------------------------------------------------------------------------
constexpr int kCellWarps = 8;

constexpr unsigned kEntryFlush = 224;   // entries per atomic on the entry counter

struct EntryRec {
    uint64_t key;
    uint32_t face;
    uint32_t pad;
};

// coordinate d of item r of a cell range (mixed radix over cnt[0..3]); counts
// of 1 and 2 (the usual case: a cell is wider than any face) take no division
__device__ __forceinline__ unsigned next_digit(unsigned &r, unsigned c) {
    unsigned q;
    if (c <= 2u) q = r >> (c - 1u);
    else q = r / c;
    const unsigned digit = r - q * c;
    r = q;
    return digit;
}

template <int PREC, int MODE>
__global__ void __launch_bounds__(32 * kCellWarps) k_cell_pass(FacePassArgs a, int face_level) {
    __shared__ uint32_t s_excl[kCellWarps][32];
    __shared__ uint2 s_lo[kCellWarps][32];
    __shared__ uint2 s_cnt[kCellWarps][32];
    __shared__ EntryRec s_out[kCellWarps][kEntryFlush + 32];   // staged entries
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long slot = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long wslot = slot - lane;           // the warp's first slot
    if (wslot >= a.total_faces) return;            // whole warps only
    // every mesh starts at a multiple of 32 slots: the warp lies in one mesh
    const PassEntry pe = a.entries[find_entry(a, wslot, true)];
    const Grid &gg = a.grids[pe.pair];
    if (gg.empty) return;
    GridView<PREC> g;
    g.load(gg);
    const MeshDev &mr = a.meshes[pe.mesh];
    const int N = mr.N, nqi = mr.nqi;
    const long long f = slot - pe.face_base;
    // a valid face: inside this mesh's slots, and not the unused last column of
    // an open mesh
    bool valid = f < pe.faces;
    const uint32_t face = (uint32_t)f;
    if (valid) {
        const uint32_t q = face >> (face_level == 0 ? 1 : 0);
        valid = (int)(q % (uint32_t)N) < nqi;
    }
    int clo[4] = {0, 0, 0, 0}, cnt[4] = {1, 1, 1, 1};
    unsigned count = 0;
    if (valid) {
        BoxT<PREC> b;
        read_fbox<PREC>(mr, face, b);
        bool out = false;
#pragma unroll
        for (int d = 0; d < 4; ++d) out |= (b.hi[d] < g.o[d]) || (b.lo[d] > g.e[d]);
        if (!out) {
            count = 1;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                clo[d] = cell_of(b.lo[d], g.o[d], g.inv[d], g.n[d]);
                const int chi = cell_of(b.hi[d], g.o[d], g.inv[d], g.n[d]);
                cnt[d] = chi - clo[d] + 1;
                count *= (unsigned)cnt[d];
            }
        }
    }
    // warp-wide exclusive scan of the counts
    unsigned incl = count;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned v = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += v;
    }
    const unsigned total = __shfl_sync(FULL, incl, 31);
    s_excl[warp][lane] = incl - count;
    s_lo[warp][lane] = make_uint2((uint32_t)clo[0] | ((uint32_t)clo[1] << 16),
                                  (uint32_t)clo[2] | ((uint32_t)clo[3] << 16));
    s_cnt[warp][lane] = make_uint2((uint32_t)cnt[0] | ((uint32_t)cnt[1] << 16),
                                   (uint32_t)cnt[2] | ((uint32_t)cnt[3] << 16));
    __syncwarp();
    const uint64_t pair_hi = (uint64_t)(uint32_t)pe.pair << 32;
    const uint32_t n0 = (uint32_t)g.n[0], n1 = (uint32_t)g.n[1], n2 = (uint32_t)g.n[2];
    EntryRec *stage = s_out[warp];
    unsigned staged = 0;
    uint64_t *const ekey = a.ent_key;
    uint32_t *const eval = a.ent_val;
    const unsigned long long cap = a.ent_cap;
    auto store = [ekey, eval, cap](unsigned long long pos, const EntryRec &r) {
        if (pos < cap) {
            ekey[pos] = r.key;
            eval[pos] = r.face;
        }
    };
    for (unsigned base = 0; base < total; base += 32) {
        const unsigned j = base + lane;
        const bool act = j < total;
        uint32_t cell = 0;
        int owner = 0;
        if (act) {
            // the lane whose range holds item j: the last with excl <= j
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (s_excl[warp][owner + step] <= j) owner += step;
            unsigned r = j - s_excl[warp][owner];
            const uint2 lo = s_lo[warp][owner], cn = s_cnt[warp][owner];
            const uint32_t c0 = (lo.x & 0xFFFFu) + next_digit(r, cn.x & 0xFFFFu);
            const uint32_t c1 = (lo.x >> 16) + next_digit(r, cn.x >> 16);
            const uint32_t c2 = (lo.y & 0xFFFFu) + next_digit(r, cn.y & 0xFFFFu);
            const uint32_t c3 = (lo.y >> 16) + next_digit(r, cn.y >> 16);
            cell = ((c3 * n2 + c2) * n1 + c1) * n0 + c0;
        }
        const uint64_t h = mix64(pair_hi | cell);
        bool emit = false;
        if (MODE == MODE_MARK) {
            if (act) {
                // bits are only ever set during this pass, so a word that already
                // holds them needs no atomic (a stale read only costs an atomic)
                uint32_t w, m;
                bloom_slot(h, a.bmA_word_bits, w, m);
                if ((a.bmA[w] & m) != m) atomicOr(a.bmA + w, m);
            }
        } else if (MODE == MODE_PROBE_MARK) {
            if (act) {
                uint32_t w, m;
                bloom_slot(h, a.bmA_word_bits, w, m);
                if ((__ldg(a.bmA + w) & m) == m) {
                    emit = true;
                    uint32_t w2, m2;
                    bloom_slot(h, a.bmH_word_bits, w2, m2);
                    if ((a.bmH[w2] & m2) != m2) atomicOr(a.bmH + w2, m2);
                }
            }
        } else if (MODE == MODE_PROBE) {
            if (act) {
                uint32_t w2, m2;
                bloom_slot(h, a.bmH_word_bits, w2, m2);
                emit = (__ldg(a.bmH + w2) & m2) == m2;
            }
        } else {  // MODE_EMIT_ALL
            emit = act;
        }
        if (MODE != MODE_MARK) {
            EntryRec r;
            r.key = pair_hi | ((uint64_t)cell << 1) | (uint64_t)pe.role;
            r.face = (uint32_t)(wslot - pe.face_base) + (uint32_t)owner;
            stage_push<kEntryFlush>(stage, staged, emit, r, &a.ctr->entries, store);
        }
    }
    if (MODE != MODE_MARK) {
        __syncwarp();
        stage_flush<kEntryFlush>(stage, staged, &a.ctr->entries, store);
    }
}

// The start of a search, in one launch: counters zeroed, per-mesh bounds
// reset, and the two occupancy bitmaps cleared (n32a and n32h words, each a
// multiple of four).
__global__ void k_search_init(Bounds *b, int n, Counters *ctr, uint32_t *bmA,
                              unsigned long long n32a, uint32_t *bmH, unsigned long long n32h) {
    const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    if (tid == 0) memset(ctr, 0, sizeof(Counters));
    if (tid < (unsigned long long)n) {
        Bounds &m = b[tid];
#pragma unroll
        for (int d = 0; d < 4; ++d) { m.lo[d] = ~0ULL; m.hi[d] = 0ULL; m.w[d] = 0ULL; }
        m.flags = 0;
        m.faces = 0;
    }
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    if (bmA)
        for (unsigned long long i = tid; i < n32a / 4; i += stride) reinterpret_cast<uint4 *>(bmA)[i] = z;
    if (bmH)
        for (unsigned long long i = tid; i < n32h / 4; i += stride) reinterpret_cast<uint4 *>(bmH)[i] = z;
}

// Trimmed world and uniform grid of each pair (Sec. 6.2.1 and its remark).
// World along coordinate d: the overlap of the two meshes' ranges; a face whose
// box misses it cannot meet any face of the other mesh.  Cell edge: cell_mult x
// the widest face extent of either mesh, so that a face spans at most two cells
// per coordinate; capped so that a pair's grid has fewer than 2^31 cells.
__global__ void k_grid_params(const Bounds *b, const int2 *pairs, int n_pairs, Grid *grids,
                              float cell_mult, const float *cm_pair) {
    // one warp per pair, lane d & 3 speaks for coordinate d: the FP64 chain of
    // one coordinate instead of four (FP64 arithmetic is slow on GB300)
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= n_pairs) return;                      // whole warps
    const int lane = threadIdx.x & 31, d = lane & 3;
    const Bounds &A = b[pairs[p].x];
    const Bounds &B = b[pairs[p].y];
    const double o = fmax(ord_dec(A.lo[d]), ord_dec(B.lo[d]));
    const double e = fmin(ord_dec(A.hi[d]), ord_dec(B.hi[d]));
    const int empty = (A.faces == 0 || B.faces == 0 || __any_sync(FULL, !(o <= e))) ? 1 : 0;
    const float cm = cm_pair ? cm_pair[p] : cell_mult;
    double step = (double)cm * fmax(ord_dec(A.w[d]), ord_dec(B.w[d]));
    const double range = empty ? 0.0 : e - o;
    int n;
    if (!(range > 0.0) || !(step > 0.0)) {
        n = 1;
        step = 0.0;
    } else {
        if (range / step > (double)(kMaxCellsPerDim - 1)) step = range / (double)(kMaxCellsPerDim - 1);
        n = (int)floor(range / step) + 1;
        if (n > kMaxCellsPerDim) n = kMaxCellsPerDim;
    }
    const double cap = 2147483647.0;
    for (int iter = 0; iter < 64; ++iter) {
        double prod = (double)n;
        prod *= __shfl_xor_sync(FULL, prod, 1);
        prod *= __shfl_xor_sync(FULL, prod, 2);
        if (prod <= cap) break;                    // the same in every lane
        const double f = sqrt(sqrt(prod / cap)) * 1.001;
        if (n > 1) {
            step *= f;
            n = (int)floor(range / step) + 1;
            if (n < 1) n = 1;
        }
    }
    if (lane < 4) {
        Grid &G = grids[p];
        const double inv = (step > 0.0) ? 1.0 / step : 0.0;
        G.o64[d] = o;
        G.e64[d] = e;
        G.inv64[d] = inv;
        G.o32[d] = (float)o;
        G.e32[d] = (float)e;
        G.inv32[d] = (float)inv;
        G.n[d] = n;
        if (d == 0) {
            G.empty = empty;
            G.pad[0] = G.pad[1] = G.pad[2] = 0;
        }
    }
}

template <int PREC, int FACE, int TK>
void launch_one(const FacePassArgs &a, int block, cudaStream_t st) {
    size_t smem = (size_t)(TK + 1) * (block + 1) * sizeof(Vtx<PREC>);
    k_bounds_pass<PREC, FACE, TK><<<(unsigned)a.total_tiles, block, smem, st>>>(a);
}

template <int PREC, int FACE>
void launch_tk(const FacePassArgs &a, int block, cudaStream_t st) {
    if (a.tile_rows == 4) launch_one<PREC, FACE, 4>(a, block, st);
    else launch_one<PREC, FACE, 8>(a, block, st);
}

template <int PREC, int FACE, int TK>
cudaError_t configure_one() {
    return cudaFuncSetAttribute(k_bounds_pass<PREC, FACE, TK>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}

template <int PREC>
void launch_cells_mode(const FacePassArgs &a, int face_level, cudaStream_t st) {
    const int B = 32 * kCellWarps;
    const unsigned grid = (unsigned)((a.total_faces + B - 1) / B);
    switch (a.mode) {
        case MODE_MARK: k_cell_pass<PREC, MODE_MARK><<<grid, B, 0, st>>>(a, face_level); break;
        case MODE_PROBE_MARK: k_cell_pass<PREC, MODE_PROBE_MARK><<<grid, B, 0, st>>>(a, face_level); break;
        case MODE_PROBE: k_cell_pass<PREC, MODE_PROBE><<<grid, B, 0, st>>>(a, face_level); break;
        default: k_cell_pass<PREC, MODE_EMIT_ALL><<<grid, B, 0, st>>>(a, face_level); break;
    }
}

}  // namespace

// Sets kernel attributes once, before any launch (and outside stream capture).
cudaError_t configure_face_pass() {
    cudaError_t e = cudaSuccess;
    cudaError_t r;
#define TMS_CFG(P, F, T) if ((r = configure_one<P, F, T>()) != cudaSuccess) e = r;
    TMS_CFG(0, 0, 4) TMS_CFG(0, 0, 8) TMS_CFG(0, 1, 4) TMS_CFG(0, 1, 8)
    TMS_CFG(1, 0, 4) TMS_CFG(1, 0, 8) TMS_CFG(1, 1, 4) TMS_CFG(1, 1, 8)
#undef TMS_CFG
    return e;
}

void launch_face_pass(const FacePassArgs &a, int precision, int face_level, int block,
                      cudaStream_t st) {
    if (a.mode == MODE_BOUNDS) {
        if (a.total_tiles <= 0) return;
        if (precision == 1) {
            if (face_level == 0) launch_tk<1, 0>(a, block, st); else launch_tk<1, 1>(a, block, st);
        } else {
            if (face_level == 0) launch_tk<0, 0>(a, block, st); else launch_tk<0, 1>(a, block, st);
        }
        return;
    }
    if (a.total_faces <= 0) return;
    if (precision == 1) launch_cells_mode<1>(a, face_level, st);
    else launch_cells_mode<0>(a, face_level, st);
}

void launch_search_init(Bounds *b, int n, Counters *ctr, uint32_t *bmA, unsigned long long n32a,
                        uint32_t *bmH, unsigned long long n32h, int grid, cudaStream_t st) {
    k_search_init<<<grid, 256, 0, st>>>(b, n, ctr, bmA, n32a, bmH, n32h);
}

void launch_grid_params(const Bounds *b, const int2 *pairs, int n_pairs, Grid *g,
                        float cell_mult, cudaStream_t st, const float *cm_pair) {
    k_grid_params<<<(n_pairs + 3) / 4, 128, 0, st>>>(b, pairs, n_pairs, g, cell_mult, cm_pair);
}

}  // namespace tms

// Narrow phase, merging of duplicate hits, output, and the adjoint.
//
// Narrow phase (arXiv 2109.14814, Sec. 6.2.4, Eq. (precise)): for triangles
// (x1, x2, x3) and (y1, y2, y3), the unknowns (a, b, c, d) solve the 4x4 system
//   [x1-x2 | x3-x2 | y2-y1 | y2-y3] (a, b, c, d)^T = y2 - x2,
// and the triangles meet iff a, b, c, d >= 0, a + b <= 1, c + d <= 1; the common
// point is x2 + a(x1-x2) + b(x3-x2).  The paper ran this on the CPU; here it is
// one thread per triangle pair in FP64 (Gaussian elimination with partial
// pivoting).  Readings of the paper fixed by this library: the inequalities are
// closed with tolerance tau (margin = min(a, b, c, d, 1-a-b, 1-c-d) >= -tau),
// and a singular system (a zero pivot) is not a hit.  The (theta, s) estimates
// are the interpolation formulas that follow Eq. (precise).
//
// Mixed precision (optional): a verified FP32 solve first.  The system is formed
// in FP32 from a split copy of the vertices (hi + lo per coordinate), with a
// bound on every entry's error.  Gaussian elimination on [A | I | r] gives z~
// and an approximate inverse C; with alpha >= |I - C A|_inf (computed with its
// rounding and input-error terms), A is nonsingular when alpha < 1 and
//   |z - z~|_inf <= | |C| |r - A z~| |_inf / (1 - alpha),
// the residual again bounded with its rounding and input errors.  A pair is
// rejected in FP32 only when the resulting upper bound of the margin is below
// -2 tau minus an allowance for the FP64 solve's own rounding (so an FP64 solve
// of the same system could not call it a hit); all other pairs, and every
// pair whose certificate fails, get the FP64 solve.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tms_common.cuh"

namespace tms {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// ---------------------------------------------------------------------------
// FP64 Gaussian elimination with partial pivoting, fully unrolled in registers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void swap_(T &a, T &b) {
    T t = a;
    a = b;
    b = t;
}

template <typename T>
__device__ __forceinline__ bool solve4_gepp(T A[4][4], T r[4], T z[4], T &det) {
    T sign = 1;
    T inv[4];
    bool ok = true;
#pragma unroll
    for (int col = 0; col < 4; ++col) {
        int p = col;
        T best = fabs(A[col][col]);
#pragma unroll
        for (int row = col + 1; row < 4; ++row) {
            T v = fabs(A[row][col]);
            if (v > best) { best = v; p = row; }
        }
        ok &= best != T(0);
#pragma unroll
        for (int row = col + 1; row < 4; ++row) {
            const bool sw = (p == row);     // branch-free select keeps A in registers
#pragma unroll
            for (int j = col; j < 4; ++j) {
                const T lo = A[col][j], hi = A[row][j];
                A[col][j] = sw ? hi : lo;
                A[row][j] = sw ? lo : hi;
            }
            const T rl = r[col], rh = r[row];
            r[col] = sw ? rh : rl;
            r[row] = sw ? rl : rh;
            sign = sw ? -sign : sign;
        }
        inv[col] = T(1) / A[col][col];
#pragma unroll
        for (int row = col + 1; row < 4; ++row) {
            T f = A[row][col] * inv[col];
#pragma unroll
            for (int j = col + 1; j < 4; ++j) A[row][j] = A[row][j] - f * A[col][j];
            r[row] = r[row] - f * r[col];
        }
    }
#pragma unroll
    for (int row = 3; row >= 0; --row) {
        T acc = r[row];
#pragma unroll
        for (int j = row + 1; j < 4; ++j) acc = acc - A[row][j] * z[j];
        z[row] = acc * inv[row];
    }
    det = sign * A[0][0] * A[1][1] * A[2][2] * A[3][3];
    return ok;
}

__device__ __forceinline__ void gather_tri(const MeshDev &m, uint32_t t, double v[3][4]) {
    int ii[3], kk[3];
    tri_ij(m, t, ii, kk);
#pragma unroll
    for (int j = 0; j < 3; ++j) load_vertex(m, ii[j], kk[j], v[j]);
}

// One entry of the FP32 system: the difference p - q of two split coordinates and
// a bound on its error against the exact difference of the FP64 coordinates.
__device__ __forceinline__ float split_diff(float hp, float lp, float hq, float lq, float &err) {
    const float u = 5.9604645e-08f;
    const float t1 = hp - hq, t2 = lp - lq;
    const float d = t1 + t2;
    // relative rounding of the three FP32 operations, the split remainders, and an
    // absolute term for coordinates below 2^-74 (whose lo part is not kept)
    err = (u * (fabsf(t1) + fabsf(t2) + fabsf(d))) * 1.0001f + (u * u) * (fabsf(hp) + fabsf(hq)) * 1.01f +
          1e-29f;
    return d;
}

__device__ __forceinline__ void gather_split(const MeshDev &m, uint32_t t, float4 v[3][2]) {
    int ii[3], kk[3];
    tri_ij(m, t, ii, kk);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const size_t idx = (size_t)kk[j] * m.N + ii[j];
        v[j][0] = __ldg(m.split + idx);
        v[j][1] = __ldg(m.split + (size_t)m.N * m.M + idx);
    }
}

__device__ __forceinline__ float comp(const float4 &v, int c) {
    return c == 0 ? v.x : (c == 1 ? v.y : (c == 2 ? v.z : v.w));
}

// (i, k) of quad q = k N + i
__device__ __forceinline__ void quad_ik(const MeshDev &m, uint32_t q, int &i, int &k) {
    const uint32_t kk = (uint32_t)__umul64hi((unsigned long long)q, m.nmagic);
    k = (int)kk;
    i = (int)(q - kk * (uint32_t)m.N);
}

// the high halves of the split copies of the quad's vertices (i,k), (i+1,k),
// (i,k+1), (i+1,k+1) (the FP32 rounding of each coordinate)
__device__ __forceinline__ void gather_quad_hi(const MeshDev &m, uint32_t q, float4 v[4]) {
    int i, k;
    quad_ik(m, q, i, k);
    const int ip = (i + 1 == m.N) ? 0 : i + 1;
    const size_t idx[4] = {(size_t)k * m.N + i, (size_t)k * m.N + ip, (size_t)(k + 1) * m.N + i,
                           (size_t)(k + 1) * m.N + ip};
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __ldg(m.split + idx[j]);
}

// Overlap of the two triangles' boxes, as the separating-axis test along each
// coordinate axis: each coordinate's interval from the split copies (widened by
// the split remainder and a relative 1e-6, more than the FP32 rounding of the
// test), and the pair dropped only when a gap exceeds 3 tau' (D_X + D_Y) plus the
// FP64 solve's reach (the triangles widened to weights >= -tau', widen3 and
// fp64_reach, with max|A| at most the largest extent and |r| at most twice the
// largest coordinate) -- so that no FP64 hit is dropped whatever tau.
__device__ __forceinline__ bool split_boxes_overlap(const float4 X[3][2], const float4 Y[3][2], float tau) {
    float xl[4], xh[4], yl[4], yh[4];
    float dmax = 0.0f, cmax = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        xl[c] = 3.4e38f; xh[c] = -3.4e38f; yl[c] = 3.4e38f; yh[c] = -3.4e38f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float hx = comp(X[j][0], c), lx = comp(X[j][1], c);
            const float dx = fabsf(lx) + 1e-6f * fabsf(hx) + 1e-29f;
            xl[c] = fminf(xl[c], hx - dx);
            xh[c] = fmaxf(xh[c], hx + dx);
            const float hy = comp(Y[j][0], c), ly = comp(Y[j][1], c);
            const float dy = fabsf(ly) + 1e-6f * fabsf(hy) + 1e-29f;
            yl[c] = fminf(yl[c], hy - dy);
            yh[c] = fmaxf(yh[c], hy + dy);
        }
        dmax = fmaxf(dmax, fmaxf(xh[c] - xl[c], yh[c] - yl[c]));
        cmax = fmaxf(cmax, fmaxf(fmaxf(fabsf(xl[c]), fabsf(xh[c])), fmaxf(fabsf(yl[c]), fabsf(yh[c]))));
    }
    const float tp = widen3(tau);
    const float reach = fp64_reach(dmax * 1.001f, 2.0f * cmax * 1.001f, tau);
    bool ov = true;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float need = (tp * ((xh[c] - xl[c]) + (yh[c] - yl[c])) + reach) * 1.001f;
        ov &= !(yl[c] - xh[c] > need || xl[c] - yh[c] > need);
    }
    return ov;
}

// true when the verified FP32 solve proves margin < -2 tau (not a hit)
__device__ __noinline__ bool fp32_verified_reject(const float4 X[3][2], const float4 Y[3][2],
                                                  float tau) {
    const float u = 5.9604645e-08f;
    float A[4][4], EA[4][4], r[4], Er[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        A[c][0] = split_diff(comp(X[0][0], c), comp(X[0][1], c), comp(X[1][0], c), comp(X[1][1], c), EA[c][0]);
        A[c][1] = split_diff(comp(X[2][0], c), comp(X[2][1], c), comp(X[1][0], c), comp(X[1][1], c), EA[c][1]);
        A[c][2] = split_diff(comp(Y[1][0], c), comp(Y[1][1], c), comp(Y[0][0], c), comp(Y[0][1], c), EA[c][2]);
        A[c][3] = split_diff(comp(Y[1][0], c), comp(Y[1][1], c), comp(Y[2][0], c), comp(Y[2][1], c), EA[c][3]);
        r[c] = split_diff(comp(Y[1][0], c), comp(Y[1][1], c), comp(X[1][0], c), comp(X[1][1], c), Er[c]);
    }
    // Gaussian elimination with partial pivoting on [A | I | r]
    float M[4][9];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) { M[i][j] = A[i][j]; M[i][4 + j] = (i == j) ? 1.0f : 0.0f; }
        M[i][8] = r[i];
    }
#pragma unroll
    for (int col = 0; col < 4; ++col) {
        int p = col;
        float best = fabsf(M[col][col]);
#pragma unroll
        for (int row = col + 1; row < 4; ++row) {
            float v = fabsf(M[row][col]);
            if (v > best) { best = v; p = row; }
        }
        if (!(best > 0.0f)) return false;
#pragma unroll
        for (int row = col + 1; row < 4; ++row) {
            const bool sw = (p == row);
#pragma unroll
            for (int j = col; j < 9; ++j) {
                const float lo = M[col][j], hi = M[row][j];
                M[col][j] = sw ? hi : lo;
                M[row][j] = sw ? lo : hi;
            }
        }
        const float inv = 1.0f / M[col][col];
#pragma unroll
        for (int row = col + 1; row < 4; ++row) {
            const float f = M[row][col] * inv;
#pragma unroll
            for (int j = col + 1; j < 9; ++j) M[row][j] = fmaf(-f, M[col][j], M[row][j]);
        }
        M[col][col] = inv;   // keep the reciprocal pivot for the back substitution
    }
    // back substitution for the 5 right-hand sides: columns 4..7 give C, 8 gives z
    float C[4][4], z[4];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        float x[4];
#pragma unroll
        for (int row = 3; row >= 0; --row) {
            float acc = M[row][4 + k];
#pragma unroll
            for (int j = row + 1; j < 4; ++j) acc = fmaf(-M[row][j], x[j], acc);
            x[row] = acc * M[row][row];
        }
#pragma unroll
        for (int row = 0; row < 4; ++row) {
            if (k < 4) C[row][k] = x[row];
            else z[row] = x[row];
        }
    }
    // alpha >= |I - C A_exact|_inf: computed I - C A, its rounding (6u (1 + |C||A|))
    // and the input error |C| EA, the last two as one product |C| W with
    // W = 6u |A| + EA
    float W[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) W[k][j] = fmaf(6.0f * u, fabsf(A[k][j]), EA[k][j]);
    float alpha = 0.0f, cnorm = 0.0f, anorm = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float row = 0.0f, crow = 0.0f, arow = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float e = (i == j) ? 1.0f : 0.0f, cw = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                e = fmaf(-C[i][k], A[k][j], e);
                cw = fmaf(fabsf(C[i][k]), W[k][j], cw);
            }
            row += fabsf(e) + 6.0f * u * ((i == j) ? 1.0f : 0.0f) + cw;
            crow += fabsf(C[i][j]);
            arow += fabsf(A[i][j]);
        }
        alpha = fmaxf(alpha, row);
        cnorm = fmaxf(cnorm, crow);
        anorm = fmaxf(anorm, arow);
    }
    alpha *= 1.0001f;
    if (!(alpha < 0.5f)) return false;
    // |r_exact - A_exact z~| componentwise
    float res[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float acc = r[i], mag = fabsf(r[i]), pert = Er[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc = fmaf(-A[i][j], z[j], acc);
            mag = fmaf(fabsf(A[i][j]), fabsf(z[j]), mag);
            pert = fmaf(EA[i][j], fabsf(z[j]), pert);
        }
        res[i] = (fabsf(acc) + 6.0f * u * mag + pert) * 1.0001f;
    }
    float err = 0.0f, zmax = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float d = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) d = fmaf(fabsf(C[i][j]), res[j], d);
        err = fmaxf(err, d);
        zmax = fmaxf(zmax, fabsf(z[i]));
    }
    err = err / (1.0f - alpha) * 1.001f;
    const float slack = 4.0f * u;
    float m = fminf(fminf(z[0], z[1]), fminf(z[2], z[3])) + err;
    m = fminf(m, 1.0f - z[0] - z[1] + 2.0f * err + slack * (1.0f + fabsf(z[0]) + fabsf(z[1])));
    m = fminf(m, 1.0f - z[2] - z[3] + 2.0f * err + slack * (1.0f + fabsf(z[2]) + fabsf(z[3])));
    // allowance for an FP64 solve of the same system (its own rounding)
    const float kappa = cnorm * anorm;
    const float allow = 2.0f * tau + 32.0f * 1.1102230e-16f * kappa * (1.0f + zmax);
    return isfinite(m) && isfinite(err) && (m < -allow);
}

// ---------------------------------------------------------------------------
// Separating-axis prefilter: a certificate of non-intersection cheaper than the
// verified solve, which it precedes.
//
// Lemma.  For any direction w let I_X = [min_i w.x_i, max_i w.x_i] (length D_X)
// and I_Y likewise.  A point of a triangle widened to weights >= -t projects
// within 3 t D_X of I_X (weights w_i = (1 + 3t) l_i - t with l on the simplex).
// If the FP64 solve reports a hit, its weights are >= -tau' and the two points
// it describes lie within fp64_reach of each other (backward error, below), so
// a gap g > 3 tau' (D_X + D_Y) + |w|_1 reach between I_X and I_Y proves that
// it reports none -- with no condition on the system, so near-parallel
// triangle planes are cleared too.
// Directions: for each triangle the two longest of the four vectors orthogonal
// to its plane (the duals of e1 ^ e2 ^ axis_k, read off the plane's Plucker
// coordinates m_ij = e1_i e2_j - e1_j e2_i); any direction is valid, these
// make the triangle's own interval almost a point.  det A is the pairing of
// the two planes' Plucker coordinates.  Every FP32 value carries a bound on its
// rounding and on the error of the split inputs, so the test is rigorous for
// the FP64 vertices.
// ---------------------------------------------------------------------------
struct SplitVec {
    float v[4];
    float E;       // |v_c - exact_c| <= E for every c
    float M;       // max_c |v_c|
};

// p - q of split vertices: t1 = hp - hq, t2 = lp - lq, v = t1 + t2 with
// |v - exact| <= 2u(1+u)|t1| + 3u^2 (|hp| + |hq|) (the split remainders and the
// three roundings; |t2| <= u (1+u)^2 (|hp| + |hq|)), evaluated with margin
__device__ __forceinline__ SplitVec split_vec(const float4 P[2], const float4 Q[2]) {
    const float u = 5.9604645e-08f;
    SplitVec r;
    float t1m = 0.0f, hm = 0.0f, vm = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float hp = comp(P[0], c), lp = comp(P[1], c), hq = comp(Q[0], c), lq = comp(Q[1], c);
        const float t1 = hp - hq, t2 = lp - lq;
        r.v[c] = t1 + t2;
        t1m = fmaxf(t1m, fabsf(t1));
        hm = fmaxf(hm, fabsf(hp) + fabsf(hq));
        vm = fmaxf(vm, fabsf(r.v[c]));
    }
    r.E = (2.001f * u) * t1m + (3.01f * u * u) * hm + 2e-29f;
    r.M = vm;
    return r;
}

// p - q from the FP32 roundings hp = RN32(p), hq = RN32(q) alone: p = hp + dp
// with |dp| <= u |hp| + 2^-150 (subnormal spacing), so t = fl(hp - hq) has
// |t - (p - q)| <= u |t| / (1 - u) + u (|hp| + |hq|) + 2^-149, bounded with margin.
// Looser than split_vec by about |hp| / |p - q|, which the quad-level test
// absorbs except for near-misses far below a face's size.
__device__ __forceinline__ SplitVec hi_vec(const float4 &P, const float4 &Q) {
    const float u = 5.9604645e-08f;
    SplitVec r;
    float tm = 0.0f, hm = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float hp = comp(P, c), hq = comp(Q, c);
        const float t = hp - hq;
        r.v[c] = t;
        tm = fmaxf(tm, fabsf(t));
        hm = fmaxf(hm, fabsf(hp) + fabsf(hq));
    }
    r.E = ((1.001f * u) * tm + (1.001f * u) * hm) * 1.001f + 3e-45f;
    r.M = tm;
    return r;
}

// a + b of two vectors with bounds
__device__ __forceinline__ SplitVec add_vec(const SplitVec &a, const SplitVec &b) {
    const float u = 5.9604645e-08f;
    SplitVec r;
    float vm = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        r.v[c] = a.v[c] + b.v[c];
        vm = fmaxf(vm, fabsf(r.v[c]));
    }
    r.E = (a.E + b.E + u * vm) * 1.001f;
    r.M = vm;
    return r;
}

// Plucker coordinates (01, 02, 03, 12, 13, 23) of the plane of u and v, and one
// bound on the error of every coordinate
__device__ __forceinline__ void plucker(const SplitVec &a, const SplitVec &b, float m[6], float &eps) {
    const float u = 5.9604645e-08f;
    const int I[6] = {0, 0, 0, 1, 1, 2}, J[6] = {1, 2, 3, 2, 3, 3};
#pragma unroll
    for (int k = 0; k < 6; ++k) m[k] = fmaf(a.v[I[k]], b.v[J[k]], -(a.v[J[k]] * b.v[I[k]]));
    eps = ((4.02f * u) * a.M * b.M + 2.0f * (a.E * b.M + b.E * a.M + a.E * b.E)) * 1.001f;
}

// the dual direction k (orthogonal to the plane and to axis k) from its
// Plucker coordinates m = (01, 02, 03, 12, 13, 23)
__device__ __forceinline__ void dual_dir(const float m[6], int k, float w[4]) {
    w[0] = k == 0 ? 0.0f : (k == 1 ? -m[5] : (k == 2 ? m[4] : -m[3]));
    w[1] = k == 1 ? 0.0f : (k == 0 ? m[5] : (k == 2 ? -m[2] : m[1]));
    w[2] = k == 2 ? 0.0f : (k == 0 ? -m[4] : (k == 1 ? m[2] : -m[0]));
    w[3] = k == 3 ? 0.0f : (k == 0 ? m[3] : (k == 1 ? -m[1] : m[0]));
}

// indices of the two longest duals
__device__ __forceinline__ void top2_duals(const float m[6], int &k1, int &k2) {
    const float s01 = m[0] * m[0], s02 = m[1] * m[1], s03 = m[2] * m[2];
    const float s12 = m[3] * m[3], s13 = m[4] * m[4], s23 = m[5] * m[5];
    const float n[4] = {s12 + s13 + s23, s02 + s03 + s23, s01 + s03 + s13, s01 + s02 + s12};
    k1 = 0;
#pragma unroll
    for (int k = 1; k < 4; ++k) k1 = n[k] > n[k1] ? k : k1;
    k2 = k1 == 0 ? 1 : 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) k2 = (k != k1 && n[k] > n[k2]) ? k : k2;
}

__device__ __forceinline__ float dot4(const float w[4], const SplitVec &v) {
    return fmaf(w[3], v.v[3], fmaf(w[2], v.v[2], fmaf(w[1], v.v[1], w[0] * v.v[0])));
}

// fp64_reach and widen3 (the FP64 solve's backward error and the widening of
// a triangle's projection) are in tms_common.cuh: the patch-pair test uses them too.

// the gap test along w for X = {0, e1, e2} and Y = {r, s1, s3} (all relative to x2):
// the widened projections apart by more than |w|_1 reach
__device__ __forceinline__ bool separated(const float w[4], const SplitVec &e1, const SplitVec &e2,
                                          const SplitVec &r, const SplitVec &s1, const SplitVec &s3,
                                          float tp, float reach) {
    const float u = 5.9604645e-08f;
    const float w1 = fabsf(w[0]) + fabsf(w[1]) + fabsf(w[2]) + fabsf(w[3]);
    // |fl(w.v) - w.v_exact| <= |w|_1 (4.01 u M_v + E_v)
    const float a1 = dot4(w, e1), a3 = dot4(w, e2);
    const float b2 = dot4(w, r), b1 = dot4(w, s1), b3 = dot4(w, s3);
    const float ex = w1 * fmaxf(fmaf(4.01f * u, e1.M, e1.E), fmaf(4.01f * u, e2.M, e2.E));
    const float ey = w1 * fmaxf(fmaxf(fmaf(4.01f * u, r.M, r.E), fmaf(4.01f * u, s1.M, s1.E)),
                                fmaf(4.01f * u, s3.M, s3.E));
    const float xl = fminf(0.0f, fminf(a1, a3)), xh = fmaxf(0.0f, fmaxf(a1, a3));
    const float yl = fminf(b2, fminf(b1, b3)), yh = fmaxf(b2, fmaxf(b1, b3));
    const float DX = (xh - xl) + 2.0f * ex, DY = (yh - yl) + 2.0f * ey;
    const float need = (tp * (DX + DY) + w1 * reach + ex + ey) * 1.001f;
    const float gap = fmaxf(yl - xh, xl - yh) * (1.0f - 4.0f * u);
    return gap > need;
}

// Quad-level form of the separating-axis test: true when no one of the four
// triangle pairs of the quad candidate can be an FP64 hit (fp64_reach).  A
// triangle's vertices are among its quad's, so its projected interval lies
// inside the quad's, and its widening (3 tau' times its length) is at most the
// quad's.  Axes: the two longest duals of each quad's first triangle.  Every
// triangle's edges are differences of the quad's vertices (|A_ij| <= 2 max of
// the edge vectors below), and every offset y2 - x2 is r0 plus at most the
// vectors to each quad's far vertex.
// One axis of the quad-level test: A's vertices at 0, a1, a2, a3 and B's at r0,
// r0 + b1, r0 + b2, r0 + b3 (all relative to A's v0) projected on w, each with
// its rounding and input error; true when the widened intervals are further
// apart than |w|_1 reach.
__device__ __forceinline__ bool quad_gap(const float w[4], const SplitVec &a1, const SplitVec &a2,
                                         const SplitVec &a3, const SplitVec &b1, const SplitVec &b2,
                                         const SplitVec &b3, const SplitVec &r0, float tp, float reach) {
    const float u = 5.9604645e-08f;
    const float w1 = fabsf(w[0]) + fabsf(w[1]) + fabsf(w[2]) + fabsf(w[3]);
    const float p1 = dot4(w, a1), p2 = dot4(w, a2), p3 = dot4(w, a3);
    const float ea = w1 * fmaxf(fmaxf(fmaf(4.01f * u, a1.M, a1.E), fmaf(4.01f * u, a2.M, a2.E)),
                                fmaf(4.01f * u, a3.M, a3.E));
    const float q0 = dot4(w, r0);
    const float s1 = q0 + dot4(w, b1), s2 = q0 + dot4(w, b2), s3 = q0 + dot4(w, b3);
    const float eb = w1 * (fmaf(4.01f * u, r0.M, r0.E) +
                           fmaxf(fmaxf(fmaf(4.01f * u, b1.M, b1.E), fmaf(4.01f * u, b2.M, b2.E)),
                                 fmaf(4.01f * u, b3.M, b3.E))) +
                     u * fmaxf(fmaxf(fabsf(s1), fabsf(s2)), fabsf(s3));
    const float xl = fminf(fminf(0.0f, p1), fminf(p2, p3)), xh = fmaxf(fmaxf(0.0f, p1), fmaxf(p2, p3));
    const float yl = fminf(fminf(q0, s1), fminf(s2, s3)), yh = fmaxf(fmaxf(q0, s1), fmaxf(s2, s3));
    const float DX = (xh - xl) + 2.0f * ea, DY = (yh - yl) + 2.0f * eb;
    const float need = (tp * (DX + DY) + w1 * reach + ea + eb) * 1.001f;
    const float gap = fmaxf(yl - xh, xl - yh) * (1.0f - 4.0f * u);
    return gap > need;
}

// the vector orthogonal to a, b and c in R^4 (cofactor expansion of the 4 x 4
// determinant with rows (x, a, b, c))
__device__ __forceinline__ float det3v(float a0, float a1, float a2, float b0, float b1, float b2,
                                       float c0, float c1, float c2) {
    return a0 * (b1 * c2 - b2 * c1) - a1 * (b0 * c2 - b2 * c0) + a2 * (b0 * c1 - b1 * c0);
}
__device__ __forceinline__ void cross4v(const float a[4], const float b[4], const float c[4], float x[4]) {
    x[0] = det3v(a[1], a[2], a[3], b[1], b[2], b[3], c[1], c[2], c[3]);
    x[1] = -det3v(a[0], a[2], a[3], b[0], b[2], b[3], c[0], c[2], c[3]);
    x[2] = det3v(a[0], a[1], a[3], b[0], b[1], b[3], c[0], c[1], c[3]);
    x[3] = -det3v(a[0], a[1], a[2], b[0], b[1], b[2], c[0], c[1], c[2]);
}

// the quad-level test on the edge vectors of both quads relative to v0 of A
__device__ __forceinline__ bool quad_sat_vectors(const SplitVec &a1, const SplitVec &a2, const SplitVec &a3,
                                                 const SplitVec &b1, const SplitVec &b2, const SplitVec &b3,
                                                 const SplitVec &r0, float tau) {
    float mA1[6], mB1[6], epsA1, epsB1;
    plucker(a1, a2, mA1, epsA1);
    plucker(b1, b2, mB1, epsB1);
    const float amax = 2.0f * fmaxf(fmaxf(fmaxf(a1.M + a1.E, a2.M + a2.E), fmaxf(a3.M + a3.E, b1.M + b1.E)),
                                    fmaxf(b2.M + b2.E, b3.M + b3.E));
    const float rmax = (r0.M + r0.E) + (a3.M + a3.E) + (b3.M + b3.E);
    const float reach = fp64_reach(amax * 1.001f, rmax * 1.001f, tau);
    const float tp = widen3(tau);
    int kA1, kA2, kB1, kB2;
    top2_duals(mA1, kA1, kA2);
    top2_duals(mB1, kB1, kB2);
#pragma unroll 1
    for (int ax = 0; ax < 4; ++ax) {
        float m[6], w[4];
#pragma unroll
        for (int k = 0; k < 6; ++k) m[k] = ax < 2 ? mA1[k] : mB1[k];
        dual_dir(m, ax == 0 ? kA1 : (ax == 1 ? kA2 : (ax == 2 ? kB1 : kB2)), w);
        if (quad_gap(w, a1, a2, a3, b1, b2, b3, r0, tp, reach)) return true;
    }
    return false;
}

// The quad-level test from the quads' FP32 vertex roundings alone (hi_vec
// bounds, half the data of the split copies).  Directions: the mixed ones
// MLO..MHI-1 -- 0: orthogonal to A's first-triangle edges a1, a2 and B's b1,
// 1: to a1, a2, b2, 2: to b1, b2, a1, 3: to b1, b2, a2 (both quads thin along
// each when their planes share a direction) -- then, with DUALS, the dual axes
// of quad_sat_vectors.  Any direction serves (the bounds hold for the FP32 w as
// computed), so w is not normalised.  A candidate it cannot clear goes on to
// the tests on the split copies.
template <int MLO, int MHI, bool DUALS>
__device__ __forceinline__ bool quad_reject_hi(const float4 QA[4], const float4 QB[4], float tau) {
    const SplitVec a1 = hi_vec(QA[1], QA[0]), a2 = hi_vec(QA[2], QA[0]);
    const SplitVec a3 = hi_vec(QA[3], QA[0]);
    const SplitVec b1 = hi_vec(QB[1], QB[0]), b2 = hi_vec(QB[2], QB[0]);
    const SplitVec b3 = hi_vec(QB[3], QB[0]);
    const SplitVec r0 = hi_vec(QB[0], QA[0]);
    const float amax = 2.0f * fmaxf(fmaxf(fmaxf(a1.M + a1.E, a2.M + a2.E), fmaxf(a3.M + a3.E, b1.M + b1.E)),
                                    fmaxf(b2.M + b2.E, b3.M + b3.E));
    const float rmax = (r0.M + r0.E) + (a3.M + a3.E) + (b3.M + b3.E);
    const float reach = fp64_reach(amax * 1.001f, rmax * 1.001f, tau);
    const float tp = widen3(tau);
    float w[4];
    if (MLO <= 0 && 0 < MHI) {
        cross4v(a1.v, a2.v, b1.v, w);
        if (quad_gap(w, a1, a2, a3, b1, b2, b3, r0, tp, reach)) return true;
    }
    if (MLO <= 1 && 1 < MHI) {
        cross4v(a1.v, a2.v, b2.v, w);
        if (quad_gap(w, a1, a2, a3, b1, b2, b3, r0, tp, reach)) return true;
    }
    if (MLO <= 2 && 2 < MHI) {
        cross4v(b1.v, b2.v, a1.v, w);
        if (quad_gap(w, a1, a2, a3, b1, b2, b3, r0, tp, reach)) return true;
    }
    if (MLO <= 3 && 3 < MHI) {
        cross4v(b1.v, b2.v, a2.v, w);
        if (quad_gap(w, a1, a2, a3, b1, b2, b3, r0, tp, reach)) return true;
    }
    if (DUALS) return quad_sat_vectors(a1, a2, a3, b1, b2, b3, r0, tau);
    return false;
}

// the mixed directions every candidate takes in k_quad_filter's first stage; the
// rest, and the dual axes, only the candidates these leave
constexpr int kQuadFirstAxes = 2;

// true when the separating-axis test proves that the FP64 solve of the pair
// reports no hit (fp64_reach)
__device__ __noinline__ bool fp32_sat_reject(const float4 X[3][2], const float4 Y[3][2],
                                                float tau) {
    // vectors relative to x2
    const SplitVec e1 = split_vec(X[0], X[1]);    // x1 - x2
    const SplitVec e2 = split_vec(X[2], X[1]);    // x3 - x2
    const SplitVec f1 = split_vec(Y[0], Y[1]);    // y1 - y2
    const SplitVec f2 = split_vec(Y[2], Y[1]);    // y3 - y2
    const SplitVec r = split_vec(Y[1], X[1]);     // y2 - x2
    const SplitVec s1 = add_vec(r, f1), s3 = add_vec(r, f2);
    float mE[6], mF[6], epsE, epsF;
    plucker(e1, e2, mE, epsE);
    plucker(f1, f2, mF, epsF);
    const float amax = fmaxf(fmaxf(e1.M + e1.E, e2.M + e2.E), fmaxf(f1.M + f1.E, f2.M + f2.E));
    const float reach = fp64_reach(amax * 1.001f, (r.M + r.E) * 1.001f, tau);
    const float tp = widen3(tau);
    int kE1, kE2, kF1, kF2;
    top2_duals(mE, kE1, kE2);
    top2_duals(mF, kF1, kF2);
    // one loop over the four axes (a small kernel fetches its code faster);
    // the plane of each axis is chosen by selects, not by an indexed array
#pragma unroll 1
    for (int ax = 0; ax < 4; ++ax) {
        float m[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) m[k] = ax < 2 ? mE[k] : mF[k];
        float w[4];
        dual_dir(m, ax == 0 ? kE1 : (ax == 1 ? kE2 : (ax == 2 ? kF1 : kF2)), w);
        if (separated(w, e1, e2, r, s1, s3, tp, reach)) return true;
    }
    return false;
}

// (theta, s) estimate for weights (u, v) in triangle t (formulas after Eq. (precise))
__device__ __forceinline__ void tri_params(const MeshDev &m, uint32_t t, double u, double v,
                                           double &th, double &sv) {
    uint32_t q = t >> 1;
    int tau = t & 1;
    int i = (int)(q % (uint32_t)m.N), k = (int)(q / (uint32_t)m.N);
    double dth = kTwoPi / m.N;
    double th_i = i * dth, th_ip = th_i + dth;
    double s_k = m.s[k], s_kp = m.s[k + 1];
    if (tau == 0) {
        th = (1.0 - u) * th_i + u * th_ip;
        sv = (1.0 - v) * s_k + v * s_kp;
    } else {
        th = u * th_i + (1.0 - u) * th_ip;
        sv = v * s_k + (1.0 - v) * s_kp;
    }
    th = fmod(th, kTwoPi);
    if (th < 0) th += kTwoPi;
}

// FP64 narrow-phase test of one triangle pair (Eq. (precise)); fills h on a hit
__device__ __forceinline__ bool narrow_fp64(const MeshDev &ma, const MeshDev &mb, uint32_t ta,
                                            uint32_t tb, double tau, tms_hit &h) {
    double x[3][4], y[3][4];
    gather_tri(ma, ta, x);
    gather_tri(mb, tb, y);
    double A[4][4], r[4], col0[4], col1[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        A[c][0] = x[0][c] - x[1][c];
        A[c][1] = x[2][c] - x[1][c];
        A[c][2] = y[1][c] - y[0][c];
        A[c][3] = y[1][c] - y[2][c];
        r[c] = y[1][c] - x[1][c];
        col0[c] = A[c][0];
        col1[c] = A[c][1];
    }
    double n2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) n2[j] = A[0][j] * A[0][j] + A[1][j] * A[1][j] + A[2][j] * A[2][j] + A[3][j] * A[3][j];
    double z[4], det;
    const bool ok = solve4_gepp<double>(A, r, z, det);
    if (!ok) return false;
    const double a = z[0], b = z[1], c = z[2], d = z[3];
    const double m = fmin(fmin(fmin(a, b), fmin(c, d)), fmin(1.0 - a - b, 1.0 - c - d));
    const bool finite = isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d);
    if (!(finite && m >= -tau)) return false;
    const double rho = fabs(det) / (sqrt(n2[0]) * sqrt(n2[1]) * sqrt(n2[2]) * sqrt(n2[3]));
    if (!(rho > 0.0)) return false;
    h.triA = ta;
    h.triB = tb;
    h.a = a; h.b = b; h.c = c; h.d = d;
#pragma unroll
    for (int k = 0; k < 4; ++k) h.P[k] = x[1][k] + a * col0[k] + b * col1[k];
    tri_params(ma, ta, a, b, h.theta_u, h.s_u);
    tri_params(mb, tb, c, d, h.theta_s, h.s_s);
    h.rho = rho;
    h.margin = m;
    h.flags = (rho < 1e-12 || fabs(m) < 1e-12) ? 1u : 0u;
    return true;
}

// Stage 1b: the triangle pairs the quad-level test (k_quad_filter) leaves, one
// per lane (with face_level 0, every triangle candidate): the (widened)
// triangle boxes, the triangle-level separating-axis test, and for the pairs
// left a per-warp queue feeding the verified solve 32 pairs at a time, so that
// the solve does not run with most lanes idle; pairs the tests cannot reject go
// to the survivor list.  With the FP32 filters off, every triangle pair of
// every candidate goes to the survivor list.
template <int FACE>
__global__ void __launch_bounds__(256, 2) k_narrow_filter(NarrowArgs a) {
    constexpr int kW = 8, kQ = 32 + 4 * 32;
    __shared__ uint32_t q_cand[kW][kQ];          // triangle pairs for the verified solve
    __shared__ uint8_t q_sub[kW][kQ];
    if (a.ctr->cand > a.cand_cap) return;
    const unsigned long long n = a.ctr->cand;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    // tau rounded up once per thread: the FP32 tests only widen by it
    const float tauf = __double2float_ru(a.tau);
    unsigned long long n_sat = 0, n_full = 0;               // tests run, per warp
    unsigned qn = 0;                                        // queued pairs (warp-uniform)

    // the verified solve of pair-queue items [base, base + cnt)
    auto drain = [&](unsigned base, unsigned cnt) {
        bool keep = false;
        uint32_t ta = 0, tb = 0, pair = 0;
        if ((unsigned)lane < cnt) {
            const uint32_t g = q_cand[warp][base + lane];
            const unsigned sub = q_sub[warp][base + lane];
            const Cand c2 = a.cand[g];
            ta = FACE == 0 ? c2.faceA : 2 * c2.faceA + (sub & 1u);
            tb = FACE == 0 ? c2.faceB : 2 * c2.faceB + (sub >> 1);
            pair = c2.pair;
            const int2 pr = a.pairs[pair];
            float4 X[3][2], Y[3][2];
            gather_split(a.meshes[pr.x], ta, X);
            gather_split(a.meshes[pr.y], tb, Y);
            keep = !fp32_verified_reject(X, Y, tauf);
        }
        n_full += cnt;
        const unsigned long long pos = warp_append(&a.ctr->fp64, keep, FULL);
        if (keep && pos < a.surv_cap) {
            Cand sv;
            sv.faceA = ta;
            sv.faceB = tb;
            sv.pair = pair;
            sv.pad = 0;
            a.surv[pos] = sv;
        }
    };
    // one triangle pair through the box and separating-axis tests; the pairs
    // they cannot reject join the pair queue (all lanes call it together)
    auto pair_tests = [&](bool valid, uint32_t g, int sub, const float4 X[3][2], const float4 Y[3][2],
                          bool boxes) {
        const bool tested = valid && (!boxes || split_boxes_overlap(X, Y, tauf));
        const bool need = tested && !fp32_sat_reject(X, Y, tauf);
        n_sat += __popc(__ballot_sync(FULL, tested));
        const uint32_t want = __ballot_sync(FULL, need);
        if (need) {
            const unsigned slot = qn + __popc(want & lt);
            q_cand[warp][slot] = g;
            q_sub[warp][slot] = (uint8_t)sub;
        }
        qn += __popc(want);
    };
    auto drain_full = [&]() {
        __syncwarp();
        while (qn >= 32) {
            qn -= 32;
            drain(qn, 32);
            __syncwarp();
        }
    };
    if (FACE == 1 && a.fp32_filter) {
        // the candidates the quad-level test (k_quad_filter) could not clear: each
        // of their four triangle pairs on a lane of its own (triangle boxes, the
        // triangle-level separating axes), the pairs left queued for the
        // verified solve, 32 at a time
        const unsigned long long ni = 4 * clamp_count(&a.ctr->qkeep, a.cand_cap);
        for (unsigned long long i0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x - lane; i0 < ni;
             i0 += stride) {
            const unsigned long long it = i0 + lane;
            const bool valid = it < ni;
            uint32_t g = 0;
            const int sub = (int)(it & 3);
            float4 X[3][2], Y[3][2];
            if (valid) {
                g = a.qsurv[it >> 2];
                const Cand cd = a.cand[g];
                const int2 pr = a.pairs[cd.pair];
                gather_split(a.meshes[pr.x], 2 * cd.faceA + (sub & 1), X);
                gather_split(a.meshes[pr.y], 2 * cd.faceB + (sub >> 1), Y);
            }
            pair_tests(valid, g, sub, X, Y, true);
            drain_full();
        }
        if (qn) {
            drain(0, qn);
            __syncwarp();
        }
        if (lane == 0) {
            if (n_sat) atomicAdd(&a.ctr->sat, n_sat);
            if (n_full) atomicAdd(&a.ctr->fp32, n_full);
        }
        return;
    }
    for (unsigned long long g0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x - lane;
         g0 < n; g0 += stride) {
        const unsigned long long g = g0 + lane;
        const bool valid = g < n;
        Cand cd;
        cd.faceA = cd.faceB = cd.pair = 0;
        if (valid) cd = a.cand[g];
        if (!a.fp32_filter) {
            // every triangle pair of the candidate to the FP64 solve
            const int nsub = FACE == 0 ? 1 : 4;
            for (int sub = 0; sub < nsub; ++sub) {
                const uint32_t ta = FACE == 0 ? cd.faceA : 2 * cd.faceA + (sub & 1);
                const uint32_t tb = FACE == 0 ? cd.faceB : 2 * cd.faceB + (sub >> 1);
                const unsigned long long pos = warp_append(&a.ctr->fp64, valid, FULL);
                if (valid && pos < a.surv_cap) {
                    Cand sv;
                    sv.faceA = ta;
                    sv.faceB = tb;
                    sv.pair = cd.pair;
                    sv.pad = 0;
                    a.surv[pos] = sv;
                }
            }
            continue;
        }
        const int2 pr = a.pairs[valid ? cd.pair : 0];
        if (FACE == 0) {
            float4 X[3][2], Y[3][2];
            if (valid) {
                gather_split(a.meshes[pr.x], cd.faceA, X);
                gather_split(a.meshes[pr.y], cd.faceB, Y);
            }
            pair_tests(valid, (uint32_t)g, 0, X, Y, false);
            drain_full();
        }
    }
    if (qn) {
        drain(0, qn);
        __syncwarp();
    }
    if (lane == 0) {
        if (n_sat) atomicAdd(&a.ctr->sat, n_sat);
        if (n_full) atomicAdd(&a.ctr->fp32, n_full);
    }
}

// Stage 1a (quad faces): the quad-level separating-axis test of every candidate
// on the FP32 roundings of its quads' vertices, the first mixed directions
// first; the candidates they leave gather in a per-warp queue, and every 32 of
// them take the other directions with all lanes busy; those still not cleared
// are listed for the per-pair path of k_narrow_filter.
constexpr int kQuadWarps = 8;
__global__ void __launch_bounds__(32 * kQuadWarps, 3) k_quad_filter(NarrowArgs a) {
    __shared__ uint32_t s_q[kQuadWarps][64];
    if (a.ctr->cand > a.cand_cap) return;
    const unsigned long long n = a.ctr->cand;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();
    const float tauf = __double2float_ru(a.tau);
    unsigned long long n_quad = 0;
    unsigned qn = 0;                                 // queued candidates (warp-uniform)
    // the mixed directions for queue items [base, base + cnt)
    auto drain = [&](unsigned base, unsigned cnt) {
        bool keep = false;
        uint32_t g = 0;
        if ((unsigned)lane < cnt) {
            g = s_q[warp][base + lane];
            const Cand cd = a.cand[g];
            const int2 pr = a.pairs[cd.pair];
            float4 QA[4], QB[4];
            gather_quad_hi(a.meshes[pr.x], cd.faceA, QA);
            gather_quad_hi(a.meshes[pr.y], cd.faceB, QB);
            keep = !quad_reject_hi<kQuadFirstAxes, 4, true>(QA, QB, tauf);
        }
        const unsigned long long pos = warp_append(&a.ctr->qkeep, keep, FULL);
        if (keep && pos < a.cand_cap) a.qsurv[pos] = g;
    };
    for (unsigned long long g0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x - lane;
         g0 < n; g0 += stride) {
        const unsigned long long g = g0 + lane;
        const bool valid = g < n;
        bool need = false;
        if (valid) {
            const Cand cd = a.cand[g];
            const int2 pr = a.pairs[cd.pair];
            float4 QA[4], QB[4];
            gather_quad_hi(a.meshes[pr.x], cd.faceA, QA);
            gather_quad_hi(a.meshes[pr.y], cd.faceB, QB);
            need = !quad_reject_hi<0, kQuadFirstAxes, false>(QA, QB, tauf);
        }
        n_quad += __popc(__ballot_sync(FULL, valid));
        const uint32_t want = __ballot_sync(FULL, need);
        if (need) s_q[warp][qn + __popc(want & lt)] = (uint32_t)g;
        qn += __popc(want);
        __syncwarp();
        if (qn >= 32) {
            qn -= 32;
            drain(qn, 32);
            __syncwarp();
        }
    }
    if (qn) {
        drain(0, qn);
        __syncwarp();
    }
    if (lane == 0 && n_quad) atomicAdd(&a.ctr->quad, n_quad);
}

// Stage 2: the FP64 solve for the survivors
__global__ void __launch_bounds__(256) k_narrow_fp64(NarrowArgs a) {
    if (a.ctr->cand > a.cand_cap || a.ctr->fp64 > a.surv_cap) return;
    const unsigned long long n = a.ctr->fp64;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (unsigned long long g0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x - lane;
         g0 < n; g0 += stride) {
        const unsigned long long g = g0 + lane;
        bool hit = false;
        tms_hit h;
        Cand s;
        s.faceA = s.faceB = s.pair = 0;
        if (g < n) {
            s = a.surv[g];
            const int2 pr = a.pairs[s.pair];
            hit = narrow_fp64(a.meshes[pr.x], a.meshes[pr.y], s.faceA, s.faceB, a.tau, h);
        }
        const unsigned long long pos = warp_append(&a.ctr->raw_hits, hit, FULL);
        if (hit && pos < a.hit_cap) {
            h.pair = s.pair;
            a.hits[pos] = h;
            a.hit_key[pos] = ((uint64_t)s.pair << (2 * a.tri_bits)) |
                             ((uint64_t)s.faceA << a.tri_bits) | (uint64_t)s.faceB;
            a.hit_val[pos] = (uint32_t)pos;
        }
    }
}

// ---------------------------------------------------------------------------
// merging of duplicate hits (shared edges and vertices)
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool quad_ok(const MeshDev &m, int i, int k) {
    if (k < 0 || k >= m.nqk) return false;
    if (m.periodic) return true;
    return i >= 0 && i < m.nqi;
}
__device__ __forceinline__ int wrap_i(const MeshDev &m, int i) {
    if (!m.periodic) return i;
    return (i % m.N + m.N) % m.N;
}
__device__ __forceinline__ void add_tri(const MeshDev &m, int i, int k, int tau, uint32_t *inc,
                                        int &n) {
    int iw = wrap_i(m, i);
    if (quad_ok(m, iw, k)) inc[n++] = 2u * ((uint32_t)k * (uint32_t)m.N + (uint32_t)iw) + (uint32_t)tau;
}

// Feature of the point with weights (u, v) in triangle t, and the triangles
// incident to that feature.  Weights (w1, w2, w3) = (u, 1-u-v, v) on
// (x1, x2, x3); one weight below tau: the opposite edge; two: the vertex left.
// Codes: (0 << 30) | t, (1 << 30) | (3 * base_vertex + edge_type), (2 << 30) | vertex.
__device__ uint32_t feature_of(const MeshDev &m, uint32_t t, double u, double v, double tau,
                               uint32_t inc[6], int &ninc) {
    const double w[3] = {u, 1.0 - u - v, v};
    const bool s0 = fabs(w[0]) < tau, s1 = fabs(w[1]) < tau, s2 = fabs(w[2]) < tau;
    const int ns = (int)s0 + (int)s1 + (int)s2;
    ninc = 0;
    if (ns == 0) {
        inc[ninc++] = t;
        return t;
    }
    const uint32_t q = t >> 1;
    const int tau_t = t & 1;
    const int i = (int)(q % (uint32_t)m.N), k = (int)(q / (uint32_t)m.N);
    const int ip = (i + 1 == m.N) ? 0 : i + 1;
    if (ns == 1) {
        // edge opposite the small weight: 0 -> (x2,x3), 1 -> (x1,x3), 2 -> (x1,x2)
        const int opp = s0 ? 0 : (s1 ? 1 : 2);
        int bi, bk, type;
        if (opp == 1) { bi = i; bk = k; type = 2; }                      // diagonal of quad (i,k)
        else if (tau_t == 0) {
            if (opp == 2) { bi = i; bk = k; type = 0; }                 // T1 (x1,x2): theta edge at (i,k)
            else { bi = i; bk = k; type = 1; }                          // T1 (x2,x3): s edge at (i,k)
        } else {
            if (opp == 2) { bi = i; bk = k + 1; type = 0; }             // T2 (x1,x2): theta edge at (i,k+1)
            else { bi = ip; bk = k; type = 1; }                         // T2 (x2,x3): s edge at (i+1,k)
        }
        if (type == 0) { add_tri(m, bi, bk, 0, inc, ninc); add_tri(m, bi, bk - 1, 1, inc, ninc); }
        else if (type == 1) { add_tri(m, bi, bk, 0, inc, ninc); add_tri(m, bi - 1, bk, 1, inc, ninc); }
        else { add_tri(m, bi, bk, 0, inc, ninc); add_tri(m, bi, bk, 1, inc, ninc); }
        return (1u << 30) | (3u * ((uint32_t)bk * (uint32_t)m.N + (uint32_t)bi) + (uint32_t)type);
    }
    int j;
    if (ns == 2) j = !s0 ? 0 : (!s1 ? 1 : 2);
    else { j = 0; if (w[1] > w[j]) j = 1; if (w[2] > w[j]) j = 2; }
    int ii[3], kk[3];
    tri_ij(m, t, ii, kk);
    const int vi = ii[j], vk = kk[j];
    add_tri(m, vi, vk, 0, inc, ninc);
    add_tri(m, vi - 1, vk, 0, inc, ninc);
    add_tri(m, vi, vk - 1, 0, inc, ninc);
    add_tri(m, vi, vk - 1, 1, inc, ninc);
    add_tri(m, vi - 1, vk - 1, 1, inc, ninc);
    add_tri(m, vi - 1, vk, 1, inc, ninc);
    return (2u << 30) | ((uint32_t)vk * (uint32_t)m.N + (uint32_t)vi);
}

__global__ void k_dedup_flags(DedupArgs a) {
    const unsigned long long n = clamp_count(&a.ctr->raw_hits, a.raw_cap);
    // a sort whose look-back gave up leaves its output unordered and its value
    // slots possibly unwritten: keep nothing, and index nothing with them
    const bool sorted = (a.ctr->status & ST_TIMEOUT) == 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        if (!sorted) {
            a.keep[i] = 0;
            continue;
        }
        const uint64_t key = a.keys[i];
        const tms_hit &h = a.raw[a.vals[i]];
        const int2 pr = a.pairs[h.pair];
        const MeshDev ma = a.meshes[pr.x], mb = a.meshes[pr.y];
        uint32_t incA[6], incB[6];
        int nA, nB;
        const uint32_t fA = feature_of(ma, h.triA, h.a, h.b, a.tau, incA, nA);
        const uint32_t fB = feature_of(mb, h.triB, h.c, h.d, a.tau, incB, nB);
        uint32_t keep = 1;
        if ((fA >> 30) != 0 || (fB >> 30) != 0) {
            for (int p = 0; p < nA && keep; ++p) {
                for (int q = 0; q < nB && keep; ++q) {
                    const uint32_t ta = incA[p], tb = incB[q];
                    if (ta == h.triA && tb == h.triB) continue;
                    const uint64_t k2 = ((uint64_t)h.pair << (2 * a.tri_bits)) |
                                        ((uint64_t)ta << a.tri_bits) | (uint64_t)tb;
                    if (k2 >= key) continue;
                    unsigned long long lo = 0, hi = i;
                    while (lo < hi) {
                        unsigned long long mid = (lo + hi) >> 1;
                        if (a.keys[mid] < k2) lo = mid + 1; else hi = mid;
                    }
                    if (lo < i && a.keys[lo] == k2) {
                        const tms_hit &o = a.raw[a.vals[lo]];
                        uint32_t t1[6], t2[6];
                        int n1, n2;
                        const uint32_t gA = feature_of(ma, o.triA, o.a, o.b, a.tau, t1, n1);
                        const uint32_t gB = feature_of(mb, o.triB, o.c, o.d, a.tau, t2, n2);
                        if (gA == fA && gB == fB) keep = 0;
                    }
                }
            }
        }
        a.keep[i] = keep;
    }
}

__global__ void k_dedup_out(DedupArgs a) {
    const unsigned long long n = clamp_count(&a.ctr->raw_hits, a.raw_cap);
    if (a.ctr->status & ST_TIMEOUT) return;   // nothing was kept (k_dedup_flags)
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        if (!a.keep[i]) continue;
        const unsigned long long pos = a.keep_scan[i];
        tms_hit h = a.raw[a.vals[i]];
        const int2 pr = a.pairs[h.pair];
        uint32_t inc[6];
        int ninc;
        const uint32_t fA = feature_of(a.meshes[pr.x], h.triA, h.a, h.b, a.tau, inc, ninc);
        const uint32_t fB = feature_of(a.meshes[pr.y], h.triB, h.c, h.d, a.tau, inc, ninc);
        if ((fA >> 30) != 0 || (fB >> 30) != 0) h.flags |= 2u;
        a.out_keys[pos] = a.keys[i];
        if (pos < a.out_cap) a.out[pos] = h;
    }
}

__global__ void k_offsets(const uint64_t *out_keys, const unsigned long long *d_out,
                          unsigned long long raw_cap, int n_pairs, int tri_bits, long long *offsets) {
    const unsigned long long n = clamp_count(d_out, raw_cap);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p <= n_pairs; p += gridDim.x * blockDim.x) {
        if (p == n_pairs) { offsets[p] = (long long)n; continue; }
        const uint64_t k = (uint64_t)p << (2 * tri_bits);
        unsigned long long lo = 0, hi = n;
        while (lo < hi) {
            unsigned long long mid = (lo + hi) >> 1;
            if (out_keys[mid] < k) lo = mid + 1; else hi = mid;
        }
        offsets[p] = (long long)lo;
    }
}

// ---------------------------------------------------------------------------
// adjoint of the hit outputs
// ---------------------------------------------------------------------------
__global__ void k_adjoint(AdjointArgs a) {
    for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < a.n;
         h += (long long)gridDim.x * blockDim.x) {
        const tms_hit hit = a.hits[h];
        double x[3][4], y[3][4];
        gather_tri(a.A, hit.triA, x);
        gather_tri(a.B, hit.triB, y);
        double M[4][4], Mt[4][4], r[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            M[c][0] = x[0][c] - x[1][c];
            M[c][1] = x[2][c] - x[1][c];
            M[c][2] = y[1][c] - y[0][c];
            M[c][3] = y[1][c] - y[2][c];
            r[c] = y[1][c] - x[1][c];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) Mt[i][j] = M[j][i];
        double gP[4] = {0, 0, 0, 0}, zbar[4] = {0, 0, 0, 0};
        if (a.gP) for (int c = 0; c < 4; ++c) gP[c] = a.gP[4 * h + c];
        if (a.gZ) for (int c = 0; c < 4; ++c) zbar[c] = a.gZ[4 * h + c];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            zbar[0] += M[c][0] * gP[c];
            zbar[1] += M[c][1] * gP[c];
        }
        double z[4], det, w[4], det2;
        const bool ok1 = solve4_gepp<double>(M, r, z, det);
        const bool ok2 = solve4_gepp<double>(Mt, zbar, w, det2);
        if (!(ok1 && ok2)) {
            if (a.galpha) a.galpha[h] = 0.0;
            continue;
        }
        const double beta[3] = {z[0], 1.0 - z[0] - z[1], z[1]};
        const double gam[3] = {z[2], 1.0 - z[2] - z[3], z[3]};
        int iA[3], kA[3], iB[3], kB[3];
        tri_ij(a.A, hit.triA, iA, kA);
        tri_ij(a.B, hit.triB, iB, kB);
        double ga = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const size_t oa = (size_t)kA[j] * a.A.N + iA[j];
            const size_t ob = (size_t)kB[j] * a.B.N + iB[j];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double gx = beta[j] * (gP[c] - w[c]);
                const double gy = gam[j] * w[c];
                if (a.gA[c]) atomicAdd(a.gA[c] + oa, gx);
                if (a.gB[c]) atomicAdd(a.gB[c] + ob, gy);
                if (a.dA[c]) ga += gx * a.dA[c][oa];
                if (a.dB[c]) ga += gy * a.dB[c][ob];
            }
        }
        if (a.galpha) a.galpha[h] = ga;
    }
}

}  // namespace

// The filter runs as one wave of resident blocks: its warps stride over the
// candidates and end by draining part-filled queues with idle lanes, so each
// extra wave adds a round of those tails (4 waves: 0.255 ms, 2: 0.241, 1: 0.232
// on the 4096 x 512 workload).  Resident blocks per SM, the same on every
// GB300, looked up by configure_narrow (outside stream capture) or at the first
// launch.
namespace {
int g_filter_resident[2] = {};

template <int FACE>
int filter_resident() {
    int &r = g_filter_resident[FACE];
    if (r == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_narrow_filter<FACE>, 256, 0) != cudaSuccess ||
            nb < 1)
            nb = 1;
        r = nb;
    }
    return r;
}
}  // namespace

void configure_narrow() {
    filter_resident<0>();
    filter_resident<1>();
}

void launch_narrow(const NarrowArgs &a, int face_level, int sms, int grid, cudaStream_t st) {
    if (face_level == 0) {
        k_narrow_filter<0><<<sms * filter_resident<0>(), 256, 0, st>>>(a);
    } else {
        if (a.fp32_filter) k_quad_filter<<<sms * 3 * 4, 32 * kQuadWarps, 0, st>>>(a);
        k_narrow_filter<1><<<sms * filter_resident<1>(), 256, 0, st>>>(a);
    }
    k_narrow_fp64<<<grid, 256, 0, st>>>(a);
}

void launch_dedup(const DedupArgs &a, int grid, cudaStream_t st) {
    k_dedup_flags<<<grid, 256, 0, st>>>(a);
    scan_u32(a.keep, a.keep_scan, &a.ctr->raw_hits, a.raw_cap, a.partials, &a.ctr->out, grid, st);
    k_dedup_out<<<grid, 256, 0, st>>>(a);
    if (a.offsets)
        k_offsets<<<(a.n_pairs + 256) / 256, 256, 0, st>>>(a.out_keys, &a.ctr->out, a.raw_cap,
                                                            a.n_pairs, a.tri_bits, a.offsets);
}

void launch_adjoint(const AdjointArgs &a, cudaStream_t st) {
    if (a.n <= 0) return;
    int grid = (int)((a.n + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_adjoint<<<grid, 256, 0, st>>>(a);
}

}  // namespace tms

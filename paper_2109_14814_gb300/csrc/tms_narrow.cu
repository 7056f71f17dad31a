// Narrow phase, merging of duplicate hits, output, and the adjoint.
//
// Narrow phase (arXiv 2109.14814, Sec. 5.2.4, Eq. (precise)): for triangles
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
// Mixed precision (optional): an FP32 solve first.  Its forward error is bounded
// from the FP32 residual and the normalised-column determinant rho: for the
// column-normalised matrix A_hat (unit columns, sigma_max <= 2),
// sigma_min >= rho / 8, so |D (z - z~)|_2 <= (8 / rho) |r - A z~|_2.  The
// residual is bounded rigorously from the FP32 computation (input rounding and
// accumulated rounding), and rho_true >= rho_fp32 / 2 whenever rho_fp32 >= 1e-2.
// A pair is rejected in FP32 only when the resulting upper bound of the margin
// is below -2 tau; every other pair gets the FP64 solve.
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
            if (p == row) {
#pragma unroll
                for (int j = col; j < 4; ++j) swap_(A[col][j], A[row][j]);
                swap_(r[col], r[row]);
                sign = -sign;
            }
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

__device__ __forceinline__ float f32_rn(double x) { return __double2float_rn(x); }

// FP32 pre-solve; true when it certifies margin < -2 tau (pair is not a hit)
__device__ __forceinline__ bool fp32_reject(const double x[3][4], const double y[3][4], double tau) {
    const float u = 5.9604645e-08f;   // 2^-24
    float A[4][4], Af[4][4], r[4], rf[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        // differences formed from FP32-rounded vertices; the rounding of the
        // vertices is an input perturbation bounded below
        float x1 = f32_rn(x[0][c]), x2 = f32_rn(x[1][c]), x3 = f32_rn(x[2][c]);
        float y1 = f32_rn(y[0][c]), y2 = f32_rn(y[1][c]), y3 = f32_rn(y[2][c]);
        A[c][0] = x1 - x2;
        A[c][1] = x3 - x2;
        A[c][2] = y2 - y1;
        A[c][3] = y2 - y3;
        r[c] = y2 - x2;
        // |exact entry - A| <= u (|v_i| + |v_j|) + u |A| per entry (vertex
        // rounding, then the subtraction)
        float ax1 = fabsf(x1), ax2 = fabsf(x2), ax3 = fabsf(x3);
        float ay1 = fabsf(y1), ay2 = fabsf(y2), ay3 = fabsf(y3);
        Af[c][0] = u * (ax1 + ax2) * 1.0001f + u * fabsf(A[c][0]);
        Af[c][1] = u * (ax3 + ax2) * 1.0001f + u * fabsf(A[c][1]);
        Af[c][2] = u * (ay2 + ay1) * 1.0001f + u * fabsf(A[c][2]);
        Af[c][3] = u * (ay2 + ay3) * 1.0001f + u * fabsf(A[c][3]);
        rf[c] = u * (ay2 + ax2) * 1.0001f + u * fabsf(r[c]);
    }
    float cn[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) cn[j] = sqrtf(A[0][j] * A[0][j] + A[1][j] * A[1][j] +
                                              A[2][j] * A[2][j] + A[3][j] * A[3][j]);
    float M[4][4], rr[4], z[4], det;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        rr[i] = r[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) M[i][j] = A[i][j];
    }
    solve4_gepp<float>(M, rr, z, det);
    const float rho = fabsf(det) / (cn[0] * cn[1] * cn[2] * cn[3]);
    if (!(rho >= 1e-2f)) return false;
    // the input rounding must be a small perturbation of the normalised matrix
    // (relative column perturbation <= 1e-3 rho keeps sigma_min >= rho / 8 up to
    // 1%); otherwise leave the pair to the FP64 solve
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float pj = sqrtf(Af[0][j] * Af[0][j] + Af[1][j] * Af[1][j] + Af[2][j] * Af[2][j] + Af[3][j] * Af[3][j]);
        if (!(pj <= 1e-3f * rho * cn[j])) return false;
    }
    // residual r - A z with a bound on its error (FP32 accumulation of 5 terms)
    float R2 = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float res = r[i];
        float mag = fabsf(r[i]);
        float pert = rf[i];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            res = fmaf(-A[i][j], z[j], res);
            mag += fabsf(A[i][j] * z[j]);
            pert += Af[i][j] * fabsf(z[j]);
        }
        float bound = fabsf(res) + 8.0f * u * mag + pert * 1.0001f;
        R2 += bound * bound;
    }
    const float R = sqrtf(R2) * 1.0001f;
    const float K = 20.0f;   // 8 (sigma_min >= rho/8) x 2 (rho_true >= rho/2) x 1.25
    float e[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) e[j] = K * R / (rho * cn[j]) * 1.0001f + 1e-30f;
    const float slack = 4.0f * u;
    float m = z[0] + e[0];
    m = fminf(m, z[1] + e[1]);
    m = fminf(m, z[2] + e[2]);
    m = fminf(m, z[3] + e[3]);
    m = fminf(m, 1.0f - z[0] - z[1] + e[0] + e[1] + slack * (1.0f + fabsf(z[0]) + fabsf(z[1])));
    m = fminf(m, 1.0f - z[2] - z[3] + e[2] + e[3] + slack * (1.0f + fabsf(z[2]) + fabsf(z[3])));
    const bool finite = isfinite(m) && isfinite(R);
    return finite && (m < (float)(-2.0 * tau));
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

__device__ __forceinline__ bool narrow_pair(const MeshDev &ma, const MeshDev &mb, uint32_t ta,
                                            uint32_t tb, double tau, int use_filter, bool &used64,
                                            tms_hit &h) {
    double x[3][4], y[3][4];
    gather_tri(ma, ta, x);
    gather_tri(mb, tb, y);
    used64 = false;
    if (use_filter && fp32_reject(x, y, tau)) return false;
    used64 = true;
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

template <int FACE>
__global__ void __launch_bounds__(256) k_narrow(NarrowArgs a) {
    if (a.ctr->cand > a.cand_cap) return;
    const unsigned long long n = a.ctr->cand;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (unsigned long long g0 = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x - lane;
         g0 < n; g0 += stride) {
        const unsigned long long g = g0 + lane;
        const bool valid = g < n;
        Cand cd;
        cd.faceA = cd.faceB = cd.pair = 0;
        if (valid) cd = a.cand[g];
        const int2 pr = a.pairs[valid ? cd.pair : 0];
        const MeshDev ma = a.meshes[pr.x];
        const MeshDev mb = a.meshes[pr.y];
        const int nsub = FACE == 0 ? 1 : 4;
#pragma unroll 1
        for (int sub = 0; sub < nsub; ++sub) {
            uint32_t ta, tb;
            if (FACE == 0) { ta = cd.faceA; tb = cd.faceB; }
            else { ta = 2 * cd.faceA + (sub & 1); tb = 2 * cd.faceB + (sub >> 1); }
            tms_hit h;
            bool hit = false, used64 = false;
            if (valid) hit = narrow_pair(ma, mb, ta, tb, a.tau, a.fp32_filter, used64, h);
            const unsigned n64 = __popc(__ballot_sync(FULL, used64));
            if (lane == 0 && n64) atomicAdd(&a.ctr->fp64, (unsigned long long)n64);
            const unsigned long long pos = warp_append(&a.ctr->raw_hits, hit, FULL);
            if (hit && pos < a.hit_cap) {
                h.pair = cd.pair;
                a.hits[pos] = h;
                a.hit_key[pos] = ((uint64_t)cd.pair << (2 * a.tri_bits)) |
                                 ((uint64_t)ta << a.tri_bits) | (uint64_t)tb;
                a.hit_val[pos] = (uint32_t)pos;
            }
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
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
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

void launch_narrow(const NarrowArgs &a, int face_level, int grid, cudaStream_t st) {
    if (face_level == 0) k_narrow<0><<<grid, 256, 0, st>>>(a);
    else k_narrow<1><<<grid, 256, 0, st>>>(a);
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

// Refinement of approximate manifold intersections (Sec. 7, Eqs. tosolve and
// dampedNewtonEquation): from each seed x = (theta_u, s_u, theta_s, s_s) the
// damped Newton iteration x <- x - alpha Df^{-1} f on
// f = W_A(theta_u, s_u) - W_B(theta_s, s_s), with W_A, W_B the closed-form
// sheet pair of tms_surface_pair and Df their exact partials, all in FP64.
//
// Layout: four lanes per seed, lane c owning coordinate c of every 4-vector
// (W, its partials, the normal frame, one row of Df).  The four sines/cosines
// and two exponentials an iteration needs are spread over the four lanes and
// exchanged by shuffles; dot products are butterfly sums over the quad (the
// same bits on every lane); the 4x4 solve is a partial-pivot elimination whose
// rows live in the lanes.  Every stop decision is taken on the quad's first
// lane and broadcast, so the four lanes always agree.  A warp loops while any
// of its eight seeds is still iterating; the loop is bounded by max_iter + 1
// evaluations per seed.
#include <cuda_runtime.h>
#include <math.h>

#include <cstddef>
#include <string>

#include "tms_common.cuh"

namespace {

constexpr int kH = TMS_SURF_MAX_HARMONICS;
constexpr int kF = TMS_SURF_MAX_FOLDS;
constexpr int kThreads = 128;          // 32 seeds per block
constexpr int kSeedsPerBlock = kThreads / 4;
constexpr unsigned kFull = 0xffffffffu;
constexpr double kPi = 3.141592653589793;
constexpr double kTwoPi = 6.283185307179586;

struct RefineArgs {
    tms_surface_pair sp;
    tms_refine_params p;
    const double *x0;
    long long ld;
    long long n;
    double *x;
    double *fnorm;
    double *rho;
    int *iters;
    int *status;
};

struct ContArgs {
    tms_surface_pair sp;
    tms_continue_params p;
    const double *alphas;   // nSteps values after the start
    int steps;              // nSteps
    const double *x0;
    long long ld;
    long long n;
    double *x;
    int *status;
    int *iters;
    double *rho;
    double *fnorm;
};

// Per-block tables, coordinate fastest (lane c reads column c).  With
// a_k = ca_k + alpha dca_k, b_k likewise:
//   T   = sum (a_k/k) cos + (b_k/k) sin     T' = sum b_k cos + (-a_k) sin
//   T'' = sum (-k a_k) cos + (-k b_k) sin
// so every harmonic term is two fused multiply-adds.  W_A's sheet is taken at
// alpha_u, B's underlying sheet at alpha_s, the normal frame at alpha_ref.
struct Coef {
    double uak[kH][4], ubk[kH][4], una[kH][4], ub[kH][4];     // at alpha_u
    double sak[kH][4], sbk[kH][4], sna[kH][4], sb[kH][4];     // at alpha_s
    double ark[kH][4], brk[kH][4], nar[kH][4], br[kH][4];     // at alpha_ref
    double kar[kH][4], kbr[kH][4];                            // at alpha_ref, T''
    // continuation: the walking sheet's tables above are taken at parameter 0 and
    // these hold their derivatives, so a branch at its own alpha uses
    // fma(alpha, d, table) -- the coefficients are affine in the parameter
    double dak[kH][4], dbk[kH][4], dna[kH][4], db[kH][4];
    double fd[kF][4];               // fold_amp * fold_dir
    double root[kF][3];             // fold roots
    double v1[4], v2[4];
    double qpi, hreg;               // Q pi and reg / 2
};

// Fills the tables for (alpha_u, alpha_s) and, for a walking sheet (walk != 0),
// the derivative tables; called by the threads of the block before a barrier.
__device__ void build_tables(Coef &cf, const tms_surface_pair &sp, double au, double as, int walk,
                             int t, int nt) {
    for (int q = t; q < kH * 4; q += nt) {
        const int h = q >> 2, c = q & 3;
        const double k = (double)(h + 1);
        const double a = sp.ca[h][c] + au * sp.dca[h][c];
        const double b = sp.cb[h][c] + au * sp.dcb[h][c];
        const double a2 = sp.ca[h][c] + as * sp.dca[h][c];
        const double b2 = sp.cb[h][c] + as * sp.dcb[h][c];
        const double ar = sp.ca[h][c] + sp.alpha_ref * sp.dca[h][c];
        const double br = sp.cb[h][c] + sp.alpha_ref * sp.dcb[h][c];
        cf.uak[h][c] = a / k;
        cf.ubk[h][c] = b / k;
        cf.una[h][c] = -a;
        cf.ub[h][c] = b;
        cf.sak[h][c] = a2 / k;
        cf.sbk[h][c] = b2 / k;
        cf.sna[h][c] = -a2;
        cf.sb[h][c] = b2;
        cf.ark[h][c] = ar / k;
        cf.brk[h][c] = br / k;
        cf.nar[h][c] = -ar;
        cf.br[h][c] = br;
        cf.kar[h][c] = -k * ar;
        cf.kbr[h][c] = -k * br;
        if (walk) {
            cf.dak[h][c] = sp.dca[h][c] / k;
            cf.dbk[h][c] = sp.dcb[h][c] / k;
            cf.dna[h][c] = -sp.dca[h][c];
            cf.db[h][c] = sp.dcb[h][c];
        }
    }
    if (t < kF * 4) cf.fd[t >> 2][t & 3] = sp.fold_amp[t >> 2] * sp.fold_dir[t >> 2][t & 3];
    if (t < kF * 3) cf.root[t / 3][t % 3] = sp.fold_root[t / 3][t % 3];
    if (t < 4) {
        cf.v1[t] = sp.v1[t];
        cf.v2[t] = sp.v2[t];
    }
    if (t == 0) {
        cf.qpi = sp.Q * kPi;
        cf.hreg = sp.reg * 0.5;
    }
}

// One seed's Newton solve, held identically by the quad's four lanes.
struct Solve {
    double x0, x1, x2, x3;   // iterate (angles unwrapped)
    int code;                // -1 while iterating, else TMS_REFINE_*
    int iters;               // updates made when the solve stopped
    int k;                   // updates made so far
    double fn, rh, rc2;      // ||f||^2, det Df, prod ||Df e_j||^2 at the last evaluation
};

__device__ __forceinline__ double quad_sum(double v) {
    v += __shfl_xor_sync(kFull, v, 1);
    v += __shfl_xor_sync(kFull, v, 2);
    return v;
}

__device__ __forceinline__ double lane_val(double v, int base, int j) {
    return __shfl_sync(kFull, v, base + j);
}

// p = (s - r0)(s - r1)(s - r2) and its first two derivatives.
__device__ __forceinline__ void cubic(double s, const double *r, double &p, double &p1,
                                      double &p2) {
    const double d0 = s - r[0], d1 = s - r[1], d2 = s - r[2];
    p = d0 * d1 * d2;
    p1 = d1 * d2 + d0 * d2 + d0 * d1;
    p2 = 2.0 * (d0 + d1 + d2);
}

// The quantities one damped-Newton iteration needs at the iterate (x0..x3): the
// stop checks, ||f||^2, the product of Df's squared column norms, det Df and the
// Newton step dx = Df^{-1} f.  Every lane of the warp calls it together (it
// exchanges values within the quad).  WALK = 1 or 2: the sheet of W_A or of B
// is taken at the quad's own parameter aw (continuation); 0: both at the
// tables' values.
struct Eval {
    int pre;       // stop decided before evaluating (non-finite or escaped iterate), or -1
    int fin;       // f and Df finite
    double r2, cn2, det, dx[4];
};

template <int WALK>
__device__ __forceinline__ void evaluate(const Coef &cf, const tms_surface_pair &sp,
                                         const tms_refine_params &pr, double lnlam, double x0,
                                         double x1, double x2, double x3, double aw, int c,
                                         int base, Eval &E) {
    const int K = sp.n_harmonics;
    const int NF = sp.n_folds;
    // ---- stop checks on the iterate (identical on the quad's lanes)
    int pre = -1;
    if (!(isfinite(x0) && isfinite(x1) && isfinite(x2) && isfinite(x3)))
        pre = TMS_REFINE_NON_FINITE;
    else if (x1 < pr.s_lo || x1 > pr.s_hi || x3 < pr.s_lo || x3 > pr.s_hi)
        pre = TMS_REFINE_ESCAPED;

    // ---- sines/cosines and exponentials, one per lane
    const double arg = c == 0 ? x0
                     : c == 1 ? x2 + sp.c0
                     : c == 2 ? sp.P * (x2 - sp.theta0)
                              : cf.qpi * (x3 - sp.s0);
    double sn, cs;
    sincos(arg, &sn, &cs);
    const double sA = lane_val(sn, base, 0), cA = lane_val(cs, base, 0);
    const double sB = lane_val(sn, base, 1), cB = lane_val(cs, base, 1);
    const double sh1 = lane_val(sn, base, 2), ch1 = lane_val(cs, base, 2);
    const double sh2 = lane_val(sn, base, 3), ch2 = lane_val(cs, base, 3);
    const double s1 = 1.0 - x3;   // s' of B's underlying sheet
    double gA, gA1, gB, gB1, gB2;
    if (sp.stretch) {
        const double e = exp(lnlam * (c == 0 ? x1 : s1));
        gA = lane_val(e, base, 0);
        gB = lane_val(e, base, 1);
        gA1 = lnlam * gA;
        gB1 = lnlam * gB;
        gB2 = lnlam * gB1;
    } else {
        gA = 1.0 + x1;
        gA1 = 1.0;
        gB = 1.0 + s1;
        gB1 = 1.0;
        gB2 = 0.0;
    }

    // ---- folds F(s) at s_u and at s': lane f evaluates fold f's cubics
    double FA = 0.0, FA1 = 0.0, FB = 0.0, FB1 = 0.0, FB2 = 0.0;
    if (NF > 0) {
        double p, p1, p2, q, q1, q2;
        const int fo = c < NF ? c : 0;
        cubic(x1, cf.root[fo], p, p1, p2);
        cubic(s1, cf.root[fo], q, q1, q2);
#pragma unroll
        for (int f = 0; f < kF; ++f) {
            if (f < NF) {
                const double w = cf.fd[f][c];
                FA = fma(w, lane_val(p, base, f), FA);
                FA1 = fma(w, lane_val(p1, base, f), FA1);
                FB = fma(w, lane_val(q, base, f), FB);
                FB1 = fma(w, lane_val(q1, base, f), FB1);
                FB2 = fma(w, lane_val(q2, base, f), FB2);
            }
        }
    }

    // ---- harmonic sums: T, T' at theta_u (alpha_u); T, T' at theta' (alpha_s);
    //      T, T', T'' at theta' (alpha_ref).  cos/sin of k theta by angle addition.
    double TA = 0.0, TAt = 0.0, TB = 0.0, TBt = 0.0, TR = 0.0, TRt = 0.0, TRtt = 0.0;
    double ckA = cA, skA = sA, ckB = cB, skB = sB;
#pragma unroll
    for (int h = 0; h < kH; ++h) {
        if (h < K) {
            double uak = cf.uak[h][c], ubk = cf.ubk[h][c], una = cf.una[h][c], ub = cf.ub[h][c];
            double sak = cf.sak[h][c], sbk = cf.sbk[h][c], sna = cf.sna[h][c], sb = cf.sb[h][c];
            if (WALK == 1) {
                uak = fma(aw, cf.dak[h][c], uak);
                ubk = fma(aw, cf.dbk[h][c], ubk);
                una = fma(aw, cf.dna[h][c], una);
                ub = fma(aw, cf.db[h][c], ub);
            } else if (WALK == 2) {
                sak = fma(aw, cf.dak[h][c], sak);
                sbk = fma(aw, cf.dbk[h][c], sbk);
                sna = fma(aw, cf.dna[h][c], sna);
                sb = fma(aw, cf.db[h][c], sb);
            }
            TA = fma(uak, ckA, fma(ubk, skA, TA));
            TAt = fma(ub, ckA, fma(una, skA, TAt));
            TB = fma(sak, ckB, fma(sbk, skB, TB));
            TBt = fma(sb, ckB, fma(sna, skB, TBt));
            TR = fma(cf.ark[h][c], ckB, fma(cf.brk[h][c], skB, TR));
            TRt = fma(cf.br[h][c], ckB, fma(cf.nar[h][c], skB, TRt));
            TRtt = fma(cf.kar[h][c], ckB, fma(cf.kbr[h][c], skB, TRtt));
            if (h + 1 < K) {
                const double nA = ckA * cA - skA * sA;
                skA = skA * cA + ckA * sA;
                ckA = nA;
                const double nB = ckB * cB - skB * sB;
                skB = skB * cB + ckB * sB;
                ckB = nB;
            }
        }
    }

    // ---- W_A and its partials; B's underlying sheet; the frame sheet
    const double WA = gA * TA + FA, WAt = gA * TAt, WAs = gA1 * TA + FA1;
    const double SB = gB * TB + FB, SBt = gB * TBt, SBs = gB1 * TB + FB1;
    const double t1 = gB * TRt, t2 = gB1 * TR + FB1;
    const double Wtt = gB * TRtt, Wts = gB1 * TRt, Wss = gB2 * TR + FB2;
    const double v1 = cf.v1[c], v2 = cf.v2[c];

    // ---- normal frame (n1, n2) and its theta- and s-partials
    const double g11 = quad_sum(t1 * t1), g12 = quad_sum(t1 * t2), g22 = quad_sum(t2 * t2);
    const double j11 = quad_sum(t1 * v1), j21 = quad_sum(t2 * v1);
    const double j12 = quad_sum(t1 * v2), j22 = quad_sum(t2 * v2);
    const double P1 = quad_sum(t1 * Wtt), P2 = quad_sum(t1 * Wts), P3 = quad_sum(Wtt * t2);
    const double P4 = quad_sum(t2 * Wts), P5 = quad_sum(t1 * Wss), P6 = quad_sum(t2 * Wss);
    const double Lt1 = quad_sum(Wtt * v1), Ls1 = quad_sum(Wts * v1), Ss1 = quad_sum(Wss * v1);
    const double Lt2 = quad_sum(Wtt * v2), Ls2 = quad_sum(Wts * v2), Ss2 = quad_sum(Wss * v2);
    const double eps = cf.hreg * (g11 + g22);
    const double G11 = g11 + eps, G12 = g12, G22 = g22 + eps;
    const double idet = 1.0 / (G11 * G22 - G12 * G12);
    // d/dtheta and d/ds of G (J^T J + eps I)
    const double tg11 = 2.0 * P1, tg12 = P2 + P3, tg22 = 2.0 * P4;
    const double te = cf.hreg * (tg11 + tg22);
    const double tG11 = tg11 + te, tG22 = tg22 + te;
    const double sg11 = -2.0 * P2, sg12 = -(P5 + P4), sg22 = -2.0 * P6;
    const double se = cf.hreg * (sg11 + sg22);
    const double sG11 = sg11 + se, sG22 = sg22 + se;

    // lane c solves for frame vector r = c & 1, then both are shared
    double yv[6];
    {
        const int r = c & 1;
        const double j1 = r ? j12 : j11, j2 = r ? j22 : j21;
        const double Lt = r ? Lt2 : Lt1, Ls = r ? Ls2 : Ls1, Ss = r ? Ss2 : Ss1;
        const double y1 = (G22 * j1 - G12 * j2) * idet, y2 = (G11 * j2 - G12 * j1) * idet;
        // theta: d t1 = Wtt, d t2 = Wts;  s: d t1 = -Wts, d t2 = -Wss
        const double a1 = Lt - (tG11 * y1 + tg12 * y2), a2 = Ls - (tg12 * y1 + tG22 * y2);
        const double b1 = -Ls - (sG11 * y1 + sg12 * y2), b2 = -Ss - (sg12 * y1 + sG22 * y2);
        yv[0] = y1;
        yv[1] = y2;
        yv[2] = (G22 * a1 - G12 * a2) * idet;
        yv[3] = (G11 * a2 - G12 * a1) * idet;
        yv[4] = (G22 * b1 - G12 * b2) * idet;
        yv[5] = (G11 * b2 - G12 * b1) * idet;
    }
    double n[2], nt[2], ns[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const double v = r == 0 ? v1 : v2;
        const double y1 = lane_val(yv[0], base, r), y2 = lane_val(yv[1], base, r);
        const double dt1 = lane_val(yv[2], base, r), dt2 = lane_val(yv[3], base, r);
        const double ds1 = lane_val(yv[4], base, r), ds2 = lane_val(yv[5], base, r);
        n[r] = v - t1 * y1 - t2 * y2;
        nt[r] = -(Wtt * y1 + Wts * y2) - (t1 * dt1 + t2 * dt2);
        ns[r] = (Wts * y1 + Wss * y2) - (t1 * ds1 + t2 * ds2);
    }

    // ---- W_B, f and the row of Df this lane owns
    const double h = sp.h_amp;
    const double H = h * (sh1 * n[0] + sh2 * n[1]);
    const double Ht = h * (sp.P * ch1 * n[0] + sh1 * nt[0] + sh2 * nt[1]);
    const double Hs = h * (sh1 * ns[0] + cf.qpi * ch2 * n[1] + sh2 * ns[1]);
    const double fc = WA - (SB + H);
    double m[4] = {WAt, WAs, -(SBt + Ht), -(-SBs + Hs)};

    const double r2 = quad_sum(fc * fc);
    double cn2 = 1.0;   // product of the squared column norms
#pragma unroll
    for (int j = 0; j < 4; ++j) cn2 *= quad_sum(m[j] * m[j]);
    int fin = isfinite(fc) && isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2]) &&
              isfinite(m[3]);
    fin &= __shfl_xor_sync(kFull, fin, 1);
    fin &= __shfl_xor_sync(kFull, fin, 2);

    // ---- Df dx = f by partial-pivot elimination over the quad's rows
    double rr = fc, det = 1.0, ip[4];
    int used = 0, pl[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double cand = ((used >> c) & 1) ? -1.0 : fabs(m[j]);
        int bl = c;
#pragma unroll
        for (int off = 1; off <= 2; off <<= 1) {
            const double oc = __shfl_xor_sync(kFull, cand, off);
            const int ol = __shfl_xor_sync(kFull, bl, off);
            if (oc > cand || (oc == cand && ol < bl)) {
                cand = oc;
                bl = ol;
            }
        }
        used |= 1 << bl;
        pl[j] = bl;
        double pj[4];
#pragma unroll
        for (int q = j; q < 4; ++q) pj[q] = lane_val(m[q], base, bl);
        const double prr = lane_val(rr, base, bl);
        det *= pj[j];
        ip[j] = pj[j] != 0.0 ? 1.0 / pj[j] : 0.0;
        if (!((used >> c) & 1)) {
            const double fct = m[j] * ip[j];
#pragma unroll
            for (int q = j + 1; q < 4; ++q) m[q] -= fct * pj[q];
            rr -= fct * prr;
            m[j] = 0.0;
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int w = u + 1; w < 4; ++w)
            if (pl[u] > pl[w]) det = -det;
    double dx[4];
#pragma unroll
    for (int j = 3; j >= 0; --j) {
        double v = rr;
#pragma unroll
        for (int q = j + 1; q < 4; ++q) v -= m[q] * dx[q];
        dx[j] = lane_val(v * ip[j], base, pl[j]);
    }

    E.pre = pre;
    E.fin = fin;
    E.r2 = r2;
    E.cn2 = cn2;
    E.det = det;
#pragma unroll
    for (int q = 0; q < 4; ++q) E.dx[q] = dx[q];
}

// The decision of Eq. (dampedNewtonEquation)'s iteration k from an evaluation:
// -1 to update, else the stop status (taken on the quad's first lane).
__device__ __forceinline__ int decide(const Eval &E, const tms_refine_params &pr, double tol2, int k,
                                      int base) {
    // ||f|| <= tol as ||f||^2 <= tol^2; |det| / prod ||col|| >= rho_min as
    // |det| >= rho_min sqrt(prod ||col||^2)
    int dec = E.pre;
    if (dec < 0) {
        if (!E.fin) dec = TMS_REFINE_NON_FINITE;
        else if (E.r2 <= tol2) dec = TMS_REFINE_CONVERGED;
        else if (k == pr.max_iter) dec = TMS_REFINE_MAX_ITER;
        else if (!(fabs(E.det) >= pr.rho_min * sqrt(E.cn2))) dec = TMS_REFINE_SINGULAR;
    }
    return __shfl_sync(kFull, dec, base);
}

// Applies a decision to a quad that is still iterating.
__device__ __forceinline__ void apply(const Eval &E, const tms_refine_params &pr, double sw2, int dec,
                                      int k, Solve &S) {
    if (S.code >= 0) return;
    if (E.pre < 0) {
        S.fn = E.r2;
        S.rh = E.det;
        S.rc2 = E.cn2;
    }
    if (dec >= 0) {
        S.code = dec;
        S.iters = k;
    } else {
        const double al = E.r2 > sw2 ? pr.alpha0 : pr.alpha1;
        S.x0 -= al * E.dx[0];
        S.x1 -= al * E.dx[1];
        S.x2 -= al * E.dx[2];
        S.x3 -= al * E.dx[3];
        S.k = k + 1;
    }
}

// The whole solve for every quad of the warp at once (the refinement): the
// iteration counter is the warp's; at most max_iter + 1 evaluations each.
__device__ __forceinline__ void newton_solve(const Coef &cf, const tms_surface_pair &sp,
                                             const tms_refine_params &pr, Solve &S, int c,
                                             int base) {
    const double lnlam = sp.stretch ? log(sp.lam) : 0.0;
    const double tol2 = pr.tol * pr.tol, sw2 = pr.switch_below * pr.switch_below;
    for (int k = 0; __any_sync(kFull, S.code < 0); ++k) {
        Eval E;
        evaluate<0>(cf, sp, pr, lnlam, S.x0, S.x1, S.x2, S.x3, 0.0, c, base, E);
        apply(E, pr, sw2, decide(E, pr, tol2, k, base), k, S);
    }
}

// One iteration for each quad at its own count S.k (the continuation).
template <int WALK>
__device__ __forceinline__ void newton_iter(const Coef &cf, const tms_surface_pair &sp,
                                            const tms_refine_params &pr, double lnlam, double tol2,
                                            double sw2, Solve &S, double aw, int c, int base) {
    Eval E;
    evaluate<WALK>(cf, sp, pr, lnlam, S.x0, S.x1, S.x2, S.x3, aw, c, base, E);
    apply(E, pr, sw2, decide(E, pr, tol2, S.k, base), S.k, S);
}

__device__ __forceinline__ double wrap_angle(double v) {
    double w = fmod(v, kTwoPi);
    if (w < 0.0) w += kTwoPi;
    else if (w == 0.0) w = 0.0;   // +0 for a -0 remainder
    return w;
}

__device__ __forceinline__ double nan_value() { return __longlong_as_double(0x7ff8000000000000LL); }

__global__ void __launch_bounds__(kThreads) k_refine(const __grid_constant__ RefineArgs a) {
    __shared__ Coef cf;
    const tms_surface_pair &sp = a.sp;
    const int t = threadIdx.x;
    build_tables(cf, sp, sp.alpha_u, sp.alpha_s, 0, t, kThreads);
    __syncthreads();

    const int lane = t & 31;
    const int c = lane & 3;
    const int base = lane & ~3;
    const long long i = (long long)blockIdx.x * kSeedsPerBlock + (t >> 2);
    const bool live = i < a.n;
    Solve S;
    S.x0 = 0.0;
    S.x1 = 0.5;
    S.x2 = 0.0;
    S.x3 = 0.5;
    if (live) {
        const double *s = a.x0 + i * a.ld;
        S.x0 = s[0];
        S.x1 = s[1];
        S.x2 = s[2];
        S.x3 = s[3];
    }
    S.code = live ? -1 : TMS_REFINE_CONVERGED;
    S.iters = 0;
    S.k = 0;
    S.fn = nan_value();
    S.rh = S.fn;
    S.rc2 = 1.0;
    newton_solve(cf, sp, a.p, S, c, base);

    if (live) {
        double xc = c == 0 ? S.x0 : c == 1 ? S.x1 : c == 2 ? S.x2 : S.x3;
        if (c == 0 || c == 2) xc = wrap_angle(xc);
        a.x[i * 4 + c] = xc;
        if (c == 0) {
            if (a.fnorm) a.fnorm[i] = sqrt(S.fn);
            if (a.rho) a.rho[i] = S.rh / sqrt(S.rc2);
            if (a.iters) a.iters[i] = S.iters;
            if (a.status) a.status[i] = S.code;
        }
    }
}

// Continuation (Sec. 8): one quad per branch walks the parameter values
// alpha_0 (the pair's own), alphas[0..steps) of the walking sheet (WALK = 1:
// W_A's alpha_u, 2: B's alpha_s).  The branches of a warp do not wait for one
// another between steps: each quad evaluates its sheet at its own current
// parameter (the coefficients are affine in it), and when its corrector stops
// it records the step and, unless the branch stopped, predicts the next step
// and goes on in the same warp-wide iteration loop, which ends when all of the
// warp's branches have.
template <int WALK>
__global__ void __launch_bounds__(kThreads) k_continue(const __grid_constant__ ContArgs a) {
    __shared__ Coef cf;
    const tms_surface_pair &sp = a.sp;
    const tms_continue_params &cp = a.p;
    const int t = threadIdx.x;
    build_tables(cf, sp, WALK == 1 ? 0.0 : sp.alpha_u, WALK == 2 ? 0.0 : sp.alpha_s, WALK, t,
                 kThreads);
    __syncthreads();
    const int lane = t & 31;
    const int c = lane & 3;
    const int base = lane & ~3;
    const long long i = (long long)blockIdx.x * kSeedsPerBlock + (t >> 2);
    const bool live = i < a.n;
    double g[4] = {0.0, 0.5, 0.0, 0.5};   // the current step's starting point
    if (live) {
        const double *s = a.x0 + i * a.ld;
#pragma unroll
        for (int q = 0; q < 4; ++q) g[q] = s[q];
    }
    double p1[4] = {0.0, 0.0, 0.0, 0.0}, p2[4] = {0.0, 0.0, 0.0, 0.0};   // x_{j-1}, x_{j-2}
    bool alive = live;
    int j = 0;
    double rho_prev = nan_value();
    const double a0 = WALK == 1 ? sp.alpha_u : sp.alpha_s;
    double aj = a0, am1 = a0, am2 = a0;   // alpha_j, alpha_{j-1}, alpha_{j-2}
    const long long K1 = (long long)a.steps + 1;
    Solve S;
    S.x0 = g[0];
    S.x1 = g[1];
    S.x2 = g[2];
    S.x3 = g[3];
    S.code = alive ? -1 : TMS_REFINE_CONVERGED;
    S.iters = 0;
    S.k = 0;
    S.fn = nan_value();
    S.rh = S.fn;
    S.rc2 = 1.0;
    const double lnlam = sp.stretch ? log(sp.lam) : 0.0;
    const double tol2 = cp.corrector.tol * cp.corrector.tol;
    const double sw2 = cp.corrector.switch_below * cp.corrector.switch_below;
    while (__any_sync(kFull, alive)) {
        newton_iter<WALK>(cf, sp, cp.corrector, lnlam, tol2, sw2, S, aj, c, base);
        if (!(alive && S.code >= 0)) continue;
        // ---- step j is done (identical on the quad's lanes; no shuffles below)
        const double xs[4] = {wrap_angle(S.x0), S.x1, wrap_angle(S.x2), S.x3};
        const double rho = S.rh / sqrt(S.rc2);
        int st = S.code;
        if (st == TMS_REFINE_CONVERGED) {
            double jump = 0.0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                double d = fabs(xs[q] - g[q]);
                if (q == 0 || q == 2) d = fabs(d - kTwoPi * rint(d / kTwoPi));
                jump = fmax(jump, d);
            }
            if (!(jump <= cp.max_jump)) st = TMS_CONT_JUMPED;
            else if (!(fabs(rho) >= cp.rho_turn)) st = TMS_CONT_TURNING;
            else if (j > 0 && (rho > 0.0) != (rho_prev > 0.0)) st = TMS_CONT_TURNING;
        }
        const long long o = i * K1 + j;
        a.x[o * 4 + c] = xs[c];
        if (c == 0) {
            a.status[o] = st;
            if (a.iters) a.iters[o] = S.iters;
            if (a.rho) a.rho[o] = rho;
            if (a.fnorm) a.fnorm[o] = sqrt(S.fn);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            p2[q] = p1[q];
            p1[q] = xs[q];
        }
        rho_prev = rho;
        if (st != TMS_REFINE_CONVERGED || j == a.steps) {
            alive = false;
            for (long long r = j + 1; r <= a.steps; ++r) {
                const long long oo = i * K1 + r;
                a.x[oo * 4 + c] = nan_value();
                if (c == 0) {
                    a.status[oo] = TMS_CONT_STOPPED;
                    if (a.iters) a.iters[oo] = 0;
                    if (a.rho) a.rho[oo] = nan_value();
                    if (a.fnorm) a.fnorm[oo] = nan_value();
                }
            }
            continue;
        }
        // ---- next step: predictor, Eq. (predictor); angle differences on the circle
        ++j;
        am2 = am1;
        am1 = aj;
        aj = a.alphas[j - 1];
        if (j == 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) g[q] = p1[q];
        } else {
            const double ratio = (aj - am1) / (am1 - am2);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                double d = p1[q] - p2[q];
                if (q == 0 || q == 2) d -= kTwoPi * rint(d / kTwoPi);
                g[q] = p1[q] + ratio * d;
            }
        }
        S.x0 = g[0];
        S.x1 = g[1];
        S.x2 = g[2];
        S.x3 = g[3];
        S.code = -1;
        S.iters = 0;
        S.k = 0;
        S.fn = nan_value();
        S.rh = S.fn;
        S.rc2 = 1.0;
    }
}

bool all_finite(const double *v, size_t n) {
    for (size_t j = 0; j < n; ++j)
        if (!isfinite(v[j])) return false;
    return true;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

tms_status arg_error(const char *msg) {
    tms::set_last_error(msg);
    return TMS_ERR_ARG;
}


tms_status check_surface(const tms_surface_pair &s, const char *who) {
    const std::string w(who);
    if (s.n_harmonics < 1 || s.n_harmonics > TMS_SURF_MAX_HARMONICS)
        return arg_error((w + ": n_harmonics outside 1..8").c_str());
    if (s.n_folds < 0 || s.n_folds > TMS_SURF_MAX_FOLDS)
        return arg_error((w + ": n_folds outside 0..4").c_str());
    if (s.stretch != 0 && s.stretch != 1) return arg_error((w + ": stretch must be 0 or 1").c_str());
    if (s.stretch == 1 && !(s.lam > 0.0)) return arg_error((w + ": lam must be > 0").c_str());
    bool fin = true;
    for (int h = 0; h < s.n_harmonics; ++h)
        fin = fin && all_finite(s.ca[h], 4) && all_finite(s.cb[h], 4) && all_finite(s.dca[h], 4) &&
              all_finite(s.dcb[h], 4);
    for (int f = 0; f < s.n_folds; ++f)
        fin = fin && isfinite(s.fold_amp[f]) && all_finite(s.fold_root[f], 3) &&
              all_finite(s.fold_dir[f], 4);
    const size_t ns = (sizeof(tms_surface_pair) - offsetof(tms_surface_pair, c0)) / sizeof(double);
    fin = fin && isfinite(s.alpha_u) && isfinite(s.alpha_s) && isfinite(s.alpha_ref) &&
          (s.stretch == 0 || isfinite(s.lam)) && all_finite(&s.c0, ns);
    if (!fin) return arg_error((w + ": non-finite surface value").c_str());
    if (!(s.reg >= 0.0)) return arg_error((w + ": reg must be >= 0").c_str());
    return TMS_OK;
}

tms_status check_corrector(const tms_refine_params &p, const char *who) {
    const std::string w(who);
    if (!(p.alpha0 > 0.0 && p.alpha0 <= 1.0 && p.alpha1 > 0.0 && p.alpha1 <= 1.0))
        return arg_error((w + ": alpha0 and alpha1 must lie in (0, 1]").c_str());
    if (!(p.tol >= 0.0) || !(p.switch_below >= 0.0) || !(p.rho_min >= 0.0))
        return arg_error((w + ": tol, switch_below and rho_min must be >= 0").c_str());
    if (!(p.s_lo < p.s_hi)) return arg_error((w + ": need s_lo < s_hi").c_str());
    if (p.max_iter < 0 || p.max_iter > 1000000)
        return arg_error((w + ": max_iter outside 0..1000000").c_str());
    return TMS_OK;
}

}  // namespace

extern "C" void tms_refine_params_default(tms_refine_params *p) {
    if (!p) return;
    p->alpha0 = 0.5;
    p->alpha1 = 0.5;
    p->switch_below = 0.0;
    p->tol = 1e-10;
    p->s_lo = -0.5;
    p->s_hi = 1.5;
    p->rho_min = 1e-14;
    p->max_iter = 200;
    p->pad = 0;
}

extern "C" tms_status tms_refine(const tms_surface_pair *surf, const tms_refine_params *params,
                                 const double *dX0, long long ldx0, long long n, double *dX,
                                 double *dFnorm, double *dRho, int32_t *dIters, int32_t *dStatus,
                                 void *stream) {
    if (!surf) return arg_error("tms_refine: surface is NULL");
    if (n < 0) return arg_error("tms_refine: n < 0");
    tms_refine_params p;
    if (params) p = *params;
    else tms_refine_params_default(&p);
    tms_status st = check_surface(*surf, "tms_refine");
    if (st == TMS_OK) st = check_corrector(p, "tms_refine");
    if (st != TMS_OK) return st;
    if (n == 0) return TMS_OK;
    if (ldx0 < 4) return arg_error("tms_refine: ldx0 < 4");
    if (!dX0 || !dX || !is_device_ptr(dX0) || !is_device_ptr(dX))
        return arg_error("tms_refine: seeds and output must be device pointers");
    if (dX == dX0 && ldx0 != 4) return arg_error("tms_refine: in place needs ldx0 == 4");
    RefineArgs a;
    a.sp = *surf;
    a.p = p;
    a.x0 = dX0;
    a.ld = ldx0;
    a.n = n;
    a.x = dX;
    a.fnorm = dFnorm;
    a.rho = dRho;
    a.iters = dIters;
    a.status = dStatus;
    const long long blocks = (n + kSeedsPerBlock - 1) / kSeedsPerBlock;
    if (blocks > 0x7fffffffLL) return arg_error("tms_refine: too many seeds");
    k_refine<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        tms::set_last_error(std::string("tms_refine launch: ") + cudaGetErrorString(e));
        return TMS_ERR_CUDA;
    }
    return TMS_OK;
}

extern "C" void tms_continue_params_default(tms_continue_params *p) {
    if (!p) return;
    tms_refine_params_default(&p->corrector);
    p->rho_turn = 1e-8;
    p->max_jump = 0.25;
    p->param = 0;
    p->pad = 0;
}

extern "C" tms_status tms_continue(const tms_surface_pair *surf, const tms_continue_params *params,
                                   const double *dAlphas, int nSteps, const double *dX0,
                                   long long ldx0, long long n, double *dX, int32_t *dStatus,
                                   int32_t *dIters, double *dRho, double *dFnorm, void *stream) {
    if (!surf) return arg_error("tms_continue: surface is NULL");
    if (n < 0) return arg_error("tms_continue: n < 0");
    if (nSteps < 0) return arg_error("tms_continue: nSteps < 0");
    tms_continue_params p;
    if (params) p = *params;
    else tms_continue_params_default(&p);
    tms_status st = check_surface(*surf, "tms_continue");
    if (st == TMS_OK) st = check_corrector(p.corrector, "tms_continue");
    if (st != TMS_OK) return st;
    if (p.param != 0 && p.param != 1) return arg_error("tms_continue: param must be 0 or 1");
    if (!(p.rho_turn >= 0.0)) return arg_error("tms_continue: rho_turn must be >= 0");
    if (!(p.max_jump > 0.0)) return arg_error("tms_continue: max_jump must be > 0");
    if (n == 0) return TMS_OK;
    if (ldx0 < 4) return arg_error("tms_continue: ldx0 < 4");
    if (!dX0 || !dX || !dStatus || !is_device_ptr(dX0) || !is_device_ptr(dX) ||
        !is_device_ptr(dStatus))
        return arg_error("tms_continue: seeds, dX and dStatus must be device pointers");
    if (nSteps > 0 && (!dAlphas || !is_device_ptr(dAlphas)))
        return arg_error("tms_continue: dAlphas must be a device pointer");
    ContArgs a;
    a.sp = *surf;
    a.p = p;
    a.alphas = dAlphas;
    a.steps = nSteps;
    a.x0 = dX0;
    a.ld = ldx0;
    a.n = n;
    a.x = dX;
    a.status = dStatus;
    a.iters = dIters;
    a.rho = dRho;
    a.fnorm = dFnorm;
    const long long blocks = (n + kSeedsPerBlock - 1) / kSeedsPerBlock;
    if (blocks > 0x7fffffffLL) return arg_error("tms_continue: too many branches");
    if (p.param == 0) k_continue<1><<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(a);
    else k_continue<2><<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        tms::set_last_error(std::string("tms_continue launch: ") + cudaGetErrorString(e));
        return TMS_ERR_CUDA;
    }
    return TMS_OK;
}

// Operations on theta grids (functions of theta stored at theta_i = 2 pi i / N,
// Sec. 4 and Sec. 6.1): translation and derivative of every column of a
// coordinate array through the FFT (Eqs. translate, translate2), and grid
// phase alignment of two circles (Eq. rhoEquationDiscrete).
//
// Translation: one CTA per complex transform of two real rows that share a
// shift (the same s column of two coordinates), packed as z = a + j b.  The
// multiplier H(k) = e^{j k rho} (times j k for the derivative) over the signed
// frequencies keeps H(-k) = conj(H(k)), with the Nyquist term real, so the two
// real results come back as the real and imaginary parts.  Forward: radix-2
// decimation in time from bit-reversed input; inverse: decimation in frequency
// to bit-reversed output, read back through the same permutation.  All in
// FP64 in shared memory.
#include <cuda_runtime.h>
#include <math.h>

#include <string>

#include "tms_common.cuh"

namespace {

constexpr int kFftThreads = 256;
constexpr int kTab = 64;   // two-level tables: e^{j x (hi * 64 + lo)} = T_hi[hi] T_lo[lo]

struct ThetaArgs {
    const double *in;
    double *out;
    long long ldc;     // doubles between coordinate blocks
    const double *rho; // per column, or null
    double rho0;
    int N, logN, cols, ncoord, derivative;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

__global__ void __launch_bounds__(kFftThreads) k_theta_fft(const ThetaArgs a) {
    extern __shared__ double2 sm[];
    const int N = a.N;
    double2 *z = sm;                 // N values
    double2 *w = sm + N;             // N/2 twiddles e^{-2 pi j m / N}
    double2 *th = w + N / 2;         // kTab: e^{-2 pi j (hi * kTab) / N}
    double2 *tl = th + kTab;         // kTab: e^{-2 pi j lo / N}
    double2 *hh = tl + kTab;         // kTab: e^{j rho hi kTab}
    double2 *hl = hh + kTab;         // kTab: e^{j rho lo}
    const int t = threadIdx.x;
    const int col = blockIdx.x % a.cols;
    const int pair = blockIdx.x / a.cols;
    const int c0 = 2 * pair, c1 = 2 * pair + 1;
    const bool two = c1 < a.ncoord;
    const double rho = a.rho ? a.rho[col] : a.rho0;
    if (t < kTab) {
        double s, c;
        sincospi(-2.0 * (double)(t * kTab) / (double)N, &s, &c);
        th[t] = make_double2(c, s);
        sincospi(-2.0 * (double)t / (double)N, &s, &c);
        tl[t] = make_double2(c, s);
        sincos(rho * (double)(t * kTab), &s, &c);
        hh[t] = make_double2(c, s);
        sincos(rho * (double)t, &s, &c);
        hl[t] = make_double2(c, s);
    }
    const double *ra = a.in + (long long)c0 * a.ldc + (long long)col * N;
    const double *rb = a.in + (long long)c1 * a.ldc + (long long)col * N;
    const int sh = 32 - a.logN;
    for (int i = t; i < N; i += kFftThreads)
        z[__brev((unsigned)i) >> sh] = make_double2(ra[i], two ? rb[i] : 0.0);
    __syncthreads();
    for (int m = t; m < N / 2; m += kFftThreads) w[m] = cmul(th[m / kTab], tl[m % kTab]);
    __syncthreads();

    // forward transform (decimation in time)
    for (int half = 1; half < N; half <<= 1) {
        const int stride = N / (2 * half);
        for (int b = t; b < N / 2; b += kFftThreads) {
            const int pos = b & (half - 1);
            const int i = ((b - pos) << 1) + pos;
            const double2 v = cmul(w[pos * stride], z[i + half]);
            const double2 u = z[i];
            z[i] = make_double2(u.x + v.x, u.y + v.y);
            z[i + half] = make_double2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }

    // multiplier over the signed frequencies
    for (int i = t; i < N; i += kFftThreads) {
        double2 v = z[i];
        if (i == N / 2) {
            double s, c;
            sincos(0.5 * (double)N * rho, &s, &c);
            const double g = a.derivative ? 0.0 : c;
            v = make_double2(v.x * g, v.y * g);
        } else {
            const int k = i < N / 2 ? i : i - N;
            const int ak = k < 0 ? -k : k;
            double2 e = cmul(hh[ak / kTab], hl[ak % kTab]);   // e^{j rho |k|}
            if (k < 0) e.y = -e.y;
            if (a.derivative) e = make_double2(-(double)k * e.y, (double)k * e.x);
            v = cmul(v, e);
        }
        z[i] = v;
    }
    __syncthreads();

    // inverse transform (decimation in frequency, conjugate twiddles)
    for (int half = N / 2; half >= 1; half >>= 1) {
        const int stride = N / (2 * half);
        for (int b = t; b < N / 2; b += kFftThreads) {
            const int pos = b & (half - 1);
            const int i = ((b - pos) << 1) + pos;
            const double2 u = z[i], v = z[i + half];
            z[i] = make_double2(u.x + v.x, u.y + v.y);
            z[i + half] = cmulc(make_double2(u.x - v.x, u.y - v.y), w[pos * stride]);
        }
        __syncthreads();
    }

    const double inv = 1.0 / (double)N;
    double *oa = a.out + (long long)c0 * a.ldc + (long long)col * N;
    double *ob = a.out + (long long)c1 * a.ldc + (long long)col * N;
    for (int i = t; i < N; i += kFftThreads) {
        const double2 v = z[__brev((unsigned)i) >> sh];
        oa[i] = v.x * inv;
        if (two) ob[i] = v.y * inv;
    }
}

// Phase alignment cost: block (x, a) computes cost_a(m) for 128 shifts m; the
// sum over i runs in order, one thread per shift, through shared tiles of the
// previous circle and of the matching window of the shifted one.
constexpr int kPhThreads = 128;
constexpr int kPhTile = 512;

struct PhaseArgs {
    const double *wr;
    const double *wp;
    double *cost;
    int N, ncoord, nalign;
};

__global__ void __launch_bounds__(kPhThreads) k_phase_cost(const PhaseArgs a) {
    extern __shared__ double ps[];
    const int C = a.ncoord, N = a.N;
    double *prev = ps;                          // C x kPhTile
    double *win = ps + C * kPhTile;             // C x (kPhTile + kPhThreads)
    const int al = blockIdx.y;
    const int m0 = blockIdx.x * kPhThreads;
    const int m = m0 + threadIdx.x;
    const double *Wr = a.wr + (long long)al * C * N;
    const double *Wp = a.wp + (long long)al * C * N;
    double acc = 0.0;
    for (int i0 = 0; i0 < N; i0 += kPhTile) {
        const int ti = min(kPhTile, N - i0);
        __syncthreads();
        for (int q = threadIdx.x; q < C * kPhTile; q += kPhThreads) {
            const int c = q / kPhTile, u = q % kPhTile;
            prev[q] = u < ti ? Wp[(long long)c * N + i0 + u] : 0.0;
        }
        const int wlen = kPhTile + kPhThreads;
        for (int q = threadIdx.x; q < C * wlen; q += kPhThreads) {
            const int c = q / wlen, u = q % wlen;
            win[q] = Wr[(long long)c * N + (i0 + m0 + u) % N];
        }
        __syncthreads();
        if (m < N) {
            for (int u = 0; u < ti; ++u) {
                double d2 = 0.0;
                for (int c = 0; c < C; ++c) {
                    const double d = win[c * wlen + u + threadIdx.x] - prev[c * kPhTile + u];
                    d2 = fma(d, d, d2);
                }
                acc += sqrt(d2);
            }
        }
    }
    if (m < N) a.cost[(long long)al * N + m] = acc;
}

// Smallest cost per alignment, ties to the smallest shift.
__global__ void __launch_bounds__(256) k_phase_argmin(const double *cost, int N, int *shift) {
    __shared__ double bv[256];
    __shared__ int bi[256];
    const double *c = cost + (long long)blockIdx.x * N;
    double best = INFINITY;
    int idx = N;
    for (int m = threadIdx.x; m < N; m += 256) {
        const double v = c[m];
        if (v < best || (v == best && m < idx)) {
            best = v;
            idx = m;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const double ov = bv[threadIdx.x + s];
            const int oi = bi[threadIdx.x + s];
            if (ov < bv[threadIdx.x] || (ov == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = ov;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) shift[blockIdx.x] = bi[0] < N ? bi[0] : 0;
}

bool device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

tms_status fail(tms_status st, const std::string &msg) {
    tms::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" tms_status tms_theta_translate(const double *dIn, double *dOut, int N, int nCols,
                                          int nCoord, long long ldc, const double *dRho,
                                          double rho0, int derivative, void *stream) {
    if (N < 8 || N > 8192 || (N & (N - 1)))
        return fail(TMS_ERR_ARG, "tms_theta_translate: N must be a power of two in 8..8192");
    if (nCols < 0 || nCoord < 1 || (derivative != 0 && derivative != 1))
        return fail(TMS_ERR_ARG, "tms_theta_translate: bad nCols, nCoord or derivative");
    if (!dRho && !isfinite(rho0)) return fail(TMS_ERR_ARG, "tms_theta_translate: rho0 not finite");
    if (nCols == 0) return TMS_OK;
    if (ldc < (long long)nCols * N) return fail(TMS_ERR_ARG, "tms_theta_translate: ldc < nCols * N");
    if (!dIn || !dOut || !device_ptr(dIn) || !device_ptr(dOut) || (dRho && !device_ptr(dRho)))
        return fail(TMS_ERR_ARG, "tms_theta_translate: arrays must be device pointers");
    int logN = 0;
    while ((1 << logN) < N) ++logN;
    const size_t smem = (size_t)(N + N / 2 + 4 * kTab) * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_theta_fft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return fail(TMS_ERR_CUDA, cudaGetErrorString(e));
    ThetaArgs a;
    a.in = dIn;
    a.out = dOut;
    a.ldc = ldc;
    a.rho = dRho;
    a.rho0 = rho0;
    a.N = N;
    a.logN = logN;
    a.cols = nCols;
    a.ncoord = nCoord;
    a.derivative = derivative;
    const long long blocks = (long long)nCols * ((nCoord + 1) / 2);
    if (blocks > 0x7fffffffLL) return fail(TMS_ERR_ARG, "tms_theta_translate: too many columns");
    k_theta_fft<<<(unsigned)blocks, kFftThreads, smem, (cudaStream_t)stream>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TMS_ERR_CUDA, std::string("tms_theta_translate: ") +
                                                        cudaGetErrorString(e));
    return TMS_OK;
}

extern "C" tms_status tms_phase_align(const double *dWr, const double *dWprev, int N, int nCoord,
                                      int nAlign, double *dCost, int32_t *dShift, void *stream) {
    if (N < 1 || nCoord < 1 || nCoord > 8 || nAlign < 0)
        return fail(TMS_ERR_ARG, "tms_phase_align: need N >= 1, 1 <= nCoord <= 8, nAlign >= 0");
    if (nAlign == 0) return TMS_OK;
    if (!dWr || !dWprev || !dCost || !dShift || !device_ptr(dWr) || !device_ptr(dWprev) ||
        !device_ptr(dCost) || !device_ptr(dShift))
        return fail(TMS_ERR_ARG, "tms_phase_align: arrays must be device pointers");
    if (nAlign > 65535) return fail(TMS_ERR_ARG, "tms_phase_align: nAlign > 65535");
    const size_t smem = (size_t)nCoord * (2 * kPhTile + kPhThreads) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_phase_cost, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return fail(TMS_ERR_CUDA, cudaGetErrorString(e));
    PhaseArgs a;
    a.wr = dWr;
    a.wp = dWprev;
    a.cost = dCost;
    a.N = N;
    a.ncoord = nCoord;
    a.nalign = nAlign;
    dim3 grid((N + kPhThreads - 1) / kPhThreads, nAlign);
    k_phase_cost<<<grid, kPhThreads, smem, (cudaStream_t)stream>>>(a);
    k_phase_argmin<<<nAlign, 256, 0, (cudaStream_t)stream>>>(dCost, N, dShift);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TMS_ERR_CUDA, std::string("tms_phase_align: ") +
                                                        cudaGetErrorString(e));
    return TMS_OK;
}

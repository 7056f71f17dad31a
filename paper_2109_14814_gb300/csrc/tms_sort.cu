// Hand-written LSD radix sort of (uint64 key, uint32 value) pairs and
// exclusive scans, both with the element count read from device memory so that
// a whole search can be captured in a CUDA graph without host round trips.
//
// Sort: per 8-bit digit, three launches over a fixed persistent grid of G
// blocks, each block owning a contiguous chunk of 2048-key tiles:
//   upsweep   per-block digit histograms  -> counts[digit][block]
//   scan      one block: exclusive scan of counts in digit-major order
//   downsweep stable ranking of each tile (warp match on the digit + per-warp
//             running counts), scatter to base[digit][block] + running offset.
// Stability: a block visits its tiles in order, warps own consecutive slices
// of a tile, and lanes within a warp iteration are in index order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "tms_common.cuh"

namespace tms {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void chunk_of(unsigned long long n, int block, int grid,
                                         unsigned long long &t0, unsigned long long &t1) {
    unsigned long long tiles = (n + kSortTile - 1) / kSortTile;
    unsigned long long per = (tiles + grid - 1) / grid;
    t0 = per * block;
    t1 = t0 + per;
    if (t0 > tiles) t0 = tiles;
    if (t1 > tiles) t1 = tiles;
}

__global__ void __launch_bounds__(kSortBlock) k_radix_upsweep(const uint64_t *keys,
                                                               const unsigned long long *d_n,
                                                               unsigned long long cap, int shift,
                                                               uint32_t *counts) {
    __shared__ uint32_t hist[kRadixBins];
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) hist[d] = 0;
    __syncthreads();
    const unsigned long long n = clamp_count(d_n, cap);
    unsigned long long t0, t1;
    chunk_of(n, blockIdx.x, gridDim.x, t0, t1);
    unsigned long long beg = t0 * kSortTile, end = t1 * kSortTile;
    if (end > n) end = n;
    for (unsigned long long i = beg + threadIdx.x; i < end; i += blockDim.x) {
        uint32_t d = (uint32_t)(keys[i] >> shift) & (kRadixBins - 1);
        atomicAdd(&hist[d], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) counts[d * gridDim.x + blockIdx.x] = hist[d];
}

// exclusive scan of len values in place, one block of 1024 threads: chunks of
// 4096 values are staged in shared memory with coalesced loads and stores, each
// thread scans 4 consecutive values, and a warp-shuffle scan joins the threads
__global__ void __launch_bounds__(1024) k_scan_small(uint32_t *v, int len) {
    constexpr int CH = 4096;
    __shared__ uint32_t buf[CH];
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < len; base += CH) {
        for (int i = threadIdx.x; i < CH; i += blockDim.x) buf[i] = (base + i < len) ? v[base + i] : 0u;
        __syncthreads();
        const int o = 4 * threadIdx.x;
        const uint32_t a0 = buf[o], a1 = buf[o + 1], a2 = buf[o + 2], a3 = buf[o + 3];
        const uint32_t tot = a0 + a1 + a2 + a3;
        uint32_t incl = tot;
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
            uint32_t wi = w;
            for (int off = 1; off < 32; off <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, wi, off);
                if (lane >= off) wi += y;
            }
            wsum[lane] = wi - w;
        }
        __syncthreads();
        const uint32_t c0 = carry;
        const uint32_t ex = c0 + wsum[warp] + incl - tot;
        buf[o] = ex;
        buf[o + 1] = ex + a0;
        buf[o + 2] = ex + a0 + a1;
        buf[o + 3] = ex + a0 + a1 + a2;
        __syncthreads();
        for (int i = threadIdx.x; i < CH; i += blockDim.x)
            if (base + i < len) v[base + i] = buf[i];
        if (threadIdx.x == blockDim.x - 1) carry = ex + tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSortBlock) k_radix_downsweep(
    const uint64_t *keys_in, const uint32_t *vals_in, uint64_t *keys_out, uint32_t *vals_out,
    const unsigned long long *d_n, unsigned long long cap, int shift, const uint32_t *counts) {
    constexpr int NW = kSortBlock / 32;
    __shared__ uint32_t wcnt[NW][kRadixBins];
    __shared__ uint32_t base[kRadixBins];
    __shared__ uint32_t tile_tot[kRadixBins];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) base[d] = counts[d * gridDim.x + blockIdx.x];
    const unsigned long long n = clamp_count(d_n, cap);
    unsigned long long t0, t1;
    chunk_of(n, blockIdx.x, gridDim.x, t0, t1);
    const uint32_t lt = lanemask_lt();
    __syncthreads();
    for (unsigned long long tile = t0; tile < t1; ++tile) {
        const unsigned long long tbase = tile * kSortTile + (unsigned long long)warp * (32 * kSortItems);
        uint64_t k[kSortItems];
        uint32_t v[kSortItems];
        uint32_t dig[kSortItems];
        uint32_t rank[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            unsigned long long idx = tbase + (unsigned long long)j * 32 + lane;
            bool ok = idx < n;
            k[j] = ok ? keys_in[idx] : 0;
            v[j] = ok ? vals_in[idx] : 0;
            dig[j] = ok ? ((uint32_t)(k[j] >> shift) & (kRadixBins - 1)) : 0xFFFFu;
        }
        for (int d = lane; d < kRadixBins; d += 32) wcnt[warp][d] = 0;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t d = dig[j];
            const uint32_t peers = __match_any_sync(FULL, d);
            const bool ok = d != 0xFFFFu;
            uint32_t before = ok ? wcnt[warp][d] : 0;
            __syncwarp();
            const int leader = __ffs(peers) - 1;
            if (ok && lane == leader) wcnt[warp][d] = before + __popc(peers);
            __syncwarp();
            rank[j] = before + __popc(peers & lt);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) {
            uint32_t acc = 0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                uint32_t c = wcnt[w][d];
                wcnt[w][d] = acc;
                acc += c;
            }
            tile_tot[d] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t d = dig[j];
            if (d != 0xFFFFu) {
                const uint32_t pos = base[d] + wcnt[warp][d] + rank[j];
                keys_out[pos] = k[j];
                vals_out[pos] = v[j];
            }
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kRadixBins; d += blockDim.x) base[d] += tile_tot[d];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// exclusive scan (reduce, scan partials, downsweep) with a device-side count
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void scan_chunk(unsigned long long n, int block, int grid,
                                           unsigned long long &b, unsigned long long &e) {
    unsigned long long per = (n + grid - 1) / grid;
    per = (per + 31) & ~31ULL;
    b = per * block;
    e = b + per;
    if (b > n) b = n;
    if (e > n) e = n;
}

template <typename T>
__device__ __forceinline__ T block_reduce_sum(T x) {
    __shared__ T wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
    if (lane == 0) wsum[warp] = x;
    __syncthreads();
    T tot = 0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wsum[w];
        wsum[0] = tot;
    }
    __syncthreads();
    tot = wsum[0];
    __syncthreads();
    return tot;
}

template <typename T>
__global__ void __launch_bounds__(kScanBlock) k_scan_reduce(const T *in, const unsigned long long *d_n,
                                                            unsigned long long cap,
                                                            unsigned long long *partials) {
    const unsigned long long n = clamp_count(d_n, cap);
    unsigned long long b, e;
    scan_chunk<T>(n, blockIdx.x, gridDim.x, b, e);
    unsigned long long s = 0;
    for (unsigned long long i = b + threadIdx.x; i < e; i += blockDim.x) s += (unsigned long long)in[i];
    s = block_reduce_sum<unsigned long long>(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_scan_partials(unsigned long long *partials, int g,
                                                        unsigned long long *d_total) {
    __shared__ unsigned long long p[1024];
    unsigned long long x = threadIdx.x < g ? partials[threadIdx.x] : 0;
    p[threadIdx.x] = x;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        unsigned long long y = threadIdx.x >= off ? p[threadIdx.x - off] : 0;
        __syncthreads();
        p[threadIdx.x] += y;
        __syncthreads();
    }
    if (threadIdx.x < g) partials[threadIdx.x] = p[threadIdx.x] - x;
    if (threadIdx.x == blockDim.x - 1 && d_total) *d_total = p[threadIdx.x];
}

template <typename T, typename O>
__global__ void __launch_bounds__(kScanBlock) k_scan_down(const T *in, O *out,
                                                          const unsigned long long *d_n,
                                                          unsigned long long cap,
                                                          const unsigned long long *partials) {
    __shared__ unsigned long long wsum[kScanBlock / 32];
    __shared__ unsigned long long carry;
    const unsigned long long n = clamp_count(d_n, cap);
    unsigned long long b, e;
    scan_chunk<T>(n, blockIdx.x, gridDim.x, b, e);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = partials[blockIdx.x];
    __syncthreads();
    for (unsigned long long base = b; base < e; base += blockDim.x) {
        unsigned long long i = base + threadIdx.x;
        unsigned long long x = (i < e) ? (unsigned long long)in[i] : 0;
        unsigned long long incl = x;
        for (int off = 1; off < 32; off <<= 1) {
            unsigned long long y = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
            unsigned long long wi = w;
            for (int off = 1; off < 32; off <<= 1) {
                unsigned long long y = __shfl_up_sync(FULL, wi, off);
                if (lane >= off) wi += y;
            }
            if (lane < (int)(blockDim.x >> 5)) wsum[lane] = wi - w;
        }
        __syncthreads();
        unsigned long long c = carry;
        if (i < e) out[i] = (O)(c + wsum[warp] + incl - x);
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + wsum[warp] + incl;
        __syncthreads();
    }
}

}  // namespace

size_t radix_counts_size(int grid) { return (size_t)kRadixBins * grid * sizeof(uint32_t); }

bool radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                uint32_t *counts, const unsigned long long *d_n, unsigned long long cap,
                int key_bits, int grid, cudaStream_t st) {
    int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    if (passes < 1) passes = 1;
    uint64_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int p = 0; p < passes; ++p) {
        const int shift = p * kRadixBits;
        k_radix_upsweep<<<grid, kSortBlock, 0, st>>>(ki, d_n, cap, shift, counts);
        k_scan_small<<<1, 1024, 0, st>>>(counts, kRadixBins * grid);
        k_radix_downsweep<<<grid, kSortBlock, 0, st>>>(ki, vi, ko, vo, d_n, cap, shift, counts);
        uint64_t *tk = ki; ki = ko; ko = tk;
        uint32_t *tv = vi; vi = vo; vo = tv;
    }
    return (passes & 1) != 0;
}

void scan_u32(const uint32_t *in, uint32_t *out, const unsigned long long *d_n,
              unsigned long long cap, unsigned long long *partials, unsigned long long *d_total,
              int grid, cudaStream_t st) {
    k_scan_reduce<uint32_t><<<grid, kScanBlock, 0, st>>>(in, d_n, cap, partials);
    k_scan_partials<<<1, 1024, 0, st>>>(partials, grid, d_total);
    k_scan_down<uint32_t, uint32_t><<<grid, kScanBlock, 0, st>>>(in, out, d_n, cap, partials);
}

void scan_u64(const unsigned long long *in, unsigned long long *out,
              const unsigned long long *d_n, unsigned long long cap,
              unsigned long long *partials, unsigned long long *d_total, int grid,
              cudaStream_t st) {
    k_scan_reduce<unsigned long long><<<grid, kScanBlock, 0, st>>>(in, d_n, cap, partials);
    k_scan_partials<<<1, 1024, 0, st>>>(partials, grid, d_total);
    k_scan_down<unsigned long long, unsigned long long><<<grid, kScanBlock, 0, st>>>(in, out, d_n, cap,
                                                                                    partials);
}

}  // namespace tms

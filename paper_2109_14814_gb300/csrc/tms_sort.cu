// Hand-written LSD radix sort of (uint64 key, uint32 value) pairs and
// exclusive scans, both with the element count read from device memory so that
// a whole search can be captured in a CUDA graph without host round trips.
//
// Sort (one sweep per kRadixBits-bit digit):
//   k_radix_hist   one read of the keys: the digit histograms of every pass,
//                  and the look-back words of the tiles in use cleared;
//   k_radix_bases  per pass, the exclusive scan of the digit counts (the
//                  global start of every digit);
//   k_radix_pass   per pass, persistent blocks take 2048-key tiles in order
//                  from an atomic counter; a tile is ranked (warp match on the
//                  digit + per-warp counts), publishes its digit counts, finds
//                  the counts of all earlier tiles by decoupled look-back,
//                  reorders itself by digit in shared memory, and writes every
//                  digit run to its place with consecutive threads on
//                  consecutive addresses.
// Stability: tiles are numbered in key order, warps own consecutive slices of
// a tile, and lanes within a warp iteration are in index order.
// A look-back wait on a tile that never publishes gives up after spin_limit
// polls and sets ST_TIMEOUT in the caller's status word; its tile's offsets are
// then wrong, so every write is checked against the element count and the
// kernel runs on to its end.  A test switch (`unpublished`) makes the look-back
// read every earlier tile as not yet published, so that this path runs on the
// device without any fault.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "tms_common.cuh"

namespace tms {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kMaxPasses = 8;                        // 64-bit keys
constexpr uint64_t kFlagAgg = 1ull << 62;            // the tile's own count
constexpr uint64_t kFlagInc = 2ull << 62;            // count of this and all earlier tiles
constexpr uint64_t kCountMask = (1ull << 62) - 1;

// scratch layout: hist[kMaxPasses][kRadixBins] (u32), tile counters[kMaxPasses] (u32),
// then per pass the look-back words of every tile, tiles x kRadixBins (u64)
constexpr size_t kHistBytes = (size_t)kMaxPasses * kRadixBins * sizeof(uint32_t);
constexpr size_t kHeadBytes = kHistBytes + 256;

__host__ __device__ inline unsigned long long tiles_for(unsigned long long cap) {
    return cap == 0 ? 1 : (cap + kSortTile - 1) / kSortTile;
}

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t *p) {
    return *reinterpret_cast<const volatile uint64_t *>(p);
}
__device__ __forceinline__ void st_volatile_u64(uint64_t *p, uint64_t v) {
    *reinterpret_cast<volatile uint64_t *>(p) = v;
}

__global__ void __launch_bounds__(kSortBlock) k_radix_hist(const uint64_t *keys,
                                                            const unsigned long long *d_n,
                                                            unsigned long long cap, int passes,
                                                            uint32_t *hist, uint64_t *look,
                                                            unsigned long long tiles_cap) {
    __shared__ uint32_t h[kMaxPasses][kRadixBins];
    for (int i = threadIdx.x; i < kMaxPasses * kRadixBins; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const unsigned long long n = clamp_count(d_n, cap);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += stride) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(uint32_t)(k >> (p * kRadixBits)) & (kRadixBins - 1)], 1u);
    }
    // clear the look-back words of the tiles this sort uses
    const unsigned long long words = tiles_for(n) * kRadixBins;
    for (int p = 0; p < passes; ++p) {
        uint64_t *lp = look + (size_t)p * tiles_cap * kRadixBins;
        for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < words;
             i += stride)
            lp[i] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadixBins; i += blockDim.x) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
}

// per pass, exclusive scan of the digit counts in place (one block, a thread a digit)
__global__ void __launch_bounds__(kRadixBins) k_radix_bases(uint32_t *hist, int passes) {
    __shared__ uint32_t wsum[kRadixBins / 32];
    const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
    for (int p = 0; p < passes; ++p) {
        const uint32_t c = hist[p * kRadixBins + d];
        uint32_t incl = c;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        hist[p * kRadixBins + d] = before + incl - c;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kSortBlock) k_radix_pass(
    const uint64_t *keys_in, const uint32_t *vals_in, uint64_t *keys_out, uint32_t *vals_out,
    const unsigned long long *d_n, unsigned long long cap, int shift, const uint32_t *base,
    uint64_t *look, uint32_t *tile_ctr, unsigned int *status, unsigned long long spin_limit,
    int unpublished) {
    static_assert(kSortBlock == kRadixBins, "one thread per digit");
    constexpr int NW = kSortBlock / 32;
    __shared__ uint16_t wcnt[NW][kRadixBins];   // per-warp digit counts, then offsets (< kSortTile)
    __shared__ uint32_t t_excl[kRadixBins];     // start of each digit's run in the tile
    __shared__ uint32_t g_off[kRadixBins];      // global start of that run
    __shared__ uint32_t wsum[NW];
    __shared__ uint64_t sk[kSortTile];
    __shared__ uint32_t sv[kSortTile];
    __shared__ uint32_t s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int dme = threadIdx.x;                 // the digit this thread speaks for
    const unsigned long long n = clamp_count(d_n, cap);
    const unsigned long long ntiles = (n + kSortTile - 1) / kSortTile;
    const uint32_t lt = lanemask_lt();
    const uint32_t my_base = base[dme];
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
        __syncthreads();
        const unsigned long long tile = s_tile;
        if (tile >= ntiles) break;
        const unsigned long long t0 = tile * kSortTile;
        const uint32_t tile_n = (uint32_t)min((unsigned long long)kSortTile, n - t0);
        // ---- load this warp's slice and rank it
        const unsigned long long wbase = t0 + (unsigned long long)warp * (32 * kSortItems);
        uint64_t k[kSortItems];
        uint32_t v[kSortItems], dig[kSortItems], rank[kSortItems];
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const unsigned long long idx = wbase + (unsigned long long)j * 32 + lane;
            const bool ok = idx < n;
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
            const uint32_t before = ok ? wcnt[warp][d] : 0;
            __syncwarp();
            if (ok && lane == __ffs(peers) - 1) wcnt[warp][d] = before + __popc(peers);
            __syncwarp();
            rank[j] = before + __popc(peers & lt);
        }
        __syncthreads();
        // ---- per digit: offsets across warps and the tile's count
        uint32_t cnt = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t c = wcnt[w][dme];
            wcnt[w][dme] = cnt;
            cnt += c;
        }
        // publish the count at once, so that later tiles never wait on this
        // tile's own look-back
        uint64_t *my_word = look + tile * kRadixBins + dme;
        st_volatile_u64(my_word, (tile == 0 ? kFlagInc : kFlagAgg) | (uint64_t)cnt);
        // start of each digit's run in the tile (block scan over digits)
        uint32_t incl = cnt;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        // decoupled look-back over the earlier tiles, four words per poll
        uint64_t prefix = 0;
        if (tile > 0) {
            long long t = (long long)tile - 1;
            unsigned long long spins = 0;
            bool done = false;
            while (!done) {
                uint64_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    w[q] = (t - q >= 0) ? ld_volatile_u64(look + (t - q) * kRadixBins + dme) : kFlagInc;
                int used = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (done || used < q) continue;        // stop at a gap or an inclusive count
                    const uint64_t flag = unpublished ? 0 : (w[q] & ~kCountMask);
                    if (flag == 0) continue;               // not yet published: poll again from here
                    if (t - q >= 0) prefix += w[q] & kCountMask;
                    ++used;
                    if (flag == kFlagInc || t - q <= 0) done = true;
                }
                t -= used;
                if (!done && used == 0) {
                    if (++spins > spin_limit) {
                        atomicOr(status, ST_TIMEOUT);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            st_volatile_u64(my_word, kFlagInc | (prefix + cnt));
        }
        g_off[dme] = my_base + (uint32_t)prefix;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        t_excl[dme] = before + incl - cnt;
        __syncthreads();
        // ---- reorder the tile by digit in shared memory
#pragma unroll
        for (int j = 0; j < kSortItems; ++j) {
            const uint32_t d = dig[j];
            if (d != 0xFFFFu) {
                const uint32_t pos = t_excl[d] + wcnt[warp][d] + rank[j];
                sk[pos] = k[j];
                sv[pos] = v[j];
            }
        }
        __syncthreads();
        // ---- write the digit runs: consecutive threads, consecutive addresses
        for (uint32_t i = threadIdx.x; i < tile_n; i += kSortBlock) {
            const uint64_t key = sk[i];
            const uint32_t d = (uint32_t)(key >> shift) & (kRadixBins - 1);
            const uint32_t out = g_off[d] + (i - t_excl[d]);
            // in bounds whenever every look-back completed; a wait that gave up
            // leaves wrong offsets, which must not reach memory
            if (out < n) {
                keys_out[out] = key;
                vals_out[out] = sv[i];
            }
        }
        __syncthreads();
    }
}

}  // namespace

size_t radix_scratch_size(unsigned long long cap, int key_bits) {
    int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    if (passes < 1) passes = 1;
    return kHeadBytes + (size_t)passes * tiles_for(cap) * kRadixBins * sizeof(uint64_t);
}

bool radix_sort(uint64_t *keys, uint32_t *vals, uint64_t *keys_alt, uint32_t *vals_alt,
                void *scratch, const unsigned long long *d_n, unsigned long long cap,
                int key_bits, int grid, unsigned int *status, unsigned long long spin_limit,
                int unpublished, cudaStream_t st) {
    if (spin_limit == 0) spin_limit = kDefaultSpinLimit;
    int passes = (key_bits + kRadixBits - 1) / kRadixBits;
    if (passes < 1) passes = 1;
    if (passes > kMaxPasses) passes = kMaxPasses;
    unsigned char *sc = static_cast<unsigned char *>(scratch);
    uint32_t *hist = reinterpret_cast<uint32_t *>(sc);
    uint32_t *tile_ctr = reinterpret_cast<uint32_t *>(sc + kHistBytes);
    uint64_t *look = reinterpret_cast<uint64_t *>(sc + kHeadBytes);
    const unsigned long long tcap = tiles_for(cap);
    const int pgrid = (int)std::min<unsigned long long>((unsigned long long)grid, tcap);
    cudaMemsetAsync(sc, 0, kHeadBytes, st);
    k_radix_hist<<<grid, kSortBlock, 0, st>>>(keys, d_n, cap, passes, hist, look, tcap);
    k_radix_bases<<<1, kRadixBins, 0, st>>>(hist, passes);
    uint64_t *ki = keys, *ko = keys_alt;
    uint32_t *vi = vals, *vo = vals_alt;
    for (int p = 0; p < passes; ++p) {
        k_radix_pass<<<pgrid, kSortBlock, 0, st>>>(ki, vi, ko, vo, d_n, cap, p * kRadixBits,
                                                   hist + p * kRadixBins,
                                                   look + (size_t)p * tcap * kRadixBins,
                                                   tile_ctr + p, status, spin_limit, unpublished);
        uint64_t *tk = ki; ki = ko; ko = tk;
        uint32_t *tv = vi; vi = vo; vo = tv;
    }
    return (passes & 1) != 0;
}

namespace {

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

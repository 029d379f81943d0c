// prepass.cu -- per-image level tables for the hierarchical kernels.
//
// Uniform tree (Section III, uniform IOT): the tree needs only the effective
// bit depth d of the data (height d+1), so one max/min reduction suffices.
//
// Adaptive tree (Section III-C): the top-level interval boundaries follow a
// frequency model that mixes 1:1 the source's global histogram (value
// insertions/removals) and a histogram of a median estimate (order-statistic
// requests).  The median estimate is the global histogram of 8x8 block means,
// the "running mean as a first approximation" the paper suggests.  A small
// uniform floor (1/64 of the mass) spreads boundaries over value ranges the
// mix does not cover, so that without information the tree stays uniform
// ("where the mix vanishes, divide equally").  The 16 top-level boundaries
// are the equal-mass quantiles of the mix, so that every top-level child is
// visited about equally often (the paper's optimality condition).  Any
// boundaries give the same filter output; only the speed changes.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "hist_common.cuh"

namespace hrm {

constexpr int PREHIST_BINS = 4096;

// One level descriptor (and, for adaptive, its two histograms) reset.
__global__ void levels_init_kernel(LevelDesc* d, int mode, uint32_t* hist) {
    if (threadIdx.x == 0) {
        d->mode = (uint32_t)mode;
        d->vmin = 0xFFFFFFFFu;
        d->vmax = 0;
        d->count = 0;
    }
    if (hist)
        for (int i = threadIdx.x; i < 2 * PREHIST_BINS; i += blockDim.x) hist[i] = 0;
}

template <typename T>
__global__ void minmax_kernel(const unsigned char* __restrict__ src, size_t sp, size_t slice, int W,
                              int H, int D, LevelDesc* d) {
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    const long rows = (long)H * D;
    const int lane = threadIdx.x & 31;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    for (long row = warp; row < rows; row += nwarps) {
        const int z = (int)(row / H), y = (int)(row % H);
        const T* p = reinterpret_cast<const T*>(src + (size_t)z * slice + (size_t)y * sp);
        for (int x = lane; x < W; x += 32) {
            uint32_t v = __ldg(p + x);
            lo = min(lo, v);
            hi = max(hi, v);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
        atomicMin(&d->vmin, lo);
        atomicMax(&d->vmax, hi);
    }
}

__device__ __forceinline__ uint32_t prehist_binw(const LevelDesc* d) {
    uint32_t span = d->vmax - d->vmin + 1;
    return (span + PREHIST_BINS - 1) / PREHIST_BINS;
}

// Source histogram and 8x8-block-mean histogram (shared-memory privatised).
template <typename T>
__global__ void prehist_kernel(const unsigned char* __restrict__ src, size_t sp, size_t slice, int W,
                               int H, int D, const LevelDesc* d, uint32_t* hist) {
    __shared__ uint32_t hs[PREHIST_BINS];
    __shared__ uint32_t he[PREHIST_BINS];
    for (int i = threadIdx.x; i < PREHIST_BINS; i += blockDim.x) hs[i] = he[i] = 0;
    __syncthreads();
    const uint32_t vmin = d->vmin;
    const uint32_t binw = prehist_binw(d);
    const int bx = (W + 7) / 8, by = (H + 7) / 8;
    const long nblk = (long)bx * by * D;
    for (long b = (long)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (long)gridDim.x * blockDim.x) {
        const int z = (int)(b / ((long)bx * by));
        const long rem = b % ((long)bx * by);
        const int y0 = (int)(rem / bx) * 8, x0 = (int)(rem % bx) * 8;
        uint32_t sum = 0, cnt = 0;
        for (int y = y0; y < min(y0 + 8, H); ++y) {
            const T* p = reinterpret_cast<const T*>(src + (size_t)z * slice + (size_t)y * sp);
            for (int x = x0; x < min(x0 + 8, W); ++x) {
                uint32_t v = __ldg(p + x);
                sum += v;
                ++cnt;
                atomicAdd(&hs[(v - vmin) / binw], 1u);
            }
        }
        const uint32_t mean = (sum + cnt / 2) / cnt;
        atomicAdd(&he[(mean - vmin) / binw], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < PREHIST_BINS; i += blockDim.x) {
        if (hs[i]) atomicAdd(&hist[i], hs[i]);
        if (he[i]) atomicAdd(&hist[PREHIST_BINS + i], he[i]);
    }
}

// Equal-mass quantile boundaries of the 1:1 mix (one block of 1024 threads).
__global__ void __launch_bounds__(1024) edges_kernel(LevelDesc* d, const uint32_t* hist) {
    __shared__ unsigned long long cum[PREHIST_BINS + 1];
    __shared__ unsigned long long part[1024];
    __shared__ unsigned long long totals[2];
    const int t = threadIdx.x;
    // totals of both histograms
    unsigned long long a = 0, b = 0;
    for (int i = t; i < PREHIST_BINS; i += 1024) {
        a += hist[i];
        b += hist[PREHIST_BINS + i];
    }
    part[t] = a;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (t < s) part[t] += part[t + s];
        __syncthreads();
    }
    if (t == 0) totals[0] = part[0];
    __syncthreads();
    part[t] = b;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (t < s) part[t] += part[t + s];
        __syncthreads();
    }
    if (t == 0) totals[1] = part[0];
    __syncthreads();
    const unsigned long long A = totals[0] ? totals[0] : 1, B = totals[1] ? totals[1] : 1;
    const unsigned long long floor_w = (2ull * A * B) / (64ull * PREHIST_BINS) + 1;
    // per-thread local sums of 4 consecutive bins, then a block scan
    unsigned long long m[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        int i = 4 * t + k;
        m[k] = (unsigned long long)hist[i] * B + (unsigned long long)hist[PREHIST_BINS + i] * A + floor_w;
        s += m[k];
    }
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        unsigned long long v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned long long run = part[t] - s;  // exclusive prefix
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cum[4 * t + k] = run;
        run += m[k];
    }
    if (t == 1023) cum[PREHIST_BINS] = run;
    __syncthreads();
    const unsigned long long total = cum[PREHIST_BINS];
    const uint32_t vmin = d->vmin, vmax = d->vmax, binw = prehist_binw(d);
    if (t <= 16) {
        uint32_t e;
        if (t == 0) {
            e = vmin;
        } else if (t == 16) {
            e = vmax + 1;
        } else {
            // smallest bin boundary i with cum[i] >= t/16 of the mass
            unsigned long long target = (total * (unsigned long long)t) / 16;
            int lo = 0, hi = PREHIST_BINS;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (cum[mid] >= target) hi = mid; else lo = mid + 1;
            }
            unsigned long long ev = (unsigned long long)vmin + (unsigned long long)lo * binw;
            e = (uint32_t)min(ev, (unsigned long long)vmax + 1);
            e = max(e, vmin);
        }
        d->edge[t] = e;
    }
    if (t == 0) d->mode = 1;
}

cudaError_t launch_levels(int elem, bool adaptive, const void* src, size_t sp, size_t slice, int W,
                          int H, int D, LevelDesc* desc, uint32_t* hist, int num_sms,
                          cudaStream_t st) {
    levels_init_kernel<<<1, 256, 0, st>>>(desc, adaptive ? 1 : 0, adaptive ? hist : nullptr);
    const long rows = (long)H * D;
    int blocks = (int)std::min<long>((rows + 7) / 8, (long)num_sms * 8);
    if (blocks < 1) blocks = 1;
    auto s = (const unsigned char*)src;
    if (elem == 1) minmax_kernel<uint8_t><<<blocks, 256, 0, st>>>(s, sp, slice, W, H, D, desc);
    else minmax_kernel<uint16_t><<<blocks, 256, 0, st>>>(s, sp, slice, W, H, D, desc);
    if (adaptive) {
        long nblk = (long)((W + 7) / 8) * ((H + 7) / 8) * D;
        int hb = (int)std::min<long>((nblk + 255) / 256, (long)num_sms * 2);
        if (hb < 1) hb = 1;
        if (elem == 1) prehist_kernel<uint8_t><<<hb, 256, 0, st>>>(s, sp, slice, W, H, D, desc, hist);
        else prehist_kernel<uint16_t><<<hb, 256, 0, st>>>(s, sp, slice, W, H, D, desc, hist);
        edges_kernel<<<1, 1024, 0, st>>>(desc, hist);
    }
    return cudaGetLastError();
}

}  // namespace hrm

namespace hrm {

// Adaptive boundaries for a descriptor whose value range is already known
// (the batched pre-pass computes the ranges of all jobs in one launch).
cudaError_t launch_levels_adaptive_only(int elem, const void* src, size_t sp, size_t slice, int W, int H,
                                        int D, LevelDesc* desc, uint32_t* hist, int num_sms,
                                        cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 2 * PREHIST_BINS, st);
    if (e != cudaSuccess) return e;
    auto s = (const unsigned char*)src;
    long nblk = (long)((W + 7) / 8) * ((H + 7) / 8) * D;
    int hb = (int)std::min<long>((nblk + 255) / 256, (long)num_sms * 2);
    if (hb < 1) hb = 1;
    if (elem == 1) prehist_kernel<uint8_t><<<hb, 256, 0, st>>>(s, sp, slice, W, H, D, desc, hist);
    else prehist_kernel<uint16_t><<<hb, 256, 0, st>>>(s, sp, slice, W, H, D, desc, hist);
    edges_kernel<<<1, 1024, 0, st>>>(desc, hist);
    return cudaGetLastError();
}

}  // namespace hrm

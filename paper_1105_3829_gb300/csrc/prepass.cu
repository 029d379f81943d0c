// prepass.cu -- per-image level tables for the hierarchical kernels.
//
// Uniform tree (Section III, uniform IOT): the tree needs only the effective
// bit depth d of the data (height d+1), so one max/min reduction suffices.
//
// Adaptive tree (Section III-C): the top level is fitted to where the
// order-statistic requests go, using a median estimate of the image -- here
// the histogram of the medians of its 4x4 blocks (the paper suggests a
// smoothed median of a typical image; block medians are robust to outliers,
// where a running mean is not).  The central range holding 99 % of the
// estimate gets 14 or 15 top-level intervals of one width w = 16^k, aligned
// to w, so every sub-tree below them is a full 16-ary tree of k levels; the
// values below and above the central range share the remaining one or two
// (deep, rarely walked) intervals.  On this GPU design the cost of a row is
// the number of distinct nodes its outputs visit per level, so the paper's
// equal-visit split of the top level (which narrows top intervals around the
// mode and leaves 1-3 bit leaf levels) is replaced by this power-of-16 split;
// when w is not narrower than the uniform tree's top intervals the uniform
// tree is kept.  Any boundaries give the same filter output; only the speed
// changes.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "hist_common.cuh"
#include "sortnet.cuh"

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

// Histogram of 4x4 block medians (the lower median, 8th smallest of 16),
// shared-memory privatised; partial blocks at the right and bottom edges
// are skipped.
template <typename T>
__global__ void prehist_kernel(const unsigned char* __restrict__ src, size_t sp, size_t slice, int W,
                               int H, int D, const LevelDesc* d, uint32_t* hist) {
    __shared__ uint32_t he[PREHIST_BINS];
    for (int i = threadIdx.x; i < PREHIST_BINS; i += blockDim.x) he[i] = 0;
    __syncthreads();
    const uint32_t vmin = d->vmin;
    const uint32_t binw = prehist_binw(d);
    const int bx = W / 4, by = H / 4;
    const long nblk = (long)bx * by * D;
    for (long b = (long)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (long)gridDim.x * blockDim.x) {
        const int z = (int)(b / ((long)bx * by));
        const long rem = b % ((long)bx * by);
        const int y0 = (int)(rem / bx) * 4, x0 = (int)(rem % bx) * 4;
        uint32_t v[16];
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const T* p = reinterpret_cast<const T*>(src + (size_t)z * slice + (size_t)(y0 + y) * sp) + x0;
#pragma unroll
            for (int x = 0; x < 4; ++x) v[4 * y + x] = __ldg(p + x);
        }
        sortnet<16>(v);  // values < 2^16: the packed-pair min/max act on the low half
        atomicAdd(&he[(v[7] - vmin) / binw], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < PREHIST_BINS; i += blockDim.x)
        if (he[i]) atomicAdd(&hist[i], he[i]);
}

// Top-level boundaries from the block-median histogram (one block of 1024
// threads): the 0.5 % and 99.5 % quantiles bound the central range.
__global__ void __launch_bounds__(1024) edges_kernel(LevelDesc* d, const uint32_t* hist) {
    __shared__ uint32_t cum[PREHIST_BINS + 1];
    __shared__ uint32_t part[1024];
    const int t = threadIdx.x;
    uint32_t m[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        m[k] = hist[4 * t + k];
        s += m[k];
    }
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const uint32_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - s;  // exclusive prefix
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cum[4 * t + k] = run;
        run += m[k];
    }
    if (t == 1023) cum[PREHIST_BINS] = run;
    __syncthreads();
    if (t != 0) return;
    const uint32_t total = cum[PREHIST_BINS];
    const uint32_t vmin = d->vmin, vmax = d->vmax, binw = prehist_binw(d);
    const int ushift = max(0, bitlen(vmax) - 4);
    if (total == 0) {  // no full 4x4 block: keep the uniform tree
        d->mode = 0;
        return;
    }
    // bin a holds the 0.5 % quantile (cum[a] <= lo_t < cum[a+1]), bin b the
    // 99.5 % one (cum[b] < hi_t <= cum[b+1]); cum is non-decreasing
    const uint64_t lo_t = (uint64_t)total * 5 / 1000, hi_t = (uint64_t)total * 995 / 1000;
    int lo = 0, hi = PREHIST_BINS - 1;
    while (lo < hi) {  // first i with cum[i+1] > lo_t
        const int mid = (lo + hi) >> 1;
        if (cum[mid + 1] > lo_t) hi = mid; else lo = mid + 1;
    }
    const int a = lo;
    lo = a;
    hi = PREHIST_BINS - 1;
    while (lo < hi) {  // last i with cum[i] < hi_t
        const int mid = (lo + hi + 1) >> 1;
        if (cum[mid] < hi_t) lo = mid; else hi = mid - 1;
    }
    const int b = lo;
    const uint64_t av = (uint64_t)vmin + (uint64_t)a * binw;
    uint64_t bv = (uint64_t)vmin + (uint64_t)(b + 1) * binw - 1;
    if (bv > vmax) bv = vmax;
    if (bv < av) {  // cannot happen for a histogram of values in [vmin, vmax]; keep the uniform tree
        d->mode = 0;
        return;
    }
    // smallest w = 16^k with 13 w >= the central range (one interval of slack for the alignment)
    uint64_t w = 16;
    while (w < (1ull << 32) && 13 * w < bv - av + 1) w <<= 4;
    if (ushift <= 0 || w >= (1ull << ushift)) {  // not finer than the uniform tree
        d->mode = 0;
        return;
    }
    const uint64_t base = (av / w) * w;
    const uint64_t top = (uint64_t)vmax + 1;
    uint64_t e[17];
    e[0] = vmin;
    int c = 1;
    if (base > vmin) e[c++] = base;
    for (uint64_t i = 1; c < 16; ++i) e[c++] = base + i * w < top ? base + i * w : top;
    e[16] = top;
    for (int k = 0; k <= 16; ++k) d->edge[k] = (uint32_t)(e[k] < top ? e[k] : top);
    d->mode = 1;
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

namespace hrm {

// Histogram of a filtered frame's values over the whole dtype range (the
// descriptor's vmin/vmax are set to 0 and 2^bits - 1 first).
template <typename T>
__global__ void outhist_kernel(const unsigned char* __restrict__ img, size_t pitch, int W, int H,
                               const LevelDesc* d, uint32_t* hist) {
    __shared__ uint32_t hs[PREHIST_BINS];
    for (int i = threadIdx.x; i < PREHIST_BINS; i += blockDim.x) hs[i] = 0;
    __syncthreads();
    const uint32_t binw = prehist_binw(d);
    const int lane = threadIdx.x & 31;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    for (long y = warp; y < H; y += nwarps) {
        const T* p = reinterpret_cast<const T*>(img + (size_t)y * pitch);
        for (int x = lane; x < W; x += 32) atomicAdd(&hs[(uint32_t)__ldg(p + x) / binw], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < PREHIST_BINS; i += blockDim.x)
        if (hs[i]) atomicAdd(&hist[i], hs[i]);
}

__global__ void full_range_kernel(LevelDesc* d, int elem) {
    if (threadIdx.x == 0) {
        d->vmin = 0;
        d->vmax = elem == 2 ? 65535u : 255u;
    }
}

cudaError_t launch_topology_from_output(int elem, const void* dst, size_t dp, int W, int H, LevelDesc* desc,
                                        uint32_t* hist, int num_sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * PREHIST_BINS, st);
    if (e != cudaSuccess) return e;
    full_range_kernel<<<1, 32, 0, st>>>(desc, elem);
    int blocks = (int)std::min<long>(((long)H + 7) / 8, (long)num_sms * 2);
    if (blocks < 1) blocks = 1;
    auto s = (const unsigned char*)dst;
    if (elem == 1) outhist_kernel<uint8_t><<<blocks, 256, 0, st>>>(s, dp, W, H, desc, hist);
    else outhist_kernel<uint16_t><<<blocks, 256, 0, st>>>(s, dp, W, H, desc, hist);
    edges_kernel<<<1, 1024, 0, st>>>(desc, hist);
    return cudaGetLastError();
}

}  // namespace hrm

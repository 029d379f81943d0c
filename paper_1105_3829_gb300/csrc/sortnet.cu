// sortnet.cu -- launch wrappers for the selection networks (2D radius 1..5, 3D radius 1).
#include "sortnet.cuh"

namespace hrm {

template <typename T, int R>
__global__ void __launch_bounds__(128) sortnet_kernel(const unsigned char* __restrict__ src, size_t sp,
                                                      unsigned char* __restrict__ dst, size_t dp, int W,
                                                      int H, int rows_per_warp) {
    const int ty = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (R == 1) sortnet3x3_tile<T>(src, sp, dst, dp, W, H, rows_per_warp, blockIdx.x, ty);
    else if (R == 2) sortnet5x5_tile<T>(src, sp, dst, dp, W, H, rows_per_warp, blockIdx.x, ty);
    else sortnet_wide_tile<T, R>(src, sp, dst, dp, W, H, rows_per_warp, blockIdx.x, ty);
}

template <typename T>
__global__ void __launch_bounds__(128) sortnet3d_kernel(const unsigned char* __restrict__ src, size_t sp, size_t ss,
                                                        unsigned char* __restrict__ dst, size_t dp, size_t ds, int W,
                                                        int H, int D, int zn) {
    // grid: x = 256-column tiles, y = rows, z = groups of 4 slice runs (one per warp)
    const int tz = blockIdx.z * (blockDim.x >> 5) + (threadIdx.x >> 5);
    sortnet3d_tile<T>(src, sp, ss, dst, dp, ds, W, H, D, zn, blockIdx.x, blockIdx.y, tz);
}

cudaError_t launch_sortnet3d(int elem, const void* src, size_t sp, size_t ss, void* dst, size_t dp, size_t ds,
                             int W, int H, int D, int zn, cudaStream_t st) {
    if (zn <= 0) zn = 32;
    const int warps = 4;
    const int tz = (D + zn - 1) / zn;
    dim3 grid((W + 255) / 256, H, (tz + warps - 1) / warps);
    auto s = (const unsigned char*)src;
    auto d = (unsigned char*)dst;
    if (elem == 1) sortnet3d_kernel<uint8_t><<<grid, 32 * warps, 0, st>>>(s, sp, ss, d, dp, ds, W, H, D, zn);
    else sortnet3d_kernel<uint16_t><<<grid, 32 * warps, 0, st>>>(s, sp, ss, d, dp, ds, W, H, D, zn);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
cudaError_t launch_sortnet2d(int elem, int radius, const void* src, size_t sp, void* dst,
                             size_t dp, int W, int H, int rows_per_warp, cudaStream_t st) {
    if (rows_per_warp <= 0) rows_per_warp = 32;
    const int warps = 4;
    dim3 block(32 * warps);
    int tiles_y = (H + rows_per_warp - 1) / rows_per_warp;
    // columns per warp tile: 256 (r <= 2), else two per output lane
    const int tw = radius <= 2 ? 256 : 2 * (32 - 2 * ((radius + 1) / 2));
    dim3 grid((W + tw - 1) / tw, (tiles_y + warps - 1) / warps);
    auto s = (const unsigned char*)src;
    auto d = (unsigned char*)dst;
#define HRM_SORTNET_CASE(RR)                                                                            \
    case RR:                                                                                            \
        if (elem == 1) sortnet_kernel<uint8_t, RR><<<grid, block, 0, st>>>(s, sp, d, dp, W, H, rows_per_warp); \
        else sortnet_kernel<uint16_t, RR><<<grid, block, 0, st>>>(s, sp, d, dp, W, H, rows_per_warp);        \
        break;
    switch (radius) {
        HRM_SORTNET_CASE(1)
        HRM_SORTNET_CASE(2)
        HRM_SORTNET_CASE(3)
        HRM_SORTNET_CASE(4)
        HRM_SORTNET_CASE(5)
        default:
            return cudaErrorInvalidValue;
    }
#undef HRM_SORTNET_CASE
    return cudaGetLastError();
}

}  // namespace hrm

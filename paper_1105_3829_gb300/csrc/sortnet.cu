// sortnet.cu -- launch wrapper for the radius 1 / 2 selection networks.
#include "sortnet.cuh"

namespace hrm {

template <typename T, int R>
__global__ void __launch_bounds__(128) sortnet_kernel(const unsigned char* __restrict__ src, size_t sp,
                                                      unsigned char* __restrict__ dst, size_t dp, int W,
                                                      int H, int rows_per_warp) {
    const int ty = blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (R == 1) sortnet3x3_tile<T>(src, sp, dst, dp, W, H, rows_per_warp, blockIdx.x, ty);
    else sortnet5x5_tile<T>(src, sp, dst, dp, W, H, rows_per_warp, blockIdx.x, ty);
}

// ---------------------------------------------------------------------------
cudaError_t launch_sortnet2d(int elem, int radius, const void* src, size_t sp, void* dst,
                             size_t dp, int W, int H, int rows_per_warp, cudaStream_t st) {
    if (rows_per_warp <= 0) rows_per_warp = 32;
    const int warps = 4;
    dim3 block(32 * warps);
    int tiles_y = (H + rows_per_warp - 1) / rows_per_warp;
    dim3 grid((W + 255) / 256, (tiles_y + warps - 1) / warps);
    auto s = (const unsigned char*)src;
    auto d = (unsigned char*)dst;
    if (radius == 1) {
        if (elem == 1) sortnet_kernel<uint8_t, 1><<<grid, block, 0, st>>>(s, sp, d, dp, W, H, rows_per_warp);
        else sortnet_kernel<uint16_t, 1><<<grid, block, 0, st>>>(s, sp, d, dp, W, H, rows_per_warp);
    } else if (radius == 2) {
        if (elem == 1) sortnet_kernel<uint8_t, 2><<<grid, block, 0, st>>>(s, sp, d, dp, W, H, rows_per_warp);
        else sortnet_kernel<uint16_t, 2><<<grid, block, 0, st>>>(s, sp, d, dp, W, H, rows_per_warp);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hrm

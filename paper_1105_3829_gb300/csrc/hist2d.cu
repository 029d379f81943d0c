// hist2d.cu -- launch wrappers for the 2D hierarchical-histogram kernel.
#include <cstdint>
#include <cuda_runtime.h>

#include "hist2d.cuh"

namespace hrm {

template <typename T, int PPL>
__global__ void __launch_bounds__(32) hist2d_kernel(Hist2DJob job) {
    extern __shared__ __align__(16) unsigned char smem[];
    hist2d_tile<T, PPL>(job, (int)blockIdx.x, smem);
}

template <typename T, int PPL>
static cudaError_t launch_one(const Hist2DJob& job, size_t smem, cudaStream_t st) {
    auto fn = hist2d_kernel<T, PPL>;
    if (smem > 48 * 1024) {  // opt in per launch: the attribute is per device and cheap to set
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fn<<<job.ntiles, 32, smem, st>>>(job);
    return cudaGetLastError();
}

cudaError_t launch_hist2d(const Hist2DJob& job, cudaStream_t st) {
    const int tw = 32 * job.ppl;
    const size_t smem = hist2d_smem_bytes(tw, job.r, job.nslots);
    if (job.elem == 1) {
        switch (job.ppl) {
            case 2: return launch_one<uint8_t, 2>(job, smem, st);
            case 4: return launch_one<uint8_t, 4>(job, smem, st);
            case 8: return launch_one<uint8_t, 8>(job, smem, st);
        }
    } else {
        switch (job.ppl) {
            case 2: return launch_one<uint16_t, 2>(job, smem, st);
            case 4: return launch_one<uint16_t, 4>(job, smem, st);
            case 8: return launch_one<uint16_t, 8>(job, smem, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace hrm

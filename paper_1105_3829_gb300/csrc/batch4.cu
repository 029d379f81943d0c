// batch4.cu -- the persistent batch kernel compiled for four resident blocks
// per SM (128 registers), in its own translation unit so both register
// budgets compile in parallel.
#include "batch_kernel.cuh"

namespace hrm {

cudaError_t launch_batch_kernel4(unsigned grid, size_t smem, cudaStream_t st, const BatchItem* items,
                                 const unsigned* offs, int nitems, unsigned* counter, unsigned total) {
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(batch_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    batch_kernel<4><<<grid, BLOCK_THREADS, smem, st>>>(items, offs, nitems, counter, total);
    return cudaGetLastError();
}

}  // namespace hrm

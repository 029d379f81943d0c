// hist.cu -- launch wrappers for the hierarchical-histogram kernel (2D and 3D).
#include <cstdint>
#include <cuda_runtime.h>

#include "hist_tile.cuh"
#include "runtime.h"

namespace hrm {

// MINB = resident tiles per SM the register budget is sized for: 3 (up to
// 168 registers) by default, 4 (128 registers) when the plan's shared memory
// lets four tiles share an SM.
template <typename T, int PPL, int CW, int MINB, int DIMS, bool GRP = false>
__global__ void __launch_bounds__(BLOCK_THREADS, MINB) hist_kernel(HistJob job) {
    extern __shared__ __align__(16) unsigned char smem[];
    hist_tile<T, PPL, CW, DIMS, GRP>(job, (int)blockIdx.x, smem);
}

template <typename T, int PPL, int CW, int MINB>
static cudaError_t launch_one(const HistJob& job, size_t smem, cudaStream_t st) {
    // 2D windows of at most 31 columns (8 or more 8-bit column records per
    // packed-byte group of the direct sums) run the instance compiled for them
    const bool grp = PPL == 1 && CW == 1 && MINB == 4 && job.dims == 2 && 255 / (2 * job.r + 1) >= 8;
    auto fn = job.dims == 3 ? hist_kernel<T, PPL, CW, MINB, 3>
                            : (grp ? hist_kernel<T, PPL, CW, MINB, 2, PPL == 1 && CW == 1 && MINB == 4>
                                   : hist_kernel<T, PPL, CW, MINB, 2>);
    if (smem > 48 * 1024) {  // opt in per launch: the attribute is per device and cheap to set
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fn<<<job.ntiles, BLOCK_THREADS, smem, st>>>(job);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_t(const HistJob& job, size_t smem, bool four, cudaStream_t st) {
    if (job.cw == 1) {
        switch (job.ppl) {
            case 1: return four ? launch_one<T, 1, 1, 4>(job, smem, st) : launch_one<T, 1, 1, 3>(job, smem, st);
            case 2: return launch_one<T, 2, 1, 3>(job, smem, st);
        }
    } else if (job.cw == 2) {
        switch (job.ppl) {
            case 1: return four ? launch_one<T, 1, 2, 4>(job, smem, st) : launch_one<T, 1, 2, 3>(job, smem, st);
            case 2: return launch_one<T, 2, 2, 3>(job, smem, st);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_hist(const HistJob& job, cudaStream_t st) {
    const size_t smem = hist_smem_bytes(BLOCK_THREADS * job.ppl, job.r, job.nslots, job.cw, job.ring, job.elem);
    const DeviceInfo& di = device_info();
    const bool four = di.smem_per_sm / (long)(smem + 1024) >= 4;
    return job.elem == 1 ? launch_t<uint8_t>(job, smem, four, st) : launch_t<uint16_t>(job, smem, four, st);
}

}  // namespace hrm

#ifdef HRM_COUNT_OPS
// Instrumented builds only: read (and optionally clear) the device counters of
// the single-image histogram kernel.
extern "C" int hrm_debug_counters(unsigned long long* out, int n, int reset) {
    if (n > hrm::CNT_NUM) n = hrm::CNT_NUM;
    cudaDeviceSynchronize();
    if (cudaMemcpyFromSymbol(out, hrm::g_hrm_counters, sizeof(unsigned long long) * n) != cudaSuccess) return -3;
    if (reset) {
        unsigned long long z[hrm::CNT_NUM] = {};
        cudaMemcpyToSymbol(hrm::g_hrm_counters, z, sizeof(z));
    }
    return 0;
}

// Instrumented builds only: restrict the counters to one tile (-1 = all).
extern "C" int hrm_debug_count_tile(int tile) {
    return cudaMemcpyToSymbol(hrm::g_hrm_count_tile, &tile, sizeof(int)) == cudaSuccess ? 0 : -3;
}

// Instrumented builds only: per-tile start/end times (ns) and SM of the last launch.
extern "C" int hrm_debug_tiles(unsigned long long* t0, unsigned long long* t1, unsigned* sm, int n) {
    if (n > hrm::CNT_TILE_CAP) n = hrm::CNT_TILE_CAP;
    cudaDeviceSynchronize();
    if (cudaMemcpyFromSymbol(t0, hrm::g_hrm_tile_t0, sizeof(unsigned long long) * n) != cudaSuccess) return -3;
    if (cudaMemcpyFromSymbol(t1, hrm::g_hrm_tile_t1, sizeof(unsigned long long) * n) != cudaSuccess) return -3;
    if (cudaMemcpyFromSymbol(sm, hrm::g_hrm_tile_sm, sizeof(unsigned) * n) != cudaSuccess) return -3;
    return 0;
}
#endif

// batch_kernel.cuh -- the persistent batch kernel: item descriptors and the
// tile loop (shared by the two register-budget instantiations).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "hist_tile.cuh"
#include "sortnet.cuh"

namespace hrm {

enum ItemKind : int { ITEM_HIST = 0, ITEM_SORT3 = 1, ITEM_SORT5 = 2, ITEM_SORT3D = 3, ITEM_SORTW = 4 };

struct BatchItem {
    HistJob job;       // tile geometry, plan and rank (selection items use src/dst/pitches/W/H)
    int kind;
    int rows_per_warp; // selection-network tiles
    int tiles_x_s;     // selection-network tiles across
    int pad;
};

__device__ __forceinline__ void run_item(const BatchItem& it, int tile, unsigned char* sm) {
    const HistJob& j = it.job;
    if (it.kind == ITEM_SORT3D) {
        // warp tiles: 256 columns x one row x rows_per_warp slices
        const int wt = tile * BLOCK_WARPS + (int)(threadIdx.x >> 5);
        const int tx = wt % it.tiles_x_s, rest = wt / it.tiles_x_s;
        const int y = rest % j.H, tz = rest / j.H;
        if (j.elem == 1)
            sortnet3d_tile<uint8_t>(j.src, j.s_row, j.s_slice, j.dst, j.d_row, j.d_slice, j.W, j.H, j.D,
                                    it.rows_per_warp, tx, y, tz);
        else
            sortnet3d_tile<uint16_t>(j.src, j.s_row, j.s_slice, j.dst, j.d_row, j.d_slice, j.W, j.H, j.D,
                                     it.rows_per_warp, tx, y, tz);
        return;
    }
    if (it.kind != ITEM_HIST) {
        // a block item holds BLOCK_WARPS selection-network warp tiles
        const int wt = tile * BLOCK_WARPS + (int)(threadIdx.x >> 5);
        const int tx = wt % it.tiles_x_s, ty = wt / it.tiles_x_s;
        if (it.kind == ITEM_SORTW) {  // radius 3..5, pruned k x k networks (the radius is in job.r)
#define HRM_WIDE(RR)                                                                                            \
    if (j.r == RR) {                                                                                            \
        if (j.elem == 1) sortnet_wide_tile<uint8_t, RR>(j.src, j.s_row, j.dst, j.d_row, j.W, j.H, it.rows_per_warp, tx, ty); \
        else sortnet_wide_tile<uint16_t, RR>(j.src, j.s_row, j.dst, j.d_row, j.W, j.H, it.rows_per_warp, tx, ty);      \
    }
            HRM_WIDE(3) HRM_WIDE(4) HRM_WIDE(5)
#undef HRM_WIDE
        } else if (it.kind == ITEM_SORT3) {
            if (j.elem == 1) sortnet3x3_tile<uint8_t>(j.src, j.s_row, j.dst, j.d_row, j.W, j.H, it.rows_per_warp, tx, ty);
            else sortnet3x3_tile<uint16_t>(j.src, j.s_row, j.dst, j.d_row, j.W, j.H, it.rows_per_warp, tx, ty);
        } else {
            if (j.elem == 1) sortnet5x5_tile<uint8_t>(j.src, j.s_row, j.dst, j.d_row, j.W, j.H, it.rows_per_warp, tx, ty);
            else sortnet5x5_tile<uint16_t>(j.src, j.s_row, j.dst, j.d_row, j.W, j.H, it.rows_per_warp, tx, ty);
        }
        return;
    }
#define HRM_CASE(T, C)                                                          \
    if (j.ppl == 1 && j.cw == C) {                                              \
        if (j.dims == 3) hist_tile<T, 1, C, 3>(j, tile, sm);                    \
        else hist_tile<T, 1, C, 2>(j, tile, sm);                                \
        return;                                                                 \
    }
    if (j.elem == 1) {
        HRM_CASE(uint8_t, 1) HRM_CASE(uint8_t, 2)
    } else {
        HRM_CASE(uint16_t, 1) HRM_CASE(uint16_t, 2)
    }
#undef HRM_CASE
    if (threadIdx.x == 0) set_error(j.err, DEV_BAD_JOB);
}

// MINB: resident blocks per SM the register budget is sized for (3: up to
// 168 registers; 4: 128, for batches whose shared memory allows four tiles).
template <int MINB>
__global__ void __launch_bounds__(BLOCK_THREADS, MINB) batch_kernel(const BatchItem* __restrict__ items,
                                                              const unsigned* __restrict__ tile_off, int nitems,
                                                              unsigned* counter, unsigned total) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_next;
    // the current item's descriptor, staged once per tile in shared memory
    // (a per-thread copy would live in local memory)
    __shared__ __align__(16) BatchItem s_item;
    static_assert(sizeof(BatchItem) % 4 == 0, "BatchItem copied as words");
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(counter, 1u);
        __syncthreads();
        const unsigned t = s_next;
        if (t >= total) break;
        int lo = 0, hi = nitems - 1;  // last item whose first tile is <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile_off[mid] <= t) lo = mid; else hi = mid - 1;
        }
        for (int i = threadIdx.x; i < (int)(sizeof(BatchItem) / 4); i += blockDim.x)
            reinterpret_cast<uint32_t*>(&s_item)[i] = reinterpret_cast<const uint32_t*>(items + lo)[i];
        __syncthreads();  // the descriptor is staged; every thread has read s_next
        run_item(s_item, (int)(t - tile_off[lo]), smem);
        __syncthreads();  // the tile's shared memory and the descriptor are free again
    }
}


// Launch of the 4-blocks-per-SM instantiation (compiled in batch4.cu).
cudaError_t launch_batch_kernel4(unsigned grid, size_t smem, cudaStream_t st, const BatchItem* items,
                                 const unsigned* offs, int nitems, unsigned* counter, unsigned total);

}  // namespace hrm

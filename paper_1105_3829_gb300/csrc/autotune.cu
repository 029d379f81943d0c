// autotune.cu -- timed search over kernel plans for one problem class.
//
// Candidates: the tree's top level (uniform over the value range, or the
// adaptive power-of-16 split of Section III-C), the selection network vs the
// histogram kernel (2D radius <= 5), tile width (128/256 outputs per tile),
// shared memory per tile for the node cache (which trades cached nodes
// against resident tiles per SM), and strip length (the default one-wave
// length and half of it: longer strips amortise the per-strip start-up,
// shorter ones balance slow tiles).  The top level is chosen first, on the
// default geometry, and the geometry grid is then searched under it.  Each
// candidate is timed with CUDA events on the caller's stream; the fastest is
// cached for the class, the default plan unless another is at least 3 %
// faster.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "runtime.h"

namespace hrm {

// Deterministic synthetic input: 12-bit (uint16) or 8-bit noise plus a ramp.
__global__ void synth_fill(unsigned char* p, size_t pitch, size_t slice, int W, int H, int D, int elem) {
    const long n = (long)W * H * D;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % W), y = (int)((i / W) % H), z = (int)(i / ((long)W * H));
        uint32_t h = (uint32_t)i * 2654435761u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        const uint32_t top = elem == 2 ? 4095u : 255u;
        const uint32_t v = ((h & top) + (uint32_t)(x + y) * (top / 1024 + 1)) & top;
        unsigned char* row = p + (size_t)z * slice + (size_t)y * pitch;
        if (elem == 2) reinterpret_cast<uint16_t*>(row)[x] = (uint16_t)v;
        else row[x] = (unsigned char)v;
    }
}

}  // namespace hrm

using namespace hrm;

extern "C" int hrm_autotune(int dtype, int dims, int width, int height, int depth, int radius,
                            unsigned flags, const void* sample, size_t sample_pitch,
                            size_t sample_slice_pitch, void* stream, hrm_plan* best) {
    if (!best) return fail(HRM_EINVAL, "null plan");
    if (dims != 2 && dims != 3) return fail(HRM_EINVAL, "dims must be 2 or 3");
    const int D = dims == 3 ? depth : 1;
    const size_t es = dtype == HRM_U16 ? 2 : 1;
    cudaStream_t st = (cudaStream_t)stream;
    if (radius == 0 || width <= 0 || height <= 0 || D <= 0) {
        *best = hrm_plan{0, 0, 0, 0};
        return HRM_OK;
    }
    const size_t pitch = ((size_t)width * es + 255) & ~(size_t)255;
    const size_t slice = pitch * height;
    void* dst = nullptr;
    void* synth = nullptr;
    cudaError_t e = cudaMalloc(&dst, slice * D);
    if (e != cudaSuccess) return fail(HRM_ENOMEM, "autotune output buffer");
    const void* src = sample;
    size_t sp = sample_pitch, ss = sample_slice_pitch;
    if (!src) {
        e = cudaMalloc(&synth, slice * D);
        if (e != cudaSuccess) {
            cudaFree(dst);
            return fail(HRM_ENOMEM, "autotune input buffer");
        }
        synth_fill<<<1024, 256, 0, st>>>((unsigned char*)synth, pitch, slice, width, height, D, (int)es);
        src = synth;
        sp = pitch;
        ss = slice;
    }
    Image im{dtype, dims, src, dst, sp, ss, pitch, slice, width, height, D};
    int rc = validate(im, radius, HRM_BORDER_REPLICATE, flags);
    const DeviceInfo& di = device_info();
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!rc) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
    }
    // best of two timed runs after one warm-up (1e30 once rc is set)
    auto time_plan = [&](const hrm_plan& cand) {
        float ms = 1e30f;
        if (!rc) rc = filter_impl(im, radius, -1, flags, 0, &cand, st);  // warm-up
        for (int rep = 0; !rc && rep < 2; ++rep) {
            cudaEventRecord(e0, st);
            rc = filter_impl(im, radius, -1, flags, 0, &cand, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = cuda_fail(cudaGetLastError(), "autotune timing");
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        return rc ? 1e30f : ms;
    };
    // The default plan (all fields 0: the planner's choices, no feedback)
    // is timed first; another plan replaces it only if it is at least
    // KEEP_MARGIN faster, so timing noise between near-equal plans cannot
    // pick a slower one.
    constexpr float KEEP_MARGIN = 0.97f;
    const hrm_plan zero{0, 0, 0, 0, 0};
    const PlanH dp = rc ? PlanH{} : resolve_plan(dtype, dims, width, height, D, radius, flags, di, &zero, false);
    const int own_tree = (flags & HRM_ADAPTIVE) ? 2 : 1;
    hrm_plan bp = zero;
    float best_ms = time_plan(zero) * KEEP_MARGIN;
    int tree = own_tree;
    if (!rc && dp.path == 2) {  // the other top level on the default geometry
        const hrm_plan other{0, 0, 0, 0, 3 - own_tree};
        const float ms = time_plan(other);
        if (ms < best_ms) {
            best_ms = ms;
            bp = other;
            tree = 3 - own_tree;
        }
    }
    std::vector<hrm_plan> cands;
    const int cw = counter_width(dims, radius);
    if (!rc) {
        if (dims == 2 && radius <= SORTNET_MAX_R2D) cands.push_back(hrm_plan{0, 0, 0, 1, 0});
        const int lines = dims == 3 ? height : 1, walk = dims == 3 ? D : height;
        for (int tw : {BLOCK_THREADS, 2 * BLOCK_THREADS}) {
            if (tw > BLOCK_THREADS && width <= tw / 2) continue;
            for (int kb : {32, 48, 64, 76, 96, 128, 160, 200}) {
                PlanH p{};
                p.ppl = tw / BLOCK_THREADS;
                p.cw = cw;
                p.es = (int)es;
                const size_t budget = (size_t)kb * 1024;
                const size_t ring = hist_ring_bytes(tw, radius, (int)es);
                p.ring = (dims == 2 && cw == 1 && ring * 3 <= budget) ? 1 : 0;
                p.nslots = std::min(slots_for(tw, radius, cw, budget - (p.ring ? ring : 0)), MAX_SLOTS);
                if (p.nslots < 3) continue;
                const size_t smem = plan_smem(p, radius);
                if (smem > (size_t)di.smem_optin) continue;
                const int sh = strip_length(dims, width, lines, walk, radius, tw, smem, di);
                for (int f : {2, 1}) {  // the default strip length and half of it
                    const int shf = std::max(8, sh / f);
                    if (f == 2 && shf == sh) continue;
                    cands.push_back(hrm_plan{tw, shf, kb, 2, tree});
                }
            }
        }
    }
    for (size_t i = 0; !rc && i < cands.size(); ++i) {
        const float ms = time_plan(cands[i]);
        if (ms < best_ms) {
            best_ms = ms;
            bp = cands[i];
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(dst);
    if (synth) cudaFree(synth);
    if (rc) return rc;
    if (bp.tile_width == 0 && bp.path == 0) {  // a default-geometry plan won: report (and cache) what it resolves to
        const int t = bp.tree;
        const PlanH rp = resolve_plan(dtype, dims, width, height, D, radius, flags, di, &bp, false);
        bp = hrm_plan{BLOCK_THREADS * rp.ppl, rp.sh, (int)((plan_smem(rp, radius) + 1023) / 1024), rp.path,
                      rp.path == 2 ? (t ? t : own_tree) : 0};
    }
    plan_store(ProblemKey{dtype, dims, width, height, D, radius, flags}, bp);
    *best = bp;
    return HRM_OK;
}

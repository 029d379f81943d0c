// runtime.h -- host runtime shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/hrm.h"
#include "hist_tile.cuh"
#include "hist_common.cuh"

namespace hrm {

// Thread-local last-error message; returns `code` for convenient `return fail(...)`.
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
void clear_error();

struct DeviceInfo {
    int device = -1;
    int num_sms = 0;
    int smem_per_sm = 0;       // bytes
    int smem_optin = 0;        // max dynamic smem per block (bytes)
    int max_blocks_per_sm = 32;
};
const DeviceInfo& device_info();  // of the current device

// Per-(device, stream) workspace: level descriptors, pre-pass histograms,
// the device error word and the batch work counters.
constexpr int WS_MAX_DESC = 4096;
struct Workspace {
    LevelDesc* desc = nullptr;   // WS_MAX_DESC descriptors
    uint32_t* hist = nullptr;    // 2 * 4096 counters (reused by every pre-pass on this stream)
    unsigned* err = nullptr;     // device error word
    unsigned* counters = nullptr;  // 64 work counters for persistent kernels
};
int workspace_for(cudaStream_t st, Workspace** out);
// The stream's workspace if one exists (never allocates), else null.
Workspace* workspace_find(cudaStream_t st);
// hrm_filter_batch_noalloc's error word for the current device, read after
// `st` finishes and cleared (0 when no such call has run on the device).
int noalloc_error_take(cudaStream_t st, unsigned* code);

// Planning.
// Largest 2D radius served by a selection network (sortnet.cuh).
constexpr int SORTNET_MAX_R2D = 5;

struct PlanH {
    int ppl;      // outputs per thread (TW = BLOCK_THREADS * ppl)
    int sh;       // strip length along the walk axis
    int nslots;   // slots per warp incl. root
    int path;     // 1 = selection network, 2 = histogram
    int cw;       // counter width (bytes)
    int ring;     // stage the last n+1 input rows in shared memory (2D)
    int es;       // element size (bytes)
    int tree;     // top level: 0 = as the call's flags say, 1 = uniform, 2 = adaptive
};
// Whether a histogram call builds the adaptive top level: the plan's tree
// choice, else the call's HRM_ADAPTIVE flag.
inline bool plan_adaptive(const PlanH& p, unsigned flags) {
    return p.tree ? p.tree == 2 : (flags & HRM_ADAPTIVE) != 0;
}
struct ProblemKey {
    int dtype, dims, width, height, depth, radius;
    unsigned flags;
};
bool plan_lookup(const ProblemKey& k, hrm_plan* p);
void plan_store(const ProblemKey& k, const hrm_plan& p);
// dims 2: lines = 1, walk = H; dims 3: lines = H (one tile row per y), walk = D.
int strip_layout(int walk, int sh, int r, int* she, int* ne);
void size_slots(PlanH& p, int dims, int r, size_t budget);
int strip_length(int dims, int W, int lines, int walk, int r, int tw, size_t smem, const DeviceInfo& di);
PlanH default_plan(int dims, int es, int W, int lines, int walk, int r, const DeviceInfo& di);
// feedback: single-image 2D calls may switch an unplanned class to the
// large-node-cache plan after its first call measured many node installs.
PlanH resolve_plan(int dtype, int dims, int W, int H, int D, int r, unsigned flags, const DeviceInfo& di,
                   const hrm_plan* force, bool feedback = false);
int slots_for(int tw, int r, int cw, size_t budget);
size_t plan_smem(const PlanH& p, int r);
int counter_width(int dims, int r);

// Kernel launchers (defined in the .cu files).
cudaError_t launch_sortnet2d(int elem, int radius, const void* src, size_t sp, void* dst, size_t dp,
                             int W, int H, int rows_per_warp, cudaStream_t st);
cudaError_t launch_sortnet3d(int elem, const void* src, size_t sp, size_t ss, void* dst, size_t dp, size_t ds,
                             int W, int H, int D, int zn, cudaStream_t st);
cudaError_t launch_hist(const HistJob& job, cudaStream_t st);
// Video topology: histogram of a filtered frame (the median estimate for the
// next frame) and the top-level boundaries from it.
cudaError_t launch_topology_from_output(int elem, const void* dst, size_t dp, int W, int H, LevelDesc* desc,
                                        uint32_t* hist, int num_sms, cudaStream_t st);
cudaError_t launch_levels(int elem, bool adaptive, const void* src, size_t sp, size_t slice, int W,
                          int H, int D, LevelDesc* desc, uint32_t* hist, int num_sms,
                          cudaStream_t st);

// Shared entry (2D / 3D, median / rank / reduced precision).
struct Image {
    int dtype, dims;
    const void* src;
    void* dst;
    size_t sp, sslice, dp, dslice;
    int W, H, D;
};
int filter_impl(const Image& im, int r, long rank, unsigned flags, int drop_bits, const hrm_plan* force,
                cudaStream_t st, const LevelDesc* given = nullptr);
int validate(const Image& im, int r, int border, unsigned flags);
// Fill a HistJob (pre-pass descriptor supplied by the caller) for one image.
int make_hist_job(const Image& im, int r, uint32_t K, unsigned flags, int drop_bits, const PlanH& p,
                  const LevelDesc* desc, unsigned* err, HistJob* job);

// Frame streams: the checks a frame's topology must pass (HRM_OK or
// HRM_EINVAL with the message set), and the enqueue of its update from the
// frame's output (records `dtype` as the descriptor's dtype on success).
int topology_check(const hrm_topology* t);
int topology_device_of(const hrm_topology* t);
int topology_update(hrm_topology* t, int dtype, const void* dst, size_t dp, int W, int H, cudaStream_t st);

}  // namespace hrm

// Frame-stream state: the top level the next frame of the stream will use.
struct hrm_topology {
    int device = -1;
    int dtype = 0;      // dtype of the frame the descriptor was made from (0: none yet)
    hrm::LevelDesc* desc = nullptr;
    uint32_t* hist = nullptr;
};

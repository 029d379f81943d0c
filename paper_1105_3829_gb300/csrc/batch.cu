// batch.cu -- many images / volumes of uneven size, dtype and radius in ONE
// persistent kernel launch over a device tile work queue, plus its CUDA-graph
// capture.
//
// Every job is cut into the same warp tiles its single-image launch would use
// (hierarchical-histogram strips, or selection-network tiles for 2D radius <= 5 and 3D radius 1);
// the tiles of all jobs form one queue.  A grid of resident warps repeatedly
// takes the next tile with an atomic counter and runs the matching tile body,
// so small and large jobs share the GPU without per-job launches or tails.
// Outputs are bit-identical to the single-image calls: each tile computes
// exactly what it computes there.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <type_traits>
#include <vector>

#include "batch_kernel.cuh"
#include "runtime.h"

namespace hrm {



// Level pre-pass for many images at once (uniform trees need only the value range).
struct LevelItem {
    const unsigned char* src;
    size_t sp, slice;
    int W, H, D, elem;
    LevelDesc* desc;
    int mode;
    int pad;
};

__global__ void batch_levels_init(const LevelItem* it, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    LevelDesc* d = it[j].desc;
    d->mode = (uint32_t)it[j].mode;
    d->vmin = 0xFFFFFFFFu;
    d->vmax = 0;
    d->count = 0;
}

__global__ void batch_minmax(const LevelItem* items, int n) {
    const int j = blockIdx.y;
    if (j >= n) return;
    const LevelItem it = items[j];
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    const long rows = (long)it.H * it.D;
    const int lane = threadIdx.x & 31;
    const long warp = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long nw = ((long)gridDim.x * blockDim.x) >> 5;
    for (long row = warp; row < rows; row += nw) {
        const int z = (int)(row / it.H), y = (int)(row % it.H);
        const unsigned char* p = it.src + (size_t)z * it.slice + (size_t)y * it.sp;
        for (int x = lane; x < it.W; x += 32) {
            const uint32_t v = it.elem == 1 ? (uint32_t)__ldg(p + x)
                                            : (uint32_t)__ldg(reinterpret_cast<const uint16_t*>(p) + x);
            lo = min(lo, v);
            hi = max(hi, v);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
        atomicMin(&it.desc->vmin, lo);
        atomicMax(&it.desc->vmax, hi);
    }
}

// ---------------------------------------------------------------------------
// Host side.

struct BatchDev {
    BatchItem* items = nullptr;
    unsigned* offs = nullptr;
    LevelItem* litems = nullptr;
    LevelDesc* descs = nullptr;
    unsigned* counter = nullptr;
    uint32_t* hist = nullptr;
    unsigned* err = nullptr;
    int cap = 0;
    void* base = nullptr;
    // pinned staging ring for asynchronous table uploads (a pageable source
    // could make cudaMemcpyAsync wait for the stream)
    static constexpr int NSTAGE = 4;
    unsigned char* stage[NSTAGE] = {};
    cudaEvent_t stage_ev[NSTAGE] = {};
    size_t stage_cap = 0;
    int stage_next = 0;
};

// The buffer is cleared on `st`, the stream its tables are uploaded and used
// on (a plain cudaMemset would run on the legacy default stream, which does
// not order against non-blocking streams).
static int batchdev_alloc(BatchDev& b, int cap, cudaStream_t st) {
    const size_t bytes = sizeof(BatchItem) * cap + sizeof(unsigned) * (cap + 1) + sizeof(LevelItem) * cap +
                         sizeof(LevelDesc) * cap + 256 + sizeof(uint32_t) * 2 * 4096 + 256;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes + 64 * 6);
    if (e != cudaSuccess) return fail(HRM_ENOMEM, std::string("batch buffer cudaMalloc: ") + cudaGetErrorString(e));
    auto align = [](unsigned char*& q) { q = (unsigned char*)(((uintptr_t)q + 63) & ~(uintptr_t)63); };
    unsigned char* q = (unsigned char*)p;
    b.base = p;
    b.cap = cap;
    align(q); b.items = (BatchItem*)q; q += sizeof(BatchItem) * cap;
    align(q); b.offs = (unsigned*)q; q += sizeof(unsigned) * (cap + 1);
    align(q); b.litems = (LevelItem*)q; q += sizeof(LevelItem) * cap;
    align(q); b.descs = (LevelDesc*)q; q += sizeof(LevelDesc) * cap;
    align(q); b.counter = (unsigned*)q; q += 128;
    b.err = (unsigned*)q; q += 128;
    align(q); b.hist = (uint32_t*)q;
    e = cudaMemsetAsync(p, 0, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch buffer memset");
    return HRM_OK;
}

static void batchdev_free(BatchDev& b) {
    if (b.base) cudaFree(b.base);
    for (int i = 0; i < BatchDev::NSTAGE; ++i) {
        if (b.stage_ev[i]) cudaEventSynchronize(b.stage_ev[i]), cudaEventDestroy(b.stage_ev[i]);
        if (b.stage[i]) cudaFreeHost(b.stage[i]);
    }
    b = BatchDev{};
}

// A vector that never allocates: fixed capacity, for the no-allocation path.
template <class T, int N>
struct FixedVec {
    T v[N];
    int n = 0;
    bool push_back(const T& x) {
        if (n >= N) return false;
        v[n++] = x;
        return true;
    }
    size_t size() const { return (size_t)n; }
    const T* data() const { return v; }
    T* begin() { return v; }
    T* end() { return v + n; }
    const T* begin() const { return v; }
    const T* end() const { return v + n; }
    const T& operator[](size_t i) const { return v[i]; }
    T& back() { return v[n - 1]; }
};

template <class T>
struct HeapVec : std::vector<T> {
    bool push_back(const T& x) {
        std::vector<T>::push_back(x);
        return true;
    }
};

struct BatchTmp {
    BatchItem it;
    double cost;
};

// A frame-stream job: its output becomes the topology's next top level.
struct TopoUpdate {
    hrm_topology* topo;
    int dtype;
    const void* dst;
    size_t dp;
    int W, H;
};

// Host-side plan of a batch: items in queue order plus the pre-pass list.
template <template <class> class V>
struct BatchPlanT {
    V<BatchItem> items;
    V<unsigned> offs;
    V<LevelItem> levels;      // uniform pre-pass items
    V<int> adaptive;          // indices into levels that need the adaptive pre-pass
    V<Image> copies;          // radius-0 jobs
    V<TopoUpdate> topos;      // frame-stream jobs, updated after the launch
    V<BatchTmp> tmp;          // planning scratch
    size_t smem = 0;
    unsigned total = 0;
};
using BatchPlan = BatchPlanT<HeapVec>;

template <template <class> class V>
static int plan_batch(const hrm_job* jobs, int njobs, const BatchDev& dev, BatchPlanT<V>& bp) {
    const DeviceInfo& di = device_info();
    using Tmp = BatchTmp;
    auto& tmp = bp.tmp;
    for (int i = 0; i < njobs; ++i) {
        const hrm_job& jb = jobs[i];
        if (jb.dims != 2 && jb.dims != 3) return fail(HRM_EINVAL, "job dims must be 2 or 3");
        Image im{jb.dtype, jb.dims, jb.src, jb.dst, jb.src_pitch, jb.src_slice_pitch, jb.dst_pitch,
                 jb.dst_slice_pitch, jb.width, jb.height, jb.dims == 3 ? jb.depth : 1};
        int rc = validate(im, jb.radius, HRM_BORDER_REPLICATE, jb.flags);
        if (rc) return fail(rc, "job " + std::to_string(i) + ": " + hrm_last_error());
        const long n = 2L * jb.radius + 1, N = jb.dims == 3 ? n * n * n : n * n;
        if (jb.rank < -1 || jb.rank >= N) return fail(HRM_EINVAL, "job " + std::to_string(i) + ": rank out of range");
        const bool median = jb.rank < 0 || jb.rank == (N - 1) / 2;
        // A frame of a stream runs as hrm_filter2d_video: the topology's top
        // level when it holds one of this dtype, else the adaptive pre-pass.
        unsigned flags = jb.flags;
        const LevelDesc* given = nullptr;
        if (jb.topo) {
            rc = topology_check(jb.topo);
            if (rc) return fail(rc, "job " + std::to_string(i) + ": " + hrm_last_error());
            if (jb.dims != 2 || !median || jb.flags)
                return fail(HRM_EINVAL, "job " + std::to_string(i) + ": a frame-stream job is a 2D median with flags 0");
            for (const TopoUpdate& u : bp.topos)
                if (u.topo == jb.topo)
                    return fail(HRM_EINVAL, "job " + std::to_string(i) + ": topology already used in this batch");
            if (im.W == 0 || im.H == 0) continue;
            if (!bp.topos.push_back(TopoUpdate{jb.topo, jb.dtype, im.dst, im.dp, im.W, im.H}))
                return fail(HRM_ENOTSUP, "too many jobs");
            if (jb.topo->dtype == jb.dtype) given = jb.topo->desc;
            else flags = HRM_ADAPTIVE;
        }
        if (im.W == 0 || im.H == 0 || im.D == 0) continue;
        if (jb.radius == 0) {
            if (!bp.copies.push_back(im)) return fail(HRM_ENOTSUP, "too many jobs");
            continue;
        }
        const uint32_t K = (uint32_t)(jb.rank < 0 ? (N + 1) / 2 : jb.rank + 1);
        PlanH p = resolve_plan(jb.dtype, jb.dims, im.W, im.H, im.D, jb.radius, flags, di, nullptr);
        if (p.ppl != 1) {  // the persistent kernel carries only 128-output tiles (register budget)
            const size_t budget = plan_smem(p, jb.radius);
            p.ppl = 1;
            size_slots(p, jb.dims, jb.radius, budget);
        }
        Tmp t{};
        const int es = jb.dtype == HRM_U16 ? 2 : 1;
        if (jb.dims == 2 && p.path == 1 && jb.radius <= SORTNET_MAX_R2D && median) {
            t.it.kind = jb.radius == 1 ? ITEM_SORT3 : (jb.radius == 2 ? ITEM_SORT5 : ITEM_SORTW);
            t.it.rows_per_warp = 32;
            // columns per warp tile: 256 (r <= 2), else two per output lane
            const int tw = jb.radius <= 2 ? 256 : 2 * (32 - 2 * ((jb.radius + 1) / 2));
            t.it.tiles_x_s = (im.W + tw - 1) / tw;
            HistJob& h = t.it.job;
            h.r = jb.radius;
            h.src = (const unsigned char*)im.src;
            h.dst = (unsigned char*)im.dst;
            h.s_row = im.sp;
            h.d_row = im.dp;
            h.W = im.W;
            h.H = im.H;
            h.elem = es;
            const int wtiles = t.it.tiles_x_s * ((im.H + 31) / 32);
            h.ntiles = (wtiles + BLOCK_WARPS - 1) / BLOCK_WARPS;
            t.cost = jb.radius <= 2 ? 1.0 : (double)jb.radius;
        } else if (jb.dims == 3 && p.path == 1 && jb.radius == 1 && median) {
            t.it.kind = ITEM_SORT3D;
            t.it.rows_per_warp = 32;  // slices per warp tile
            t.it.tiles_x_s = (im.W + 255) / 256;
            HistJob& h = t.it.job;
            h.src = (const unsigned char*)im.src;
            h.dst = (unsigned char*)im.dst;
            h.s_row = im.sp;
            h.s_slice = im.sslice;
            h.d_row = im.dp;
            h.d_slice = im.dslice;
            h.W = im.W;
            h.H = im.H;
            h.D = im.D;
            h.elem = es;
            const long wtiles = (long)t.it.tiles_x_s * im.H * ((im.D + 31) / 32);
            h.ntiles = (int)((wtiles + BLOCK_WARPS - 1) / BLOCK_WARPS);
            t.cost = 2.0;
        } else {
            const LevelDesc* desc = given;
            const bool adaptive = plan_adaptive(p, flags);
            if (!desc && (es == 2 || adaptive)) {
                const int li = (int)bp.levels.size();
                if (li >= dev.cap) return fail(HRM_ENOTSUP, "too many jobs for the batch buffer");
                LevelItem L{(const unsigned char*)im.src, im.sp, im.dims == 3 ? im.sslice : 0, im.W, im.H,
                            im.D, es, dev.descs + li, adaptive ? 1 : 0, 0};
                if (!bp.levels.push_back(L)) return fail(HRM_ENOTSUP, "too many jobs");
                if (adaptive && !bp.adaptive.push_back(li)) return fail(HRM_ENOTSUP, "too many jobs");
                desc = dev.descs + li;
            }
            t.it.kind = ITEM_HIST;
            rc = make_hist_job(im, jb.radius, K, flags, 0, p, desc, dev.err, &t.it.job);
            if (rc) return rc;
            bp.smem = std::max(bp.smem, plan_smem(p, jb.radius));
            // expensive tiles first: work per tile grows with the strip and the window
            t.cost = (double)p.sh * ((double)BLOCK_THREADS * p.ppl + 2.0 * jb.radius) * (jb.dims == 3 ? n : 1);
        }
        if (!tmp.push_back(t)) return fail(HRM_ENOTSUP, "too many jobs");
    }
    // expensive tiles first (stable; the fixed-capacity path sorts in place)
    if constexpr (std::is_same<V<int>, HeapVec<int>>::value) {
        std::stable_sort(tmp.begin(), tmp.end(), [](const Tmp& a, const Tmp& b) { return a.cost > b.cost; });
    } else {
        for (int i = 1; i < (int)tmp.size(); ++i)
            for (int j = i; j > 0 && tmp.begin()[j - 1].cost < tmp.begin()[j].cost; --j)
                std::swap(tmp.begin()[j - 1], tmp.begin()[j]);
    }
    if ((int)tmp.size() > dev.cap) return fail(HRM_ENOTSUP, "too many jobs for the batch buffer");
    unsigned off = 0;
    for (const Tmp& t : tmp) {
        bp.items.push_back(t.it);
        bp.offs.push_back(off);
        off += (unsigned)t.it.job.ntiles;
    }
    bp.offs.push_back(off);
    bp.total = off;
    return HRM_OK;
}

cudaError_t launch_levels_adaptive_only(int elem, const void* src, size_t sp, size_t slice, int W, int H,
                                        int D, LevelDesc* desc, uint32_t* hist, int num_sms, cudaStream_t st);

template <class Plan>
static int enqueue_filters(const Plan& bp, const BatchDev& dev, cudaStream_t st);

// Enqueue a planned batch whose tables are already on the device, then the
// frame streams' topology updates from their outputs.
template <class Plan>
static int enqueue_batch(const Plan& bp, const BatchDev& dev, cudaStream_t st) {
    int rc = enqueue_filters(bp, dev, st);
    for (const TopoUpdate& u : bp.topos) {
        if (rc) break;
        rc = topology_update(u.topo, u.dtype, u.dst, u.dp, u.W, u.H, st);
    }
    return rc;
}

template <class Plan>
static int enqueue_filters(const Plan& bp, const BatchDev& dev, cudaStream_t st) {
    const DeviceInfo& di = device_info();
    cudaError_t e;
    for (const Image& im : bp.copies) {
        const size_t es = im.dtype == HRM_U16 ? 2 : 1;
        for (int z = 0; z < im.D; ++z) {
            e = cudaMemcpy2DAsync((unsigned char*)im.dst + z * im.dslice, im.dp,
                                  (const unsigned char*)im.src + z * im.sslice, im.sp, im.W * es, im.H,
                                  cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "batch copy");
        }
    }
    if (bp.total == 0) return HRM_OK;
    const int nl = (int)bp.levels.size();
    if (nl > 0) {
        batch_levels_init<<<(nl + 127) / 128, 128, 0, st>>>(dev.litems, nl);
        dim3 g(std::max(1, std::min(64, di.num_sms * 8 / std::max(1, nl))), nl);
        batch_minmax<<<g, 256, 0, st>>>(dev.litems, nl);
        for (int li : bp.adaptive) {
            const LevelItem& L = bp.levels[li];
            e = launch_levels_adaptive_only(L.elem, L.src, L.sp, L.slice, L.W, L.H, L.D, L.desc, dev.hist,
                                            di.num_sms, st);
            if (e != cudaSuccess) return cuda_fail(e, "adaptive pre-pass");
        }
    }
    e = cudaMemsetAsync(dev.counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e, "batch counter reset");
    const size_t smem = bp.smem;
    if (smem > (size_t)di.smem_optin) return fail(HRM_ENOTSUP, "batch plan exceeds shared memory");
    int per_sm = std::max(1, std::min(di.max_blocks_per_sm, (int)(di.smem_per_sm / (smem + 1024))));
    if (per_sm >= 4) {  // four tiles fit: the 128-register instantiation
        per_sm = 4;
        const unsigned grid = (unsigned)std::min<long>((long)di.num_sms * per_sm, (long)bp.total);
        e = launch_batch_kernel4(grid, smem, st, dev.items, dev.offs, (int)bp.items.size(), dev.counter, bp.total);
    } else {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(batch_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_fail(e, "batch smem attribute");
        }
        per_sm = std::min(per_sm, 3);
        const unsigned grid = (unsigned)std::min<long>((long)di.num_sms * per_sm, (long)bp.total);
        batch_kernel<3><<<grid, BLOCK_THREADS, smem, st>>>(dev.items, dev.offs, (int)bp.items.size(), dev.counter,
                                                           bp.total);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HRM_OK : cuda_fail(e, "batch kernel launch");
}

static int upload_plan(const BatchPlan& bp, BatchDev& dev, cudaStream_t st, bool sync) {
    cudaError_t e = cudaSuccess;
    const size_t n_items = sizeof(BatchItem) * bp.items.size(), n_offs = sizeof(unsigned) * bp.offs.size(),
                 n_lev = sizeof(LevelItem) * bp.levels.size();
    if (sync) {
        auto cp = [&](void* d, const void* h, size_t n) {
            if (n && e == cudaSuccess) e = cudaMemcpy(d, h, n, cudaMemcpyHostToDevice);
        };
        cp(dev.items, bp.items.data(), n_items);
        cp(dev.offs, bp.offs.data(), n_offs);
        cp(dev.litems, bp.levels.data(), n_lev);
        return e == cudaSuccess ? HRM_OK : cuda_fail(e, "batch table upload");
    }
    const size_t need = n_items + n_offs + n_lev;
    if (dev.stage_cap < need) {
        for (int i = 0; i < BatchDev::NSTAGE; ++i) {
            if (dev.stage_ev[i]) cudaEventSynchronize(dev.stage_ev[i]);
            if (dev.stage[i]) cudaFreeHost(dev.stage[i]);
            dev.stage[i] = nullptr;
            e = cudaMallocHost((void**)&dev.stage[i], need);
            if (e != cudaSuccess) return fail(HRM_ENOMEM, "pinned staging buffer");
            if (!dev.stage_ev[i]) {
                e = cudaEventCreateWithFlags(&dev.stage_ev[i], cudaEventDisableTiming);
                if (e != cudaSuccess) return cuda_fail(e, "staging event");
            }
        }
        dev.stage_cap = need;
    }
    const int k = dev.stage_next;
    dev.stage_next = (k + 1) % BatchDev::NSTAGE;
    e = cudaEventSynchronize(dev.stage_ev[k]);  // that slot's previous upload has been consumed
    if (e != cudaSuccess) return cuda_fail(e, "staging event wait");
    unsigned char* h = dev.stage[k];
    memcpy(h, bp.items.data(), n_items);
    memcpy(h + n_items, bp.offs.data(), n_offs);
    if (n_lev) memcpy(h + n_items + n_offs, bp.levels.data(), n_lev);
    if (n_items) e = cudaMemcpyAsync(dev.items, h, n_items, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_offs) e = cudaMemcpyAsync(dev.offs, h + n_items, n_offs, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_lev) e = cudaMemcpyAsync(dev.litems, h + n_items + n_offs, n_lev, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(dev.stage_ev[k], st);
    return e == cudaSuccess ? HRM_OK : cuda_fail(e, "batch table upload");
}

// Per-(device, stream) batch buffers for hrm_filter_batch (a map: the
// returned reference stays valid while other streams add entries).
static std::mutex g_bmu;
static std::map<std::pair<int, cudaStream_t>, BatchDev> g_bufs;

static int batch_buffers(cudaStream_t st, int need, BatchDev** out) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_bufs.find({dev, st});
    if (it != g_bufs.end()) {
        if (it->second.cap < need) {
            cudaStreamSynchronize(st);  // the old tables may still be in use
            batchdev_free(it->second);
            int rc = batchdev_alloc(it->second, std::max(need, 256), st);
            if (rc) return rc;
        }
        *out = &it->second;
        return HRM_OK;
    }
    BatchDev& b = g_bufs[{dev, st}];
    int rc = batchdev_alloc(b, std::max(need, 256), st);
    if (rc) {
        g_bufs.erase({dev, st});
        return rc;
    }
    *out = &b;
    return HRM_OK;
}

// ---------------------------------------------------------------------------
// Batch without allocation (hrm_filter_batch_noalloc): the job table, tile
// offsets, level descriptors, queue counter, error word and pre-pass
// histograms live in one file-scope device array instead of cudaMalloc'ed
// buffers.  In host code `g_noalloc_scratch` names a host-side stand-in, so its
// device address is fetched with cudaGetSymbolAddress once per device (with
// that device current) and passed to the kernels.

constexpr int NOALLOC_MAX_JOBS = 64;
constexpr size_t NOALLOC_SCRATCH_BYTES = 64 * 1024;

constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t NA_ITEMS = 0;
constexpr size_t NA_OFFS = na_align(NA_ITEMS + sizeof(BatchItem) * NOALLOC_MAX_JOBS);
constexpr size_t NA_LEVELS = na_align(NA_OFFS + sizeof(unsigned) * (NOALLOC_MAX_JOBS + 1));
constexpr size_t NA_DESCS = na_align(NA_LEVELS + sizeof(LevelItem) * NOALLOC_MAX_JOBS);
constexpr size_t NA_COUNTER = na_align(NA_DESCS + sizeof(LevelDesc) * NOALLOC_MAX_JOBS);
constexpr size_t NA_ERR = NA_COUNTER + 128;
constexpr size_t NA_HIST = na_align(NA_ERR + 128);
constexpr size_t NA_END = NA_HIST + sizeof(uint32_t) * 2 * 4096;
static_assert(NA_END <= NOALLOC_SCRATCH_BYTES, "no-allocation scratch layout exceeds its array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static std::mutex g_na_mu;
static unsigned char* g_na_addr[64];  // device address of the array, per device ordinal

static int noalloc_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(HRM_ENOTSUP, "device ordinal >= 64");
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_na_addr[dev] = (unsigned char*)p;
    }
    *out = g_na_addr[dev];
    return HRM_OK;
}

template <class T>
using NAVec = FixedVec<T, NOALLOC_MAX_JOBS + 1>;

// Read and clear the no-allocation path's error word for the current device
// after `st` has finished (hrm_device_status).  A device on which no
// no-allocation call has run reports 0 without touching the GPU.
int noalloc_error_take(cudaStream_t st, unsigned* code) {
    *code = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (dev >= 0 && dev < 64) base = g_na_addr[dev];
    }
    if (!base) return HRM_OK;
    unsigned* err = (unsigned*)(base + NA_ERR);
    e = cudaMemcpyAsync(code, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && *code) {
        e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e == cudaSuccess ? HRM_OK : cuda_fail(e, "no-allocation error word");
}

}  // namespace hrm

using namespace hrm;

extern "C" int hrm_filter_batch_noalloc(const hrm_job* jobs, int njobs, void* stream) {
    if (njobs < 0 || (njobs > 0 && !jobs)) return fail(HRM_EINVAL, "bad job list");
    if (njobs > NOALLOC_MAX_JOBS)
        return fail(HRM_EINVAL, "hrm_filter_batch_noalloc takes at most 64 jobs per call (got " +
                                    std::to_string(njobs) + "); split the batch or use hrm_filter_batch");
    if (njobs == 0) return HRM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = nullptr;
    int rc = noalloc_scratch(&base);
    if (rc) return rc;
    BatchDev dev;
    dev.items = (BatchItem*)(base + NA_ITEMS);
    dev.offs = (unsigned*)(base + NA_OFFS);
    dev.litems = (LevelItem*)(base + NA_LEVELS);
    dev.descs = (LevelDesc*)(base + NA_DESCS);
    dev.counter = (unsigned*)(base + NA_COUNTER);
    dev.err = (unsigned*)(base + NA_ERR);
    dev.hist = (uint32_t*)(base + NA_HIST);
    dev.cap = NOALLOC_MAX_JOBS;
    BatchPlanT<NAVec> plan;  // fixed capacity on the stack: no heap or device allocation
    rc = plan_batch(jobs, njobs, dev, plan);
    if (rc) return rc;
    // The array keeps the previous call's contents: enqueue_batch clears the
    // queue counter and the level descriptors.  The error word starts at zero
    // (the array is zero-initialised when the library loads) and is left set
    // by any kernel that raises it until hrm_device_status reads and clears it.
    cudaError_t e = cudaSuccess;
    auto up = [&](void* d, const void* h, size_t n) {
        if (n && e == cudaSuccess) e = cudaMemcpyAsync(d, h, n, cudaMemcpyHostToDevice, st);
    };
    up(dev.items, plan.items.data(), sizeof(BatchItem) * plan.items.size());
    up(dev.offs, plan.offs.data(), sizeof(unsigned) * plan.offs.size());
    up(dev.litems, plan.levels.data(), sizeof(LevelItem) * plan.levels.size());
    if (e != cudaSuccess) return cuda_fail(e, "no-allocation batch upload");
    return enqueue_batch(plan, dev, st);
}

// Test hook, deliberately not declared in include/hrm.h: plant an error code
// from the host in the error word of the no-allocation array of the current
// device (which = 0) or of a graph (which = 1), so that tests can check that
// hrm_device_status / hrm_batch_graph_status report and clear it without
// making any kernel fail.
extern "C" int hrm_debug_set_error_word(int which, void* graph, unsigned code);

struct hrm_batch_graph {
    BatchDev dev;
    BatchPlan plan;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

int hrm_filter_batch(const hrm_job* jobs, int njobs, void* stream) {
    if (njobs < 0 || (njobs > 0 && !jobs)) return fail(HRM_EINVAL, "bad job list");
    if (njobs == 0) return HRM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    BatchDev* dev = nullptr;
    int rc = batch_buffers(st, njobs, &dev);
    if (rc) return rc;
    Workspace* ws = nullptr;
    rc = workspace_for(st, &ws);
    if (rc) return rc;
    dev->err = ws->err;  // kernel error flags surface through hrm_device_status(stream)
    BatchPlan bp;
    rc = plan_batch(jobs, njobs, *dev, bp);
    if (rc) return rc;
    rc = upload_plan(bp, *dev, st, false);
    if (rc) return rc;
    return enqueue_batch(bp, *dev, st);
}

int hrm_batch_graph_create(const hrm_job* jobs, int njobs, void* stream, hrm_batch_graph** out) {
    if (!out || njobs <= 0 || !jobs) return fail(HRM_EINVAL, "bad job list");
    (void)stream;
    // the graph freezes whether a frame reads its topology or runs its own
    // pre-pass: only the former is a frame stream on every replay
    for (int i = 0; i < njobs; ++i)
        if (jobs[i].topo && jobs[i].topo->dtype != jobs[i].dtype)
            return fail(HRM_EINVAL, "job " + std::to_string(i) +
                                        ": a graph takes a topology only once it holds a top level of the job's dtype");
    auto* g = new hrm_batch_graph();
    int rc = batchdev_alloc(g->dev, std::max(njobs, 1), nullptr);  // the table upload below is synchronous
    if (rc) { delete g; return rc; }
    rc = plan_batch(jobs, njobs, g->dev, g->plan);
    if (!rc) rc = upload_plan(g->plan, g->dev, nullptr, true);
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaSuccess;
    if (!rc) {
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) rc = cuda_fail(e, "capture stream");
    }
    if (!rc) {
        // configure kernel attributes before capture (not stream operations)
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamBeginCapture");
        else {
            rc = enqueue_batch(g->plan, g->dev, cs);
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(cs, &graph);
            if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture");
            g->graph = graph;
            if (!rc) {
                e = cudaGraphInstantiate(&g->exec, g->graph, 0);
                if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
            }
        }
    }
    if (cs) cudaStreamDestroy(cs);
    if (rc) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        batchdev_free(g->dev);
        delete g;
        return rc;
    }
    *out = g;
    return HRM_OK;
}

int hrm_batch_graph_launch(hrm_batch_graph* g, void* stream) {
    if (!g || !g->exec) return fail(HRM_EINVAL, "null graph");
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? HRM_OK : cuda_fail(e, "cudaGraphLaunch");
}

int hrm_batch_graph_status(hrm_batch_graph* g, void* stream) {
    if (!g || !g->dev.err) return fail(HRM_EINVAL, "null graph");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned code = 0;
    cudaError_t e = cudaMemcpyAsync(&code, g->dev.err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && code) {
        e = cudaMemsetAsync(g->dev.err, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "graph status");
    if (code) return fail(HRM_EDEVICE, "a replay of this graph reported device error code " + std::to_string(code));
    return HRM_OK;
}

int hrm_debug_set_error_word(int which, void* graph, unsigned code) {
    unsigned* word = nullptr;
    if (which == 0) {
        unsigned char* base = nullptr;
        const int rc = noalloc_scratch(&base);
        if (rc) return rc;
        word = (unsigned*)(base + NA_ERR);
    } else if (which == 1 && graph) {
        word = ((hrm_batch_graph*)graph)->dev.err;
    }
    if (!word) return fail(HRM_EINVAL, "hrm_debug_set_error_word: unknown target");
    const cudaError_t e = cudaMemcpy(word, &code, sizeof(unsigned), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? HRM_OK : cuda_fail(e, "hrm_debug_set_error_word");
}

int hrm_batch_graph_destroy(hrm_batch_graph* g) {
    if (!g) return HRM_OK;
    cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    batchdev_free(g->dev);
    delete g;
    return HRM_OK;
}

}  // extern "C"

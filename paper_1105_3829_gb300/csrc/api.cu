// api.cu -- C-ABI entry points for the single-image filters, the workspace,
// device info, error reporting and planning.
#include <cuda_runtime.h>

#include <new>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>

#include "runtime.h"

namespace hrm {

// ---- errors -----------------------------------------------------------------
static thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}
int cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return HRM_ECUDA;
}
void clear_error() { g_err.clear(); }

// ---- device info ----------------------------------------------------------------
static std::mutex g_mu;
static std::map<int, DeviceInfo> g_devs;

const DeviceInfo& device_info() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_devs.find(dev);
    if (it != g_devs.end()) return it->second;
    DeviceInfo di;
    di.device = dev;
    cudaDeviceGetAttribute(&di.num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&di.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&di.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&di.max_blocks_per_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    if (di.num_sms <= 0) di.num_sms = 1;
    if (di.smem_per_sm <= 0) di.smem_per_sm = 100 * 1024;
    if (di.smem_optin <= 0) di.smem_optin = 48 * 1024;
    if (di.max_blocks_per_sm <= 0) di.max_blocks_per_sm = 16;
    return g_devs[dev] = di;
}

// ---- workspace -----------------------------------------------------------------
static std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

int workspace_for(cudaStream_t st, Workspace** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(dev, st);
    auto it = g_ws.find(key);
    if (it != g_ws.end()) {
        *out = &it->second;
        return HRM_OK;
    }
    Workspace w;
    const size_t bytes = sizeof(LevelDesc) * WS_MAX_DESC + sizeof(uint32_t) * 2 * 4096 + 256 + 64 * 4;
    void* base = nullptr;
    e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) return fail(HRM_ENOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
    unsigned char* p = (unsigned char*)base;
    w.desc = (LevelDesc*)p;
    p += sizeof(LevelDesc) * WS_MAX_DESC;
    w.hist = (uint32_t*)p;
    p += sizeof(uint32_t) * 2 * 4096;
    w.err = (unsigned*)p;
    p += 256;
    w.counters = (unsigned*)p;
    e = cudaMemsetAsync(base, 0, bytes, st);  // ordered with the stream's own work
    if (e != cudaSuccess) return cuda_fail(e, "workspace memset");
    *out = &(g_ws[key] = w);
    return HRM_OK;
}

Workspace* workspace_find(cudaStream_t st) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ws.find(std::make_pair(dev, st));
    return it == g_ws.end() ? nullptr : &it->second;
}

// ---- planning ----------------------------------------------------------------------
static std::map<std::tuple<int, int, int, int, int, int, unsigned>, hrm_plan> g_plans;

static std::tuple<int, int, int, int, int, int, unsigned> tkey(const ProblemKey& k) {
    return std::make_tuple(k.dtype, k.dims, k.width, k.height, k.depth, k.radius, k.flags);
}
// Environment (read once per process): HRM_PLAN_CACHE=<file> loads saved
// plans (hrm_plan_save format) before the first lookup; HRM_FORCE_PATH=hist
// or =sortnet forces the histogram kernel or the selection networks (where a
// network exists for the problem) for every call.
static void env_plans_once() {
    static std::once_flag once;
    std::call_once(once, [] {
        const char* f = std::getenv("HRM_PLAN_CACHE");
        if (f && *f) {
            if (hrm_plan_load(f) != HRM_OK) clear_error();  // a missing or bad file leaves the defaults
        }
    });
}

static int env_forced_path() {
    static const int v = [] {
        const char* s = std::getenv("HRM_FORCE_PATH");
        if (!s) return 0;
        if (!std::strcmp(s, "sortnet")) return 1;
        if (!std::strcmp(s, "hist")) return 2;
        return 0;
    }();
    return v;
}

bool plan_lookup(const ProblemKey& k, hrm_plan* p) {
    env_plans_once();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_plans.find(tkey(k));
    if (it == g_plans.end()) return false;
    *p = it->second;
    return true;
}
void plan_store(const ProblemKey& k, const hrm_plan& p) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_plans[tkey(k)] = p;
}

int counter_width(int dims, int r) {
    const long n = 2L * r + 1;
    return (dims == 3 && n * n > 255) ? 2 : 1;
}

int slots_for(int tw, int r, int cw, size_t budget) {
    const long nc = tw + 2L * r;
    long avail = (long)budget - META_BYTES - (nc + 1) * 32;
    long s = avail / (nc * 16 * cw);
    if (s > MAX_SLOTS) s = MAX_SLOTS;
    return (int)s;
}

size_t plan_smem(const PlanH& p, int r) {
    return hist_smem_bytes(BLOCK_THREADS * p.ppl, r, p.nslots, p.cw, p.ring, p.es);
}

// Fill slots (and the ring decision) for a given per-tile shared-memory budget.
void size_slots(PlanH& p, int dims, int r, size_t budget) {
    const int tw = BLOCK_THREADS * p.ppl;
    const size_t ring = hist_ring_bytes(tw, r, p.es);
#ifdef HRM_NO_RING
    p.ring = 0;
#else
    p.ring = (dims == 2 && p.cw == 1 && ring * 3 <= budget) ? 1 : 0;
#endif
    const size_t rest = budget > (p.ring ? ring : 0) ? budget - (p.ring ? ring : 0) : 0;
    p.nslots = std::max(2, std::min(slots_for(tw, r, p.cw, rest), MAX_SLOTS));
}

// Strip length: in 2D about two waves of interior tiles over the resident
// tile slots for 12 <= r < 32 and one wave otherwise (measured on the x-ray
// workload; larger windows pay more per strip start-up) (the slow rows near the image edges are in short edge
// strips that start first, see strip_layout); in 3D about two waves for
// 5 <= r < 8 and four otherwise (measured on the 256^3 volume).  At least n rows (min 96) so the
// per-strip start-up -- building the root from n rows and the first cached
// nodes -- stays a small share of a strip.
int strip_length(int dims, int W, int lines, int walk, int r, int tw, size_t smem, const DeviceInfo& di) {
    int bps = (int)(di.smem_per_sm / (smem + 1024));
    bps = std::max(1, std::min(bps, di.max_blocks_per_sm));
    const long tiles_x = (W + tw - 1) / tw;
    const long target = (long)di.num_sms * bps * (dims == 3 ? ((r >= 5 && r < 8) ? 2 : 4) : ((r >= 12 && r < 32) ? 2 : 1));
    long sh = (walk * tiles_x * (long)lines + target - 1) / target;
    const long n = 2L * r + 1;
    sh = std::max(sh, std::min(n, 96L));
    sh = std::max(sh, 8L);
    sh = std::min(sh, (long)walk);
    return (int)std::max(1L, sh);
}

// Edge strips: the r steps at each end of the walk axis, whose windows are
// clamped, are cut into strips of 8 so that the slow tiles near the image
// corners (their medians move to new tree nodes almost every step) stay
// short; the interior keeps strips of sh.  Returns the number of strips.
int strip_layout(int walk, int sh, int r, int* she, int* ne) {
    *she = 0;
    *ne = 0;
    if (sh <= 0) return 0;
    const int e = 8;
    const int k = (r + e - 1) / e;
    if (r >= 8 && e < sh && 2L * k * e + sh <= walk) {
        *she = e;
        *ne = k;
    }
    const long rest = walk - 2L * *ne * *she;
    return 2 * *ne + (int)((rest + sh - 1) / sh);
}

PlanH default_plan(int dims, int es, int W, int lines, int walk, int r, const DeviceInfo& di) {
    PlanH p{};
    p.es = es;
    p.path = ((dims == 2 && r <= SORTNET_MAX_R2D) || (dims == 3 && r == 1)) ? 1 : 2;
    p.cw = counter_width(dims, r);
    p.ppl = 1;  // 128 outputs per tile
    // shared memory per tile: four resident tiles (16 warps; the kernel is
    // then compiled for 128 registers) per SM in 2D -- node builds over the
    // requesting outputs' columns are cheap enough that more warps beat more
    // cached nodes -- and in 3D for 5 <= r < 40; three otherwise
    const int tiles_per_sm = (dims == 2 || (r >= 5 && r < 40)) ? 4 : 3;
    const size_t per_sm = (size_t)di.smem_per_sm / tiles_per_sm - 1024;
    const size_t budget = std::min((size_t)di.smem_optin, per_sm);
    size_slots(p, dims, r, budget);
    p.sh = strip_length(dims, W, lines, walk, r, BLOCK_THREADS * p.ppl, plan_smem(p, r), di);
    return p;
}

static void apply_plan(PlanH& p, const hrm_plan& hp, int dims, int W, int lines, int walk, int r,
                       const DeviceInfo& di) {
    if (hp.tile_width == BLOCK_THREADS || hp.tile_width == 2 * BLOCK_THREADS) p.ppl = hp.tile_width / BLOCK_THREADS;
    if (hp.slot_kbytes > 0) size_slots(p, dims, r, (size_t)hp.slot_kbytes * 1024);
    else size_slots(p, dims, r, plan_smem(p, r));
    p.sh = hp.strip_height > 0 ? std::min(hp.strip_height, walk)
                               : strip_length(dims, W, lines, walk, r, BLOCK_THREADS * p.ppl, plan_smem(p, r), di);
    if (hp.path == 1 || hp.path == 2) p.path = hp.path;
    if (hp.tree == 1 || hp.tree == 2) p.tree = hp.tree;
}

// ---- node-cache feedback (2D histogram kernel, default plans only) ----------------
// The default plan (four tiles of ~55 KB per SM) suits images whose tile rows
// reuse a few tree nodes.  Rows that visit a few dozen distinct nodes (noisy
// 16-bit images with a compact mode) rebuild nodes all the time and run 2-3x
// faster with as many node slots as fit in up to 200 KB per tile (one or two
// tiles per SM); rows that visit even more (wide 16-bit distributions) rebuild
// with either cache and lose by the fewer warps.  Which case a problem class
// is cannot be seen on the host without reading the image, so the class is
// measured: its first call counts the node installs of its tiles into a
// device counter and copies the count back asynchronously.  The second call
// waits for that copy; if a tile row installed more than FB_DEEP_RATE nodes,
// it runs the large-cache plan and is counted the same way, the third call
// waits for that count, and the class keeps the large cache only if it cut the
// installs at least FB_KEEP_CUT-fold, else it returns to the default for good.
// From the third call on a class runs one settled plan (stable latency);
// outputs never depend on the plan.  A set, tuned or
// forced plan takes precedence and switches the feedback off for its class.
constexpr int FB_MAX = 4096;             // counters per device
constexpr double FB_DEEP_RATE = 0.75;    // node installs per tile row that call for a trial
constexpr double FB_KEEP_CUT = 3.0;      // the trial must cut the installs this much
constexpr int FB_DEEP_KBYTES = 200;      // shared-memory budget per tile of the large-cache plan
struct FbDevice {
    unsigned* d = nullptr;  // FB_MAX device counters
    unsigned* h = nullptr;  // their pinned copies
    int used = 0;
};
// States: 0 unmeasured; 1 default count in flight; 2 decided (deep or not);
// 3 trial of the large cache due; 4 trial count in flight.
struct FbClass {
    int state = 0;
    int idx = -1;
    double rows = 0;        // tile rows of a counted launch
    double rate0 = 0;       // installs per tile row with the default plan
    cudaEvent_t ev = nullptr;
    bool deep = false;
};
static std::map<int, FbDevice> g_fbdev;
static std::map<std::pair<int, std::tuple<int, int, int, int, int, int, unsigned>>, FbClass> g_fb;

static bool fb_eligible(const ProblemKey& k, const hrm_plan* force) {
    hrm_plan hp;
    return k.dims == 2 && !force && !env_forced_path() && !plan_lookup(k, &hp);
}

// Should this call of the class run the large-cache plan?  (Never blocks.)
static bool fb_deep(const ProblemKey& k) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_fb.find({dev, tkey(k)});
    if (it == g_fb.end()) return false;
    FbClass& c = it->second;
    if (c.state == 1 || c.state == 4) {
        // wait for the previous call's 4-byte count: the second call of a
        // class decides whether to try the large cache, the third whether to
        // keep it, and every later call runs the settled plan
        const bool clean = cudaPeekAtLastError() == cudaSuccess;
        const cudaError_t q = cudaEventSynchronize(c.ev);
        if (q == cudaSuccess) {
            const double rate = c.rows > 0 ? (double)g_fbdev[dev].h[c.idx] / c.rows : 0.0;
            if (c.state == 1) {
                c.rate0 = rate;
                c.state = rate > FB_DEEP_RATE ? 3 : 2;
                c.deep = false;
            } else {
                c.deep = rate * FB_KEEP_CUT <= c.rate0;
                c.state = 2;
            }
        } else {
            if (clean) cudaGetLastError();  // the count is lost: keep the default plan
            c.state = 2;
            c.deep = false;
        }
    }
    return c.state == 3 || c.state == 4 || (c.state == 2 && c.deep);
}

// A counted launch is due (first call, or the trial of the large cache): a
// zeroed device counter for it, else null.
static unsigned* fb_begin(const ProblemKey& k, double rows, cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    FbClass& c = g_fb[{dev, tkey(k)}];
    if (c.state != 0 && c.state != 3) return nullptr;
    const int next = c.state == 0 ? 1 : 4;
    c.state = 2;  // unless everything below succeeds, the class keeps the default plan
    c.deep = false;
    FbDevice& fd = g_fbdev[dev];
    if (!fd.d) {
        if (cudaMalloc(&fd.d, sizeof(unsigned) * FB_MAX) != cudaSuccess) return (void)cudaGetLastError(), nullptr;
        if (cudaMallocHost(&fd.h, sizeof(unsigned) * FB_MAX) != cudaSuccess) return (void)cudaGetLastError(), nullptr;
        memset(fd.h, 0, sizeof(unsigned) * FB_MAX);
    }
    if (!fd.h) return nullptr;
    if (c.idx < 0) {
        if (fd.used >= FB_MAX) return nullptr;
        if (cudaEventCreateWithFlags(&c.ev, cudaEventDisableTiming) != cudaSuccess)
            return (void)cudaGetLastError(), nullptr;
        c.idx = fd.used++;
    }
    c.rows = rows;
    if (cudaMemsetAsync(fd.d + c.idx, 0, sizeof(unsigned), st) != cudaSuccess) return (void)cudaGetLastError(), nullptr;
    c.state = next;
    return fd.d + c.idx;
}

// After a counted launch: bring the count back and mark when it lands.
static void fb_end(const ProblemKey& k, cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_mu);
    FbClass& c = g_fb[{dev, tkey(k)}];
    FbDevice& fd = g_fbdev[dev];
    if (cudaMemcpyAsync(fd.h + c.idx, fd.d + c.idx, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(c.ev, st) != cudaSuccess) {
        cudaGetLastError();
        c.state = 2;
        c.deep = false;
    }
}

PlanH resolve_plan(int dtype, int dims, int W, int H, int D, int r, unsigned flags, const DeviceInfo& di,
                   const hrm_plan* force, bool feedback) {
    const int lines = dims == 3 ? H : 1;
    const int walk = dims == 3 ? D : H;
    const int es = dtype == HRM_U16 ? 2 : 1;
    PlanH p = default_plan(dims, es, W, lines, walk, r, di);
    hrm_plan hp;
    const ProblemKey key{dtype, dims, W, H, D, r, flags};
    if (plan_lookup(key, &hp)) apply_plan(p, hp, dims, W, lines, walk, r, di);
    else if (feedback && p.path == 2 && fb_eligible(key, force) && fb_deep(key)) {
        const hrm_plan deep{0, p.sh, FB_DEEP_KBYTES, 0};  // one tile per SM, the default strips
        apply_plan(p, deep, dims, W, lines, walk, r, di);
    }
    if (force) apply_plan(p, *force, dims, W, lines, walk, r, di);
    else if (env_forced_path()) p.path = env_forced_path();
    // the shared-memory plan must fit the device
    while (p.nslots > 2 && plan_smem(p, r) > (size_t)di.smem_optin) --p.nslots;
    if (plan_smem(p, r) > (size_t)di.smem_optin) p.ring = 0;
    while (p.ppl > 1 && plan_smem(p, r) > (size_t)di.smem_optin) p.ppl /= 2;
    return p;
}

// ---- validation ---------------------------------------------------------------------
static bool overlap(const void* a, size_t alen, const void* b, size_t blen) {
    auto x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + blen && y < x + alen;
}

int validate(const Image& im, int r, int border, unsigned flags) {
    if (im.dtype != HRM_U8 && im.dtype != HRM_U16) return fail(HRM_EINVAL, "dtype must be HRM_U8 or HRM_U16");
    if (border != HRM_BORDER_REPLICATE) return fail(HRM_EINVAL, "only HRM_BORDER_REPLICATE is supported");
    if (flags & ~(unsigned)HRM_ADAPTIVE) return fail(HRM_EINVAL, "unknown flag bits");
    if (im.W < 0 || im.H < 0 || im.D < 0) return fail(HRM_EINVAL, "negative image size");
    const int rmax = im.dims == 3 ? HRM_MAX_RADIUS_3D : HRM_MAX_RADIUS_2D;
    if (r < 0 || r > rmax) return fail(HRM_EINVAL, "radius out of range");
    if (im.W == 0 || im.H == 0 || im.D == 0) return HRM_OK;
    const size_t es = im.dtype == HRM_U16 ? 2 : 1;
    if (!im.src || !im.dst) return fail(HRM_EINVAL, "null image pointer");
    if (im.sp < im.W * es || im.dp < im.W * es) return fail(HRM_EINVAL, "pitch smaller than a row");
    if (((uintptr_t)im.src | (uintptr_t)im.dst | im.sp | im.dp) % es) return fail(HRM_EINVAL, "misaligned pointer or pitch");
    size_t sl = (size_t)(im.H - 1) * im.sp + im.W * es, dl = (size_t)(im.H - 1) * im.dp + im.W * es;
    if (im.dims == 3 && im.D > 1) {  // a single slice never uses its slice pitch
        if (im.sslice < (size_t)im.H * im.sp || im.dslice < (size_t)im.H * im.dp)
            return fail(HRM_EINVAL, "slice pitch smaller than a slice");
        if ((im.sslice | im.dslice) % es) return fail(HRM_EINVAL, "misaligned slice pitch");
        sl += (size_t)(im.D - 1) * im.sslice;
        dl += (size_t)(im.D - 1) * im.dslice;
    }
    if (overlap(im.src, sl, im.dst, dl)) return fail(HRM_EINVAL, "src and dst overlap");
    return HRM_OK;
}

// ---- filters ---------------------------------------------------------------------------
int make_hist_job(const Image& im, int r, uint32_t K, unsigned flags, int drop_bits, const PlanH& p,
                  const LevelDesc* desc, unsigned* err, HistJob* job) {
    (void)flags;
    const int es = im.dtype == HRM_U16 ? 2 : 1;
    HistJob j{};
    j.src = (const unsigned char*)im.src;
    j.dst = (unsigned char*)im.dst;
    j.s_row = im.sp;
    j.s_slice = im.sslice;
    j.d_row = im.dp;
    j.d_slice = im.dslice;
    j.W = im.W;
    j.H = im.H;
    j.D = im.dims == 3 ? im.D : 1;
    j.dims = im.dims;
    j.r = r;
    j.K = K;
    j.drop_bits = drop_bits;
    j.elem = es;
    j.err = err;
    j.desc = desc;
    j.fixed_shift = desc ? 0 : 4;
    j.ppl = p.ppl;
    j.cw = p.cw;
    j.sh = p.sh;
    j.nslots = p.nslots;
    j.ring = p.ring;
    const int tw = BLOCK_THREADS * p.ppl;
    const int walk = im.dims == 3 ? im.D : im.H;
    const int lines = im.dims == 3 ? im.H : 1;
    j.tiles_x = (im.W + tw - 1) / tw;
    const int nstrips = strip_layout(walk, p.sh, r, &j.she, &j.ne);
    j.nint = nstrips - 2 * j.ne;
    const long nt = im.dims == 2 && j.tiles_x >= 2
                        ? 4L * j.ne * j.she + 2L * j.ne * (j.tiles_x - 2) + (long)j.tiles_x * j.nint
                        : (long)j.tiles_x * lines * nstrips;
    if (nt > 0x7FFFFFFFL) return fail(HRM_ENOTSUP, "too many tiles");
    j.ntiles = (int)nt;
    *job = j;
    return HRM_OK;
}

static int copy_image(const Image& im, cudaStream_t st) {
    const size_t es = im.dtype == HRM_U16 ? 2 : 1;
    cudaError_t e = cudaSuccess;
    if (im.dims == 2) {
        e = cudaMemcpy2DAsync(im.dst, im.dp, im.src, im.sp, im.W * es, im.H, cudaMemcpyDeviceToDevice, st);
    } else {
        for (int z = 0; z < im.D && e == cudaSuccess; ++z)
            e = cudaMemcpy2DAsync((unsigned char*)im.dst + z * im.dslice, im.dp,
                                  (const unsigned char*)im.src + z * im.sslice, im.sp, im.W * es, im.H,
                                  cudaMemcpyDeviceToDevice, st);
    }
    return e == cudaSuccess ? HRM_OK : cuda_fail(e, "cudaMemcpy2DAsync");
}

int filter_impl(const Image& im, int r, long rank, unsigned flags, int drop_bits, const hrm_plan* force,
                cudaStream_t st, const LevelDesc* given) {
    if (im.W == 0 || im.H == 0 || im.D == 0) return HRM_OK;
    const int es = im.dtype == HRM_U16 ? 2 : 1;
    const long n = 2L * r + 1, N = im.dims == 3 ? n * n * n : n * n;
    if (rank < -1 || rank >= N) return fail(HRM_EINVAL, "rank out of range");
    const bool median = rank < 0 || rank == (N - 1) / 2;
    const uint32_t K = (uint32_t)(rank < 0 ? (N + 1) / 2 : rank + 1);
    if (r == 0) return copy_image(im, st);
    const DeviceInfo& di = device_info();
    const PlanH p = resolve_plan(im.dtype, im.dims, im.W, im.H, im.D, r, flags, di, force, true);
    cudaError_t e;
    if (im.dims == 2 && p.path == 1 && r <= SORTNET_MAX_R2D && median && drop_bits == 0) {
        // rows per warp: about 32 warp tiles per SM (latency hiding for the
        // memory-bound 3x3 network), but at least 8 rows so the 2r rows each
        // warp reads ahead stay a small share
        const long tw = r <= 2 ? 256 : 2 * (32 - 2 * ((r + 1) / 2));
        const long tiles_x = (im.W + tw - 1) / tw;
        const long want = (long)di.num_sms * 32;
        const int rpw = (int)std::max(8L, std::min(32L, (im.H * tiles_x + want - 1) / want));
        e = launch_sortnet2d(es, r, im.src, im.sp, im.dst, im.dp, im.W, im.H, rpw, st);
        return e == cudaSuccess ? HRM_OK : cuda_fail(e, "sortnet launch");
    }
    if (im.dims == 3 && p.path == 1 && r == 1 && median && drop_bits == 0 && im.H <= 65535) {
        e = launch_sortnet3d(es, im.src, im.sp, im.sslice, im.dst, im.dp, im.dslice, im.W, im.H, im.D, 32, st);
        return e == cudaSuccess ? HRM_OK : cuda_fail(e, "sortnet3d launch");
    }
    Workspace* ws = nullptr;
    int rc = workspace_for(st, &ws);
    if (rc) return rc;
    const bool adaptive = plan_adaptive(p, flags);
    const LevelDesc* desc = given;
    if (!desc && (es == 2 || adaptive)) {
        e = launch_levels(es, adaptive, im.src, im.sp, im.dims == 3 ? im.sslice : 0, im.W, im.H,
                          im.dims == 3 ? im.D : 1, ws->desc, ws->hist, di.num_sms, st);
        if (e != cudaSuccess) return cuda_fail(e, "level pre-pass launch");
        desc = ws->desc;
    }
    HistJob job;
    rc = make_hist_job(im, r, K, flags, drop_bits, p, desc, ws->err, &job);
    if (rc) return rc;
    if (plan_smem(p, r) > (size_t)di.smem_optin)
        return fail(HRM_ENOTSUP, "plan needs more shared memory than the device offers");
    const ProblemKey key{im.dtype, im.dims, im.W, im.H, im.D, r, flags};
    if (p.path == 2 && drop_bits == 0 && fb_eligible(key, force)) {
        const double rows = (double)((im.W + BLOCK_THREADS * p.ppl - 1) / (BLOCK_THREADS * p.ppl)) * im.H;
        job.stats = fb_begin(key, rows, st);
    }
    e = launch_hist(job, st);
    if (e != cudaSuccess) return cuda_fail(e, "hist launch");
    if (job.stats) fb_end(key, st);
    return HRM_OK;
}

int topology_check(const hrm_topology* t) {
    if (!t) return fail(HRM_EINVAL, "null topology");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return fail(HRM_EINVAL, "topology belongs to another device");
    return HRM_OK;
}

int topology_device_of(const hrm_topology* t) { return t->device; }

int topology_update(hrm_topology* t, int dtype, const void* dst, size_t dp, int W, int H, cudaStream_t st) {
    const cudaError_t e = launch_topology_from_output(dtype == HRM_U16 ? 2 : 1, dst, dp, W, H, t->desc, t->hist,
                                                      device_info().num_sms, st);
    if (e != cudaSuccess) return cuda_fail(e, "topology update launch");
    t->dtype = dtype;
    return HRM_OK;
}

}  // namespace hrm

using namespace hrm;

extern "C" {

int hrm_version(void) { return HRM_VERSION; }

const char* hrm_last_error(void) { return g_err.c_str(); }

int hrm_filter2d(int dtype, const void* src, size_t src_pitch, void* dst, size_t dst_pitch, int width,
                 int height, int radius, int border, unsigned flags, void* stream) {
    Image im{dtype, 2, src, dst, src_pitch, 0, dst_pitch, 0, width, height, 1};
    int rc = validate(im, radius, border, flags);
    if (rc) return rc;
    return filter_impl(im, radius, -1, flags, 0, nullptr, (cudaStream_t)stream);
}

int hrm_rank_filter2d(int dtype, const void* src, size_t src_pitch, void* dst, size_t dst_pitch,
                      int width, int height, int radius, long rank, int border, unsigned flags,
                      void* stream) {
    Image im{dtype, 2, src, dst, src_pitch, 0, dst_pitch, 0, width, height, 1};
    int rc = validate(im, radius, border, flags);
    if (rc) return rc;
    const long n = 2L * radius + 1;
    if (rank < 0 || rank >= n * n) return fail(HRM_EINVAL, "rank out of range");
    return filter_impl(im, radius, rank, flags, 0, nullptr, (cudaStream_t)stream);
}

int hrm_filter3d(int dtype, const void* src, size_t src_pitch, size_t src_slice_pitch, void* dst,
                 size_t dst_pitch, size_t dst_slice_pitch, int width, int height, int depth, int radius,
                 int border, unsigned flags, void* stream) {
    Image im{dtype, 3, src, dst, src_pitch, src_slice_pitch, dst_pitch, dst_slice_pitch, width, height, depth};
    int rc = validate(im, radius, border, flags);
    if (rc) return rc;
    return filter_impl(im, radius, -1, flags, 0, nullptr, (cudaStream_t)stream);
}

int hrm_rank_filter3d(int dtype, const void* src, size_t src_pitch, size_t src_slice_pitch, void* dst,
                      size_t dst_pitch, size_t dst_slice_pitch, int width, int height, int depth,
                      int radius, long rank, int border, unsigned flags, void* stream) {
    Image im{dtype, 3, src, dst, src_pitch, src_slice_pitch, dst_pitch, dst_slice_pitch, width, height, depth};
    int rc = validate(im, radius, border, flags);
    if (rc) return rc;
    const long n = 2L * radius + 1;
    if (rank < 0 || rank >= n * n * n) return fail(HRM_EINVAL, "rank out of range");
    return filter_impl(im, radius, rank, flags, 0, nullptr, (cudaStream_t)stream);
}

int hrm_filter2d_lowprec(int dtype, const void* src, size_t src_pitch, void* dst, size_t dst_pitch,
                         int width, int height, int radius, int drop_bits, void* stream) {
    Image im{dtype, 2, src, dst, src_pitch, 0, dst_pitch, 0, width, height, 1};
    int rc = validate(im, radius, HRM_BORDER_REPLICATE, 0);
    if (rc) return rc;
    if (drop_bits < 0 || drop_bits > 12) return fail(HRM_EINVAL, "drop_bits must be in 0..12");
    if (drop_bits == 0) return filter_impl(im, radius, -1, 0, 0, nullptr, (cudaStream_t)stream);
    hrm_plan force{0, 0, 0, 2};  // the early-stopping walk lives in the histogram kernel
    return filter_impl(im, radius, -1, 0, drop_bits, &force, (cudaStream_t)stream);
}

int hrm_topology_create(hrm_topology** out) {
    if (!out) return fail(HRM_EINVAL, "null topology pointer");
    *out = nullptr;
    auto* t = new (std::nothrow) hrm_topology();
    if (!t) return fail(HRM_ENOMEM, "topology");
    cudaGetDevice(&t->device);
    if (cudaMalloc(&t->desc, sizeof(LevelDesc)) != cudaSuccess ||
        cudaMalloc(&t->hist, sizeof(uint32_t) * 4096) != cudaSuccess) {
        cudaFree(t->desc);
        cudaFree(t->hist);
        delete t;
        clear_error();
        return fail(HRM_ENOMEM, "topology device buffers");
    }
    *out = t;
    return HRM_OK;
}

int hrm_topology_destroy(hrm_topology* t) {
    if (!t) return HRM_OK;
    cudaDeviceSynchronize();  // calls that use the topology may still be in flight
    cudaFree(t->desc);
    cudaFree(t->hist);
    delete t;
    return HRM_OK;
}

int hrm_filter2d_video(int dtype, const void* src, size_t src_pitch, void* dst, size_t dst_pitch, int width,
                       int height, int radius, hrm_topology* topo, void* stream) {
    int rc = topology_check(topo);
    if (rc) return rc;
    Image im{dtype, 2, src, dst, src_pitch, 0, dst_pitch, 0, width, height, 1};
    rc = validate(im, radius, HRM_BORDER_REPLICATE, 0);
    if (rc) return rc;
    if (width == 0 || height == 0) return HRM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const LevelDesc* given = topo->dtype == dtype ? topo->desc : nullptr;
    rc = filter_impl(im, radius, -1, given ? 0u : (unsigned)HRM_ADAPTIVE, 0, nullptr, st, given);
    if (rc) return rc;
    return topology_update(topo, dtype, dst, dst_pitch, width, height, st);
}

int hrm_topology_get(hrm_topology* topo, void* stream, hrm_topology_info* out) {
    if (!topo || !out) return fail(HRM_EINVAL, "null topology or info pointer");
    LevelDesc d{};
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaMemcpy(&d, topo->desc, sizeof(d), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "topology read");
    *out = hrm_topology_info{};
    out->dtype = topo->dtype;
    if (topo->dtype) {
        out->mode = d.mode;
        out->vmin = d.vmin;
        out->vmax = d.vmax;
        if (d.mode == 1)  // a uniform top level leaves edge[] unused: report zeros
            for (int i = 0; i < 17; ++i) out->edge[i] = d.edge[i];
    }
    return HRM_OK;
}

int hrm_device_status(void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    // a stream without a workspace has run no kernel that writes one: nothing
    // is allocated here, so callers of the no-allocation path may call this too
    Workspace* ws = workspace_find(st);
    unsigned host = 0;
    cudaError_t e = cudaSuccess;
    if (ws) e = cudaMemcpyAsync(&host, ws->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "device status");
    if (host) {
        e = cudaMemsetAsync(ws->err, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "device status clear");
    }
    unsigned na = 0;
    const int rc = noalloc_error_take(st, &na);
    if (rc) return rc;
    if (host) return fail(HRM_EDEVICE, "kernel reported device error code " + std::to_string(host));
    if (na)
        return fail(HRM_EDEVICE, "a hrm_filter_batch_noalloc kernel reported device error code " +
                                     std::to_string(na));
    return HRM_OK;
}

int hrm_get_plan(int dtype, int dims, int width, int height, int depth, int radius, unsigned flags,
                 hrm_plan* plan) {
    if (!plan) return fail(HRM_EINVAL, "null plan");
    if (dims != 2 && dims != 3) return fail(HRM_EINVAL, "dims must be 2 or 3");
    ProblemKey k{dtype, dims, width, height, depth, radius, flags};
    if (plan_lookup(k, plan)) return HRM_OK;
    const DeviceInfo& di = device_info();
    PlanH p = resolve_plan(dtype, dims, width, height, depth, radius, flags, di, nullptr, true);
    plan->tile_width = BLOCK_THREADS * p.ppl;
    plan->strip_height = p.sh;
    plan->slot_kbytes = (int)((plan_smem(p, radius) + 1023) / 1024);
    plan->path = p.path;
    plan->tree = p.path == 2 ? (plan_adaptive(p, flags) ? 2 : 1) : 0;
    return HRM_OK;
}

int hrm_set_plan(int dtype, int dims, int width, int height, int depth, int radius, unsigned flags,
                 const hrm_plan* plan) {
    if (!plan) return fail(HRM_EINVAL, "null plan");
    if (dims != 2 && dims != 3) return fail(HRM_EINVAL, "dims must be 2 or 3");
    if (plan->tile_width != 0 && plan->tile_width != 128 && plan->tile_width != 256)
        return fail(HRM_EINVAL, "tile_width must be 128 or 256");
    if (plan->path < 0 || plan->path > 2) return fail(HRM_EINVAL, "path must be 0, 1 or 2");
    if (plan->tree < 0 || plan->tree > 2) return fail(HRM_EINVAL, "tree must be 0, 1 or 2");
    plan_store(ProblemKey{dtype, dims, width, height, depth, radius, flags}, *plan);
    return HRM_OK;
}

int hrm_plan_save(const char* path) {
    if (!path) return fail(HRM_EINVAL, "null path");
    std::ofstream f(path);
    if (!f) return fail(HRM_EINVAL, std::string("cannot write ") + path);
    std::lock_guard<std::mutex> lk(g_mu);
    f << "# hrm plan cache v2: dtype dims width height depth radius flags tile_width strip_height slot_kbytes path tree\n";
    for (auto& kv : g_plans) {
        auto& k = kv.first;
        auto& p = kv.second;
        f << std::get<0>(k) << ' ' << std::get<1>(k) << ' ' << std::get<2>(k) << ' ' << std::get<3>(k) << ' '
          << std::get<4>(k) << ' ' << std::get<5>(k) << ' ' << std::get<6>(k) << ' ' << p.tile_width << ' '
          << p.strip_height << ' ' << p.slot_kbytes << ' ' << p.path << ' ' << p.tree << '\n';
    }
    return f ? HRM_OK : fail(HRM_EINVAL, "write failed");
}

int hrm_plan_load(const char* path) {
    if (!path) return fail(HRM_EINVAL, "null path");
    std::ifstream f(path);
    if (!f) return fail(HRM_EINVAL, std::string("cannot read ") + path);
    std::string line;
    int nload = 0;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream is(line);
        ProblemKey k{};
        hrm_plan p{};
        if (!(is >> k.dtype >> k.dims >> k.width >> k.height >> k.depth >> k.radius >> k.flags >>
              p.tile_width >> p.strip_height >> p.slot_kbytes >> p.path))
            return fail(HRM_EINVAL, "malformed plan line: " + line);
        std::string rest;
        if (is >> rest) {  // the tree field (absent in lines written before it existed)
            if (rest.size() != 1 || rest[0] < '0' || rest[0] > '2' || (is >> rest))
                return fail(HRM_EINVAL, "malformed plan line: " + line);
            p.tree = rest[0] - '0';
        }
        plan_store(k, p);
        ++nload;
    }
    return HRM_OK;
}

}  // extern "C"

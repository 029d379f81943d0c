// hist_common.cuh -- level descriptor and per-warp helpers shared by the 2D
// and 3D hierarchical-histogram kernels and the batched kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "hrm_common.cuh"

namespace hrm {

// Level structure of the interval-occurrences tree (Section III).
//
// Top level: 16 coarse intervals [e_c, e_{c+1}).  Uniform mode (Section III,
// uniform IOT): e_c = c << shift with shift = max(0, bitlen(vmax) - 4), i.e.
// the tree of effective bit depth d = bitlen(vmax) anchored at 0.  Adaptive
// mode (Section III-C): e_c are data-driven (a power-of-16 split of the range
// a median estimate occupies; see prepass.cu).  Below each coarse interval the
// tree is uniform, with D_c = bitlen(width_c - 1) bits taken 4 bits (16
// children) per level.
struct LevelDesc {
    uint32_t mode;      // 0 = uniform, 1 = adaptive
    uint32_t vmin;      // observed minimum (filled by the pre-pass)
    uint32_t vmax;      // observed maximum
    uint32_t count;     // pixels seen
    uint32_t edge[17];  // adaptive coarse edges, edge[16] = vmax + 1
    uint32_t pad[11];
};
static_assert(sizeof(LevelDesc) == 128, "LevelDesc layout");

// Optional instrumentation (build with -DHRM_COUNT_OPS): per-phase cycle and
// event counters, accumulated per warp and flushed once per tile.  The normal
// library compiles all of it away.
enum CountId {
    CNT_TILES = 0, CNT_ROWS, CNT_CYC_TOTAL, CNT_CYC_INIT, CNT_CYC_COLUMNS, CNT_CYC_RESOLVE,
    CNT_CYC_INSTALL, CNT_CYC_WINDOW, CNT_CYC_ADVANCE, CNT_INSTALLS, CNT_ROUNDS, CNT_PREFIXES,
    CNT_DIRECT_ROUNDS, CNT_LEVELS, CNT_CYC_ALLOC, CNT_NUM
};
#ifdef HRM_COUNT_OPS
static __device__ unsigned long long g_hrm_counters[CNT_NUM];
static __device__ int g_hrm_count_tile = -1;  // >= 0: only that tile adds to the counters
// per-tile timeline of the last launch (tile id -> start/end global time, SM)
constexpr int CNT_TILE_CAP = 1 << 15;
static __device__ unsigned long long g_hrm_tile_t0[CNT_TILE_CAP], g_hrm_tile_t1[CNT_TILE_CAP];
static __device__ unsigned g_hrm_tile_sm[CNT_TILE_CAP];
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned sm_id() {
    unsigned s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}
struct OpCounters {
    unsigned long long v[CNT_NUM];
    long long t0;
    __device__ void reset() { for (int i = 0; i < CNT_NUM; ++i) v[i] = 0; }
    __device__ void add(int i, unsigned long long x) { v[i] += x; }
    __device__ void mark() { t0 = clock64(); }
    __device__ void lap(int i) { long long t = clock64(); v[i] += (unsigned long long)(t - t0); t0 = t; }
    __device__ void flush(int tile = -1) {
        if (g_hrm_count_tile >= 0 && tile != g_hrm_count_tile) return;
        if ((threadIdx.x & 31) == 0)
            for (int i = 0; i < CNT_NUM; ++i) if (v[i]) atomicAdd(&g_hrm_counters[i], v[i]);
    }
    __device__ void tile(int id, unsigned long long ns0) {
        if (id >= 0 && id < CNT_TILE_CAP) {
            g_hrm_tile_t0[id] = ns0;
            g_hrm_tile_t1[id] = global_ns();
            g_hrm_tile_sm[id] = sm_id();
        }
    }
    __device__ unsigned long long now_ns() { return global_ns(); }
};
#else
struct OpCounters {
    __device__ void tile(int, unsigned long long) {}
    __device__ unsigned long long now_ns() { return 0; }
    __device__ void reset() {}
    __device__ void add(int, unsigned long long) {}
    __device__ void mark() {}
    __device__ void lap(int) {}
    __device__ void flush(int = -1) {}
};
#endif

constexpr uint32_t KEY_NONE = 0xFFFFFFFFu;
constexpr int HASH_SIZE = 64;
constexpr int MAX_SLOTS = 32;
constexpr int META_BYTES = 4096;  // per-tile metadata block (see Meta)
// Node requests recorded per round.  A round installs at most one node per
// free slot (< MAX_SLOTS), so later requests would wait for the next round
// anyway; requests that find the tables full are simply retried then.
constexpr int REQ_MAX = 64;
constexpr int PREQ_SIZE = 64;     // pending-request hash (deduplicates requests)
constexpr uint8_t NO_SLOT = 0xFF;

// Per-warp metadata in shared memory.  Resident nodes are found through
// direct tables for the first two levels below the root (level 1: coarse
// interval c; level 2: c and the first 4-bit digit) and through a small hash
// for deeper levels (16-bit data only).
struct Meta {
    uint32_t e[17];        // coarse edges
    uint32_t D[16];        // sub-tree bits per coarse interval
    uint32_t key[MAX_SLOTS];
    uint32_t stamp[MAX_SLOTS];
    uint32_t pin[MAX_SLOTS];
    uint32_t hash[HASH_SIZE];  // levels >= 3: (key << 8) | slot
    uint32_t lmask[8];     // lmask[l] bit c: a slot at level l for coarse c exists; lmask[0] = OR of all
    int32_t ushift;        // >= 0: uniform shift; -1: adaptive
    uint32_t ndeep;        // resident slots at levels >= 3
    uint32_t pad[2];
    uint8_t lut1[16];      // level 1: c -> slot
    uint8_t lut2[256];     // level 2: (c << 4) | d1 -> slot
    // block coordination (one tile per thread block)
    uint32_t preq[PREQ_SIZE];   // pending requests of this round (keys)
    uint32_t req[REQ_MAX];      // distinct requested keys in arrival order
    uint32_t nbuild;
    uint32_t ninst;             // build entries installed by this tile (node-cache feedback)
    uint32_t pad2[2];
    uint32_t build_slot[MAX_SLOTS];
    uint32_t build_key[MAX_SLOTS];
    uint32_t wtot[8][8];        // per-warp totals of the block prefix scan
    // Column spans.  A node below the root is built only over the tile
    // columns its requesting outputs' windows cover (plus a margin) and
    // widened in place when a later output needs more; clo/chi is the range
    // of a slot's records that hold counts (the rest is stale).
    int16_t clo[MAX_SLOTS], chi[MAX_SLOTS];
    int32_t preq_lo[PREQ_SIZE], preq_hi[PREQ_SIZE];  // span wanted by each pending request
    uint8_t req_h[REQ_MAX];                           // its pending-hash position
    int16_t build_lo[MAX_SLOTS], build_hi[MAX_SLOTS];  // columns of each build entry
    uint32_t build_off[MAX_SLOTS + 1];                // prefix of the entries' widths
    // Per-round bookkeeping, triple-buffered: round k uses rs[k % 3] and
    // clears rs[(k + 1) % 3] for round k + 1.  The first round of a level is
    // resolved before the barrier that closes the previous level, while other
    // warps may still read rs[(k - 1) % 3]; the buffer being cleared was last
    // read in round k - 2, before round k - 1's barrier.
    struct Round {
        uint32_t nreq;          // requests recorded
        uint32_t used;          // slots used by the outputs resolved this round
        uint32_t maxres;        // most outputs of one thread resolved this round
        uint32_t pad;
        int32_t span_lo[MAX_SLOTS];
        int32_t span_hi[MAX_SLOTS];
    } rs[3];
};
static_assert(sizeof(Meta) <= META_BYTES, "Meta too large");

__device__ __forceinline__ uint32_t node_key(int level, int c, uint32_t pre) {
    return ((uint32_t)level << 20) | ((uint32_t)c << 16) | pre;
}
__device__ __forceinline__ uint32_t hash_of(uint32_t key) { return (key * 2654435761u) >> 26; }

__device__ __forceinline__ int coarse_of(const Meta& m, uint32_t v) {
    if (m.ushift >= 0) return min((int)(v >> m.ushift), 15);
    int c = 0;
    c += v >= m.e[c + 8] ? 8 : 0;
    c += v >= m.e[c + 4] ? 4 : 0;
    c += v >= m.e[c + 2] ? 2 : 0;
    c += v >= m.e[c + 1] ? 1 : 0;
    return c;
}

__device__ __forceinline__ int hash_lookup(const Meta& m, uint32_t key) {
    uint32_t h = hash_of(key);
#pragma unroll 1
    for (int i = 0; i < HASH_SIZE; ++i) {
        const uint32_t ent = m.hash[h];
        if (ent == KEY_NONE) return -1;
        if ((ent >> 8) == key) return (int)(ent & 0xFFu);
        h = (h + 1) & (HASH_SIZE - 1);
    }
    return -1;
}

// Slot holding node (level >= 1, coarse interval c, digit prefix pre), or -1.
__device__ __forceinline__ int slot_lookup(const Meta& m, int level, int c, uint32_t pre) {
    int s;
    if (level == 1) s = m.lut1[c];
    else if (level == 2) s = m.lut2[(c << 4) | (int)(pre & 15u)];
    else return m.ndeep ? hash_lookup(m, node_key(level, c, pre)) : -1;
    return s == NO_SLOT ? -1 : s;
}

__device__ __forceinline__ int slot_lookup(const Meta& m, uint32_t key) {
    return slot_lookup(m, (int)(key >> 20), (int)((key >> 16) & 15), key & 0xFFFFu);
}

// Reset all tables with only the root (slot 0) resident (call from warp 0).
__device__ __forceinline__ void slots_reset(Meta& m) {
    const int lane = threadIdx.x & 31;
    m.key[lane] = lane == 0 ? 0u : KEY_NONE;
    m.stamp[lane] = lane == 0 ? 0xFFFFFFFFu : 0u;
    m.pin[lane] = 0;
    m.hash[lane] = KEY_NONE;
    m.hash[lane + 32] = KEY_NONE;
    if (lane < 8) m.lmask[lane] = 0;
    if (lane < 16) m.lut1[lane] = NO_SLOT;
    reinterpret_cast<uint32_t*>(m.lut2)[lane] = 0xFFFFFFFFu;
    reinterpret_cast<uint32_t*>(m.lut2)[lane + 32] = 0xFFFFFFFFu;
#pragma unroll
    for (int i = lane; i < PREQ_SIZE; i += 32) {
        m.preq[i] = KEY_NONE;
        m.preq_lo[i] = 0x7FFFFFFF;
        m.preq_hi[i] = -1;
    }
    m.clo[lane] = 0x7FFF;
    m.chi[lane] = -1;
    for (int b = 0; b < 3; ++b) {
        m.rs[b].span_lo[lane] = 0x7FFFFFFF;
        m.rs[b].span_hi[lane] = -1;
    }
    if (lane < 3) {
        m.rs[lane].nreq = 0;
        m.rs[lane].used = 0;
        m.rs[lane].maxres = 0;
    }
    if (lane == 0) {
        m.ndeep = 0;
        m.nbuild = 0;
    }
    __syncwarp();
}

// Clear round buffer b (whole warp).
__device__ __forceinline__ void round_clear(Meta::Round& rb) {
    const int lane = threadIdx.x & 31;
    rb.span_lo[lane] = 0x7FFFFFFF;
    rb.span_hi[lane] = -1;
    if (lane == 0) {
        rb.nreq = 0;
        rb.used = 0;
        rb.maxres = 0;
    }
}

// Record a missing node for this round; duplicates collapse through a small
// hash of pending keys.  A request that finds the table full is simply not
// recorded (its outputs retry next round; the first request always fits).
__device__ __forceinline__ void request_node(Meta& m, Meta::Round& rb, uint32_t key, int lo, int hi) {
    uint32_t h = hash_of(key) & (PREQ_SIZE - 1);
    for (int i = 0; i < PREQ_SIZE; ++i) {
        const uint32_t prev = atomicCAS(&m.preq[h], KEY_NONE, key);
        if (prev == KEY_NONE || prev == key) {
            atomicMin(&m.preq_lo[h], lo);
            atomicMax(&m.preq_hi[h], hi);
            if (prev == KEY_NONE) {
                const uint32_t at = atomicAdd(&rb.nreq, 1u);
                if (at < REQ_MAX) {
                    m.req[at] = key;
                    m.req_h[at] = (uint8_t)h;
                }
            }
            return;
        }
        h = (h + 1) & (PREQ_SIZE - 1);
    }
}

// Do the records of slot s hold counts for the window columns [xl, xl+2r]?
__device__ __forceinline__ bool span_ok(const Meta& m, int s, int xl, int r) {
    return (int)m.clo[s] <= xl && xl + 2 * r <= (int)m.chi[s];
}

// Give slot v to node nk (one thread): the direct tables of levels 1 and 2
// are updated in O(1); returns whether a level >= 3 node left or entered
// (the hash of deep nodes then needs slot_tables_refresh).
__device__ __forceinline__ bool slot_set_key(Meta& m, int v, uint32_t nk) {
    const uint32_t ok = m.key[v];
    const int ol = ok == KEY_NONE ? 0 : (int)(ok >> 20), nl = nk == KEY_NONE ? 0 : (int)(nk >> 20);
    if (ol == 1) m.lut1[(ok >> 16) & 15] = NO_SLOT;
    if (ol == 2) m.lut2[(((ok >> 16) & 15) << 4) | (ok & 15)] = NO_SLOT;
    if (nl == 1) m.lut1[(nk >> 16) & 15] = (uint8_t)v;
    if (nl == 2) m.lut2[(((nk >> 16) & 15) << 4) | (nk & 15)] = (uint8_t)v;
    m.key[v] = nk;
    return ol >= 3 || nl >= 3;
}

// After a round's slot assignments (whole warp): level masks from all slot
// keys and, when deep nodes changed, the hash of deep nodes (lanes insert
// their own slot's key concurrently with linear probing).
__device__ __forceinline__ void slot_tables_refresh(Meta& m, int nslots, bool deep_changed) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const uint32_t k = (lane > 0 && lane < nslots) ? m.key[lane] : KEY_NONE;
    const int kl = k == KEY_NONE ? 0 : (int)(k >> 20);
    const uint32_t bit = k == KEY_NONE ? 0u : 1u << ((k >> 16) & 15);
    uint32_t any = 0;
#pragma unroll
    for (int l = 1; l < 5; ++l) {
        const uint32_t ml = __reduce_or_sync(0xffffffffu, kl == l ? bit : 0u);
        if (lane == 0) m.lmask[l] = ml;
        any |= ml;
    }
    const unsigned deep = __popc(__ballot_sync(0xffffffffu, kl >= 3));
    if (lane == 0) {
        m.lmask[0] = any;
        m.ndeep = deep;
    }
    if (deep_changed) {
        m.hash[lane] = KEY_NONE;
        m.hash[lane + 32] = KEY_NONE;
        __syncwarp();
        if (kl >= 3) {
            uint32_t h = hash_of(k);
            for (int i = 0; i < HASH_SIZE; ++i) {  // <= 31 keys in 64 entries: always finds room
                if (atomicCAS(&m.hash[h], KEY_NONE, (k << 8) | (uint32_t)lane) == KEY_NONE) break;
                h = (h + 1) & (HASH_SIZE - 1);
            }
        }
    }
    __syncwarp();
}

// Load the level table for one image into m (whole warp).
__device__ __forceinline__ void load_levels(Meta& m, const LevelDesc* desc, int fixed_shift) {
    const int lane = threadIdx.x & 31;
    int ushift;
    uint32_t ev = 0;
    if (desc == nullptr) {
        ushift = fixed_shift;
    } else if (desc->mode == 0) {
        ushift = max(0, bitlen(desc->vmax) - 4);
    } else {
        ushift = -1;
        if (lane < 17) ev = desc->edge[lane];
    }
    if (ushift >= 0) ev = (uint32_t)lane << ushift;
    if (lane < 17) m.e[lane] = ev;
    __syncwarp();
    if (lane < 16) {
        if (ushift >= 0) {
            m.D[lane] = (uint32_t)ushift;
        } else {
            uint32_t w = m.e[lane + 1] > m.e[lane] ? m.e[lane + 1] - m.e[lane] : 1u;
            m.D[lane] = (uint32_t)bitlen(w - 1);
        }
    }
    if (lane == 0) m.ushift = ushift;
    __syncwarp();
}

// ---- 16-bin counts as 8 packed uint16 pairs --------------------------------

// Add the 16 byte-counts held in q (bins 0..15) into the pair accumulator.
__device__ __forceinline__ void acc_add(uint32_t (&a)[8], const uint4& q) {
    a[0] += lo_pair(q.x); a[1] += hi_pair(q.x);
    a[2] += lo_pair(q.y); a[3] += hi_pair(q.y);
    a[4] += lo_pair(q.z); a[5] += hi_pair(q.z);
    a[6] += lo_pair(q.w); a[7] += hi_pair(q.w);
}

// get_order_statistic over one 16-child node (Section III): descend the
// implicit binary tree over the 16 window counts, going left when the left
// subtree holds at least K values, else subtracting its count and going right.
// Returns the child index; K becomes the rank within that child.
__device__ __forceinline__ int select16(const uint32_t (&w)[8], uint32_t& K) {
    uint32_t s = w[0] + w[1] + w[2] + w[3];
    uint32_t left = (s & 0xFFFFu) + (s >> 16);
    bool rt = K > left;
    K -= rt ? left : 0u;
    uint32_t a0 = rt ? w[4] : w[0], a1 = rt ? w[5] : w[1], a2 = rt ? w[6] : w[2], a3 = rt ? w[7] : w[3];
    int b = rt ? 8 : 0;
    s = a0 + a1;
    left = (s & 0xFFFFu) + (s >> 16);
    rt = K > left;
    K -= rt ? left : 0u;
    uint32_t c0 = rt ? a2 : a0, c1 = rt ? a3 : a1;
    b += rt ? 4 : 0;
    left = (c0 & 0xFFFFu) + (c0 >> 16);
    rt = K > left;
    K -= rt ? left : 0u;
    uint32_t d = rt ? c1 : c0;
    b += rt ? 2 : 0;
    left = d & 0xFFFFu;
    rt = K > left;
    K -= rt ? left : 0u;
    b += rt ? 1 : 0;
    return b;
}

// Byte counter update inside a 16-byte column record: bin b += delta (+1/-1).
__device__ __forceinline__ void bump(uint32_t* rec, int b, int delta) {
    uint32_t inc = 1u << (8 * (b & 3));
    if (delta > 0) rec[b >> 2] += inc;
    else rec[b >> 2] -= inc;
}

// Add bin b into four packed byte counters held in registers.
__device__ __forceinline__ void reg_bump(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, int b) {
    uint32_t inc = 1u << (8 * (b & 3));
    int w = b >> 2;
    c0 += w == 0 ? inc : 0u;
    c1 += w == 1 ? inc : 0u;
    c2 += w == 2 ? inc : 0u;
    c3 += w == 3 ? inc : 0u;
}

}  // namespace hrm

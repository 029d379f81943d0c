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
// mode (Section III-C): e_c are data-driven (equal-mass quantiles of the mixed
// frequency model).  Below each coarse interval the tree is uniform, with
// D_c = bitlen(width_c - 1) bits taken 4 bits (16 children) per level.
struct LevelDesc {
    uint32_t mode;      // 0 = uniform, 1 = adaptive
    uint32_t vmin;      // observed minimum (filled by the pre-pass)
    uint32_t vmax;      // observed maximum
    uint32_t count;     // pixels seen
    uint32_t edge[17];  // adaptive coarse edges, edge[16] = vmax + 1
    uint32_t pad[11];
};
static_assert(sizeof(LevelDesc) == 128, "LevelDesc layout");

constexpr uint32_t KEY_NONE = 0xFFFFFFFFu;
constexpr int HASH_SIZE = 64;
constexpr int MAX_SLOTS = 32;
constexpr int META_BYTES = 1024;  // per-warp metadata block (see Meta)

// Per-warp metadata in shared memory.
struct Meta {
    uint32_t e[17];        // coarse edges
    uint32_t D[16];        // sub-tree bits per coarse interval
    uint32_t key[MAX_SLOTS];
    uint32_t stamp[MAX_SLOTS];
    uint32_t pin[MAX_SLOTS];
    uint32_t hash[HASH_SIZE];
    uint32_t lmask[8];     // lmask[l] bit c: a slot at level l for coarse c exists; lmask[0] = OR of all
    int32_t ushift;        // >= 0: uniform shift; -1: adaptive
    uint32_t pad[3];
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

__device__ __forceinline__ int slot_lookup(const Meta& m, uint32_t key) {
    uint32_t h = hash_of(key);
#pragma unroll 1
    for (int i = 0; i < HASH_SIZE; ++i) {
        uint32_t ent = m.hash[h];
        if (ent == KEY_NONE) return -1;
        if ((ent >> 8) == key) return (int)(ent & 0xFFu);
        h = (h + 1) & (HASH_SIZE - 1);
    }
    return -1;
}

// Rebuild the hash table and level masks from m.key[] (whole warp).
__device__ __forceinline__ void rehash(Meta& m, int nslots) {
    const int lane = threadIdx.x & 31;
    m.hash[lane] = KEY_NONE;
    m.hash[lane + 32] = KEY_NONE;
    __syncwarp();
    if (lane == 0) {
        uint32_t lm[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int s = 1; s < nslots; ++s) {
            uint32_t k = m.key[s];
            if (k == KEY_NONE) continue;
            int l = (int)(k >> 20), c = (int)((k >> 16) & 15);
            lm[l] |= 1u << c;
            lm[0] |= 1u << c;
            uint32_t h = hash_of(k);
            while (m.hash[h] != KEY_NONE) h = (h + 1) & (HASH_SIZE - 1);
            m.hash[h] = (k << 8) | (uint32_t)s;
        }
        for (int l = 0; l < 8; ++l) m.lmask[l] = lm[l];
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

// hist_tile.cuh -- hierarchical recursive running median: one thread block,
// one tile.
//
// A tile is a row of TW = 32*W*PPL outputs along x that a block of W warps
// walks along the "walk axis" (y for 2D images, z for 3D volumes): Section
// III, column IOTs slid along the walk axis, the window IOT assembled across
// x.  Every thread owns PPL outputs of each row and about 1/(32W) of the
// columns; the phases of a row are separated by block barriers.
//
// Per block, in shared memory:
//   * "column" histograms for the TW + 2r columns the tile's windows touch.
//     In 2D a column is the n pixels of image column x inside the window's
//     rows; in 3D it is the n x n slab of voxels (rows y-r..y+r, slices
//     z-r..z+r) at x, and the window is the sum of n such slabs -- the same
//     recursion one dimension up (Section III, N-dimensional extension).
//   * The 16-interval top level (the root node) is always resident; deeper
//     nodes live in a small LRU cache of "slots".  A slot holds, for every
//     column, the 16 child counts of one tree node (8-bit counters when a
//     column holds <= 255 values, 16-bit otherwise).
//   * Advancing one step along the walk axis removes the leaving layer and
//     inserts the entering layer of every column into every resident node on
//     the value's path (Section III-B, add_value / remove_value: one +-1 per
//     level).  A layer is one pixel in 2D and n voxels in 3D.
//   * The window counts of a node are the sums of its column counts over the n
//     columns of each output's window (Section III: window IOT = sum of
//     column IOTs).  They are formed on demand, only for nodes the walk visits
//     (Section III, on-demand window update).  When many outputs share a node,
//     one prefix sum over the tile's columns serves all of them (the parallel
//     form of the window recursion "+entering column -leaving column"); when
//     few do, each output sums its n columns directly.
//   * get_order_statistic (Section III): at each level the window counts of
//     the 16 children of the current node are searched by a binary descent for
//     the child holding rank K; K drops by the counts to its left and the walk
//     continues in that child.  The leaf reached is exactly the K-th smallest
//     value of the window.
//   * A node needed for the first time (the paper's non-elementary update) is
//     built from the staged input values of every column.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "hist_common.cuh"

namespace hrm {

constexpr int BLOCK_WARPS = 4;     // warps per tile
constexpr int BLOCK_THREADS = 32 * BLOCK_WARPS;
// Extra columns on each side of a requested node span, so that medians
// drifting sideways by a few columns per row do not widen it every row.
constexpr int SPAN_MARGIN = 16;

struct HistJob {
    const unsigned char* src;
    unsigned char* dst;
    size_t s_row, s_slice;   // source pitches (bytes)
    size_t d_row, d_slice;   // destination pitches (bytes)
    int W, H, D;             // D = 1 for 2D
    int dims;                // 2 or 3
    int r;
    int sh;                  // strip length along the walk axis (interior strips)
    int she, ne;             // edge strips: ne strips of she steps at each end of the walk axis
    int nint;                // interior strips (2D tile order, see hist_tile)
    int tiles_x;             // tiles across x
    int ntiles;
    uint32_t K;              // 1-based target rank
    int nslots;              // slots per warp including the root
    const LevelDesc* desc;   // nullptr: uniform with fixed_shift
    int fixed_shift;
    int drop_bits;           // reduced precision: stop once <= drop_bits bits remain (0 = exact)
    int elem;                // 1 or 2 bytes per value
    int ppl;                 // outputs per thread (TW = 32 * BLOCK_WARPS * ppl)
    int cw;                  // counter width in bytes (1 or 2)
    int ring;                // 2D only: stage the last n+1 input rows in shared memory
    unsigned* err;           // device error word (may be null)
    unsigned* stats;         // null, or a counter that receives the tiles' node installs
};

// Ring of the last n+1 input rows (2D): (n+1) rows x NC columns, padded to 16 bytes.
__host__ __device__ inline size_t hist_ring_bytes(int tw, int r, int elem) {
    size_t b = (size_t)(2 * r + 2) * (size_t)(tw + 2 * r) * elem;
    return (b + 15) & ~(size_t)15;
}

__host__ __device__ inline size_t hist_smem_bytes(int tw, int r, int nslots, int cw, int ring = 0, int elem = 2) {
    int nc = tw + 2 * r;
    return (size_t)META_BYTES + (size_t)(nc + 1) * 32 + (size_t)nslots * nc * 16 * cw +
           (ring ? hist_ring_bytes(tw, r, elem) : 0);
}

// ---- counter records (16 bins, CW bytes per bin) ---------------------------------

template <int CW>
__device__ __forceinline__ void rec_add(uint32_t (&a)[8], const unsigned char* rec) {
    if (CW == 1) {
        acc_add(a, *reinterpret_cast<const uint4*>(rec));
    } else {
        const uint4 q0 = reinterpret_cast<const uint4*>(rec)[0];
        const uint4 q1 = reinterpret_cast<const uint4*>(rec)[1];
        a[0] += q0.x; a[1] += q0.y; a[2] += q0.z; a[3] += q0.w;
        a[4] += q1.x; a[5] += q1.y; a[6] += q1.z; a[7] += q1.w;
    }
}

template <int CW>
__device__ __forceinline__ void rec_bump(unsigned char* rec, int b, int delta) {
    uint32_t* w = reinterpret_cast<uint32_t*>(rec);
    if (CW == 1) {
        const uint32_t inc = 1u << (8 * (b & 3));
        if (delta > 0) w[b >> 2] += inc; else w[b >> 2] -= inc;
    } else {
        const uint32_t inc = 1u << (16 * (b & 1));
        if (delta > 0) w[b >> 1] += inc; else w[b >> 1] -= inc;
    }
}

// Register counters used while building a record: 8 words (CW = 2) or the first 4 (CW = 1).
template <int CW>
__device__ __forceinline__ void reg_count(uint32_t (&c)[8], int b) {
    if (CW == 1) {
        const uint32_t inc = 1u << (8 * (b & 3));
        const int w = b >> 2;
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] += w == k ? inc : 0u;
    } else {
        const uint32_t inc = 1u << (16 * (b & 1));
        const int w = b >> 1;
#pragma unroll
        for (int k = 0; k < 8; ++k) c[k] += w == k ? inc : 0u;
    }
}

template <int CW>
__device__ __forceinline__ void rec_store(unsigned char* rec, const uint32_t (&c)[8]) {
    uint4* q = reinterpret_cast<uint4*>(rec);
    q[0] = make_uint4(c[0], c[1], c[2], c[3]);
    if (CW == 2) q[1] = make_uint4(c[4], c[5], c[6], c[7]);
}

// ---- geometry -----------------------------------------------------------------

struct Geo {
    const unsigned char* src;
    size_t tstride, istride;  // bytes per walk step / per layer index
    int tmax, imax;           // clamp limits (walk axis, layer axis)
    int ibase;                // first layer coordinate before clamping
    int layer;                // values per column per walk step (1 in 2D, n in 3D)
};

template <typename T>
__device__ __forceinline__ uint32_t geo_ld(const Geo& g, int t, int i, int gx) {
    const int tc = clampi(t, 0, g.tmax);
    const int ic = clampi(g.ibase + i, 0, g.imax);
    return (uint32_t)__ldg(reinterpret_cast<const T*>(g.src + (size_t)tc * g.tstride + (size_t)ic * g.istride) + gx);
}

__device__ __forceinline__ int ring_idx(int u, int M) { return (u + M) % M; }

// Node geometry: value range [lo, hi) of node `key` and the shift that turns
// (v - lo) into its child index (level 0: the coarse interval).
struct NodeRange {
    int level;
    uint32_t lo, hi;
    uint32_t width;  // hi - lo (levels > 0)
    int dshift;
};

__device__ __forceinline__ NodeRange node_range(const Meta& m, uint32_t key) {
    NodeRange nr;
    nr.level = (int)(key >> 20);
    nr.lo = 0;
    nr.hi = 0xFFFFFFFFu;
    nr.dshift = 0;
    if (nr.level > 0) {
        const int c = (int)((key >> 16) & 15);
        const uint32_t pre = key & 0xFFFFu;
        const int top = (int)m.D[c] - 4 * (nr.level - 1);
        const int b = min(4, top);
        nr.lo = m.e[c] + (pre << top);
        nr.hi = min(nr.lo + (1u << top), m.e[c + 1]);
        nr.dshift = top - b;
    }
    nr.width = nr.hi - nr.lo;
    return nr;
}

// Build the records of the m.nbuild build entries (slot, column range) at walk
// position t (whole block).  Work items are (entry, aligned column pair):
// both columns of a pair share the value loads (one 32-bit shared-memory load
// from the ring in 2D, else one row address per walk step) and the index
// arithmetic, and give two independent counting chains.  A pair may reach
// one column outside the entry's range; that column gets its correct current
// counts too, which is harmless (NC is even, so pairs stay inside the tile).
// The per-value work is a clamp and a multiply-add at most (no division):
// installs near the image corners, where medians move to new nodes every
// row, are dominated by this loop.
template <typename T, int CW, int DIMS>
__device__ void build_slots(const HistJob& a, const Geo& g, const Meta& m, unsigned char* slots, int NC,
                            int x0, int t, const T* ring) {
    const int r = a.r;
    const int n = 2 * r + 1;
    const int nb = (int)m.nbuild;
    const int items = (int)m.build_off[nb];
    int b = 0;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        while (b + 1 < nb && (int)m.build_off[b + 1] <= it) ++b;  // items ascend per thread
        const int c0 = 2 * (((int)m.build_lo[b] >> 1) + (it - (int)m.build_off[b]));
        const NodeRange nr = node_range(m, m.build_key[b]);
        uint32_t cnt0[8] = {0, 0, 0, 0, 0, 0, 0, 0}, cnt1[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        // Below the root a value belongs to the node iff (v - lo) < width
        // (unsigned).  Nodes deep in a wide distribution hold few of a
        // column's values, so the counting sits behind one test per pair.
        auto count2 = [&](uint32_t v0, uint32_t v1) {
            if (nr.level == 0) {
                reg_count<CW>(cnt0, coarse_of(m, v0));
                reg_count<CW>(cnt1, coarse_of(m, v1));
                return;
            }
            const uint32_t e0 = v0 - nr.lo, e1 = v1 - nr.lo;
            const bool in0 = e0 < nr.width, in1 = e1 < nr.width;
            if (__builtin_expect(in0 || in1, 0)) {
                if (in0) reg_count<CW>(cnt0, (int)(e0 >> nr.dshift));
                if (in1) reg_count<CW>(cnt1, (int)(e1 >> nr.dshift));
            }
        };
        if (ring) {
            const int M = 2 * r + 2;
            int idx = ring_idx(t - r, M);
            const T* col = ring + c0;
#pragma unroll 4
            for (int k = 0; k < n; ++k) {
                if (sizeof(T) == 2) {
                    const uint32_t w = *reinterpret_cast<const uint32_t*>(col + (size_t)idx * NC);
                    count2(w & 0xFFFFu, w >> 16);
                } else {
                    const uint32_t w = *reinterpret_cast<const unsigned short*>(col + (size_t)idx * NC);
                    count2(w & 0xFFu, w >> 8);
                }
                idx = idx + 1 == M ? 0 : idx + 1;
            }
        } else {
            const int gx0 = clampi(x0 - r + c0, 0, a.W - 1), gx1 = clampi(x0 - r + c0 + 1, 0, a.W - 1);
            if (DIMS == 2) {  // one value per walk step
                for (int k0 = 0; k0 < n; k0 += 8) {
                    uint32_t v0[8], v1[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int tc = clampi(t - r + min(k0 + u, n - 1), 0, g.tmax);
                        const T* rp = reinterpret_cast<const T*>(g.src + (size_t)tc * g.tstride);
                        v0[u] = __ldg(rp + gx0);
                        v1[u] = __ldg(rp + gx1);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (k0 + u >= n) break;
                        count2(v0[u], v1[u]);
                    }
                }
            } else {  // 3D: a slab of `layer` rows per walk step
                for (int k = 0; k < n; ++k) {
                    const unsigned char* sl = g.src + (size_t)clampi(t - r + k, 0, g.tmax) * g.tstride;
                    for (int i0 = 0; i0 < g.layer; i0 += 4) {  // 8 loads in flight
                        uint32_t v0[4], v1[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int ic = clampi(g.ibase + min(i0 + u, g.layer - 1), 0, g.imax);
                            const T* rp = reinterpret_cast<const T*>(sl + (size_t)ic * g.istride);
                            v0[u] = __ldg(rp + gx0);
                            v1[u] = __ldg(rp + gx1);
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (i0 + u >= g.layer) break;
                            count2(v0[u], v1[u]);
                        }
                    }
                }
            }
        }
        unsigned char* rec = slots + ((size_t)m.build_slot[b] * NC + c0) * 16 * CW;
        rec_store<CW>(rec, cnt0);
        rec_store<CW>(rec + 16 * CW, cnt1);
    }
}

// Packed counter deltas of one record: word w of bin b gets +-(1 << lane_shift).
// Adding the accumulated delta to the record in one step is exact whenever the
// final counts are in range (the arithmetic is modulo 2^32 per word).
template <int CW>
__device__ __forceinline__ void delta_add(uint32_t (&dw)[4 * CW], int b, int sign) {
    constexpr int NW = 4 * CW;  // words per record
    constexpr int per = 4 / CW; // counters per word
    const uint32_t inc = 1u << ((32 / per) * (b % per));
    const int w = b / per;
#pragma unroll
    for (int k = 0; k < NW; ++k) dw[k] += w == k ? (sign > 0 ? inc : 0u - inc) : 0u;
}

// Insert (+1) or remove (-1) value v of column cx in every resident node below
// the root on its path (Section III-B: one counter per level).
template <int CW>
__device__ __forceinline__ void deep_update(const Meta& m, unsigned char* slots, int NC, int cx, uint32_t v,
                                            int c, int delta) {
    if (!((m.lmask[0] >> c) & 1u)) return;
    const uint32_t u = v - m.e[c];
    const int D = (int)m.D[c];
    for (int level = 1; 4 * (level - 1) < D; ++level) {
        if (!((m.lmask[level] >> c) & 1u)) continue;
        const int top = D - 4 * (level - 1);
        const int s = slot_lookup(m, level, c, u >> top);
        if (s < 0) continue;
        const int b = min(4, top);
        const int d = (int)((u >> (top - b)) & ((1u << b) - 1u));
        rec_bump<CW>(slots + ((size_t)s * NC + cx) * 16 * CW, d, delta);
    }
}

// 2D, 8-bit counters: remove vo and insert vi of column cx in the resident
// nodes below the root (Section III-B: one +-1 per level), with the level
// masks held in registers.  Levels 1 and 2 (direct slot tables) are handled
// together: both values' slot lookups are issued at once, then each touched
// counter word is bumped.  Deeper levels (16-bit data) take the generic path.
struct LevelMasks {
    uint32_t l0, l1, l2;
    bool deep;  // some resident node lies at level >= 3
};

__device__ __forceinline__ void pair_update(const Meta& m, const LevelMasks& lm, unsigned char* slots, int NC,
                                            int cx, uint32_t vo, int co, uint32_t vi, int ci) {
    const bool ao = (lm.l0 >> co) & 1u, ai = (lm.l0 >> ci) & 1u;
    if (!ao && !ai) return;
    int s1o = -1, s1i = -1, s2o = -1, s2i = -1, d1o = 0, d1i = 0, d2o = 0, d2i = 0;
    int Do = 0, Di = 0;
    uint32_t uo = 0, ui = 0;
    if (ao) {
        uo = vo - m.e[co];
        Do = (int)m.D[co];
        const int b1 = min(4, Do);
        d1o = (int)((uo >> (Do - b1)) & ((1u << b1) - 1u));
        if ((lm.l1 >> co) & 1u) s1o = m.lut1[co];
        if (Do > 4 && ((lm.l2 >> co) & 1u)) {
            const int b2 = min(4, Do - 4);
            d2o = (int)((uo >> (Do - 4 - b2)) & ((1u << b2) - 1u));
            s2o = m.lut2[(co << 4) | (int)((uo >> (Do - 4)) & 15u)];
        }
    }
    if (ai) {
        ui = vi - m.e[ci];
        Di = (int)m.D[ci];
        const int b1 = min(4, Di);
        d1i = (int)((ui >> (Di - b1)) & ((1u << b1) - 1u));
        if ((lm.l1 >> ci) & 1u) s1i = m.lut1[ci];
        if (Di > 4 && ((lm.l2 >> ci) & 1u)) {
            const int b2 = min(4, Di - 4);
            d2i = (int)((ui >> (Di - 4 - b2)) & ((1u << b2) - 1u));
            s2i = m.lut2[(ci << 4) | (int)((ui >> (Di - 4)) & 15u)];
        }
    }
    // one 32-bit counter word per (value, level): load, add, store; the two
    // values' words at one level may coincide (same node), so each update is
    // a separate read-modify-write in program order
    auto bump = [&](int sl, int d, int delta) {
        uint32_t* w = reinterpret_cast<uint32_t*>(slots + ((size_t)sl * NC + cx) * 16) + (d >> 2);
        const uint32_t inc = 1u << (8 * (d & 3));
        *w = delta > 0 ? *w + inc : *w - inc;
    };
    if (s1o != NO_SLOT && s1o >= 0) bump(s1o, d1o, -1);
    if (s1i != NO_SLOT && s1i >= 0) bump(s1i, d1i, +1);
    if (s2o != NO_SLOT && s2o >= 0) bump(s2o, d2o, -1);
    if (s2i != NO_SLOT && s2i >= 0) bump(s2i, d2i, +1);
    if (lm.deep) {  // levels >= 3 through the hash of deep nodes
        for (int q = 0; q < 2; ++q) {
            const bool act = q ? ai : ao;
            const int c = q ? ci : co, D = q ? Di : Do;
            const uint32_t u = q ? ui : uo;
            if (!act) continue;
            for (int level = 3; 4 * (level - 1) < D; ++level) {
                if (!((m.lmask[level] >> c) & 1u)) continue;
                const int top = D - 4 * (level - 1);
                const int sl = slot_lookup(m, level, c, u >> top);
                if (sl < 0) continue;
                const int b = min(4, top);
                const int d = (int)((u >> (top - b)) & ((1u << b) - 1u));
                rec_bump<1>(slots + ((size_t)sl * NC + cx) * 16, d, q ? +1 : -1);
            }
        }
    }
}

// Block-wide inclusive prefix over columns [lo, hi] of slot s into
// pfx[1 .. hi-lo+1] (pfx[0] = 0).  The scratch holds two planes of
// (NC+1) uint4 each -- words 0..3 then words 4..7 of every column -- so that
// consecutive lanes touch consecutive 16-byte granules (no bank conflicts).
// Each thread scans an odd-length chunk of
// columns (odd so that a quarter-warp's 16-byte records fall in distinct
// bank groups), then chunk totals are scanned across lanes and warps.
template <int CW>
__device__ void block_prefix(Meta& m, const unsigned char* slots, uint4* pfx, int NC, int s, int lo, int hi) {
    const int plane = NC + 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt = blockDim.x;
    const int mcols = hi - lo + 1;
    // odd chunk length: consecutive threads start on different banks; warps
    // whose threads hold no columns skip the scan
    const int q = ((mcols + nt - 1) / nt) | 1;
    const int c_begin = lo + tid * q;
    const int c_end = min(c_begin + q, hi + 1);
    uint32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const unsigned char* base = slots + (size_t)s * NC * 16 * CW;
    for (int c0 = c_begin; c0 < c_end; c0 += 4) {
        uint4 rec[4][CW];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int cx = min(c0 + u, c_end - 1);
#pragma unroll
            for (int h = 0; h < CW; ++h) rec[u][h] = reinterpret_cast<const uint4*>(base + (size_t)cx * 16 * CW)[h];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (c0 + u >= c_end) break;
            if (CW == 1) {
                acc_add(acc, rec[u][0]);
            } else {
                acc[0] += rec[u][0].x; acc[1] += rec[u][0].y; acc[2] += rec[u][0].z; acc[3] += rec[u][0].w;
                acc[4] += rec[u][CW - 1].x; acc[5] += rec[u][CW - 1].y; acc[6] += rec[u][CW - 1].z; acc[7] += rec[u][CW - 1].w;
            }
            const int e = c0 + u - lo + 1;
            pfx[e] = make_uint4(acc[0], acc[1], acc[2], acc[3]);
            pfx[plane + e] = make_uint4(acc[4], acc[5], acc[6], acc[7]);
        }
    }
    uint32_t inc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) inc[k] = acc[k];
    if (lo + (tid - lane) * q <= hi) {  // this warp holds columns (uniform per warp)
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t tv = __shfl_up_sync(0xffffffffu, inc[k], off);
                if (lane >= off) inc[k] += tv;
            }
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int k = 0; k < 8; ++k) m.wtot[warp][k] = inc[k];
    }
    __syncthreads();
    uint32_t carry[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) carry[k] = inc[k] - acc[k];
    for (int w = 0; w < warp; ++w)
#pragma unroll
        for (int k = 0; k < 8; ++k) carry[k] += m.wtot[w][k];
    for (int cx = c_begin; cx < c_end; ++cx) {
        const int e = cx - lo + 1;
        uint4 u0 = pfx[e], u1 = pfx[plane + e];
        u0.x += carry[0]; u0.y += carry[1]; u0.z += carry[2]; u0.w += carry[3];
        u1.x += carry[4]; u1.y += carry[5]; u1.z += carry[6]; u1.w += carry[7];
        pfx[e] = u0;
        pfx[plane + e] = u1;
    }
    if (tid == 0) {
        pfx[0] = make_uint4(0, 0, 0, 0);
        pfx[plane] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
}

// Record, for the round buffer, which slots this warp's resolved outputs use
// and the column span of those outputs.  Lanes of a warp nearly always share
// one or two slots, so the bookkeeping is reduced within the warp first and
// each distinct slot costs one shared-memory atomic per warp (same-address
// atomics from all lanes would serialise).
template <int PPL>
__device__ __forceinline__ void note_used(Meta::Round& rb, const int (&slot)[PPL], const bool (&res)[PPL],
                                          int tid, int nt) {
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < PPL; ++k)
        if (res[k]) mine |= 1u << slot[k];
    uint32_t wused = __reduce_or_sync(0xffffffffu, mine);
    if (wused && (threadIdx.x & 31) == 0) atomicOr(&rb.used, wused);
    while (wused) {
        const int s = __ffs(wused) - 1;
        wused &= wused - 1;
        unsigned lo = 0x7FFFFFFFu, hi = 0;
#pragma unroll
        for (int k = 0; k < PPL; ++k)
            if (res[k] && slot[k] == s) {
                lo = min(lo, (unsigned)(tid + nt * k));
                hi = max(hi, (unsigned)(tid + nt * k) + 1u);
            }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&rb.span_lo[s], (int)lo);
            atomicMax(&rb.span_hi[s], (int)hi - 1);
        }
    }
}

// GRP: the kernel instance for small windows (at least 8 column records per
// packed-byte group in the direct window sums, see below); other instances
// keep the plain loop, which the compiler schedules better for them.
template <typename T, int PPL, int CW, int DIMS, bool GRP = false>
__device__ void hist_tile(const HistJob& a, int tile, unsigned char* sm) {
    constexpr int NT = BLOCK_THREADS;
    constexpr int TW = NT * PPL;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = a.r;
    const int n = 2 * r + 1;
    const int NC = TW + 2 * r;
    const int S = a.nslots;
    // Tile order (low ids start first).  2D with two or more tile columns:
    // the edge strips' first and last tile columns one row per tile (at the
    // image corners nearly every output's median needs its own tree node, so
    // a corner row costs tens of interior rows: single-row tiles spread them
    // over many blocks instead of making one 8-row tile the longest of the
    // launch), then the other edge-strip tiles, then the interior strips'
    // first and last tile columns -- their windows are clamped in x, so they
    // run slower -- then the other interior tiles.  3D: x fastest, then the row, then the
    // strip.
    int tx, yrow = 0, strip, sub = -1;
    if (DIMS == 2 && a.tiles_x >= 2) {
        // the two corner tile columns of the edge strips: one tile per row
        const int nC = 2 * (2 * a.ne * a.she);
        const int nE = 2 * a.ne * (a.tiles_x - 2);
        if (tile < nC) {
            tx = (tile & 1) ? a.tiles_x - 1 : 0;
            const int q = tile >> 1;
            strip = q / a.she;
            sub = q % a.she;
        } else if (tile < nC + nE) {
            const int k = tile - nC;
            strip = k / (a.tiles_x - 2);
            tx = 1 + k % (a.tiles_x - 2);
        } else {
            int k = tile - nC - nE;
            if (k < 2 * a.nint) {
                tx = (k & 1) ? a.tiles_x - 1 : 0;
                strip = 2 * a.ne + (k >> 1);
            } else {
                k -= 2 * a.nint;
                strip = 2 * a.ne + k / (a.tiles_x - 2);
                tx = 1 + k % (a.tiles_x - 2);
            }
        }
    } else {
        tx = tile % a.tiles_x;
        const int rest = tile / a.tiles_x;
        strip = rest;
        if (DIMS == 3) {
            yrow = rest % a.H;
            strip = rest / a.H;
        }
    }
    const int L = DIMS == 3 ? a.D : a.H;  // walk-axis length
    // Steps within r of either end of the walk axis see clamped windows whose
    // medians are much noisier (more tree nodes per row; near the image
    // corners several times the work of an interior step).  They come first
    // (low tile ids start first) in short edge strips, alternating ends;
    // the interior follows in strips of sh steps.
    const int x0 = tx * TW;
    int ts, te;
    if (strip < 2 * a.ne) {
        const int k = strip >> 1;
        if ((strip & 1) == 0) {
            ts = k * a.she;
            te = ts + a.she;
        } else {
            te = L - k * a.she;
            ts = te - a.she;
        }
        if (sub >= 0) {  // a single row of a corner tile column
            ts += sub;
            te = ts + 1;
        }
    } else {
        const int lo = a.ne * a.she;
        ts = lo + (strip - 2 * a.ne) * a.sh;
        te = min(ts + a.sh, L - lo);
    }
    if (ts >= L || ts >= te || x0 >= a.W) return;  // uniform across the block

    Geo g;
    g.src = a.src;
    if (DIMS == 3) {
        g.tstride = a.s_slice;
        g.istride = a.s_row;
        g.tmax = a.D - 1;
        g.imax = a.H - 1;
        g.ibase = yrow - r;
        g.layer = n;
    } else {
        g.tstride = a.s_row;
        g.istride = 0;
        g.tmax = a.H - 1;
        g.imax = 0;
        g.ibase = 0;
        g.layer = 1;
    }
    unsigned char* drow0 = a.dst + (DIMS == 3 ? (size_t)yrow * a.d_row : 0);
    const size_t dstep = DIMS == 3 ? a.d_slice : a.d_row;

    Meta& m = *reinterpret_cast<Meta*>(sm);
    uint4* pfx = reinterpret_cast<uint4*>(sm + META_BYTES);
    unsigned char* slots = sm + META_BYTES + (size_t)(NC + 1) * 32;
    const bool use_ring = a.ring && DIMS == 2 && CW == 1;
    T* ring = use_ring ? reinterpret_cast<T*>(slots + (size_t)S * NC * 16 * CW) : nullptr;
    const int M = 2 * r + 2;  // ring rows
    // the thread's columns cx = tid + NT*j, j < CPL, cover NC <= TW + 2*127
    constexpr int CPL = PPL + 2;

    OpCounters oc;
    oc.reset();
    const unsigned long long ns_tile0 = oc.now_ns();
    const long long t_tile0 = clock64();
    oc.mark();
    if (warp == 0) {
        load_levels(m, a.desc, a.fixed_shift);
        slots_reset(m);
        if (lane == 0) m.ninst = 0;
    }
    if (use_ring) {  // stage input rows ts-r-1 .. ts+r
        for (int u = ts - r - 1; u <= ts + r; ++u) {
            const T* row = reinterpret_cast<const T*>(a.src + (size_t)clampi(u, 0, L - 1) * a.s_row);
            T* dst = ring + (size_t)ring_idx(u, M) * NC;
            for (int cx = tid; cx < NC; cx += NT) dst[cx] = __ldg(row + clampi(x0 - r + cx, 0, a.W - 1));
        }
    }
    __syncthreads();
    if (tid == 0) {
        m.nbuild = 1;
        m.build_slot[0] = 0;
        m.build_key[0] = 0;
        m.build_lo[0] = 0;
        m.build_hi[0] = (int16_t)(NC - 1);
        m.build_off[0] = 0;
        m.build_off[1] = NC / 2;  // in column pairs
        m.clo[0] = 0;
        m.chi[0] = (int16_t)(NC - 1);
    }
    __syncthreads();
    build_slots<T, CW, DIMS>(a, g, m, slots, NC, x0, ts, ring);
    __syncthreads();
    if (tid == 0) m.nbuild = 0;

    // 2D: the entering (and, without the ring, the leaving) values of the next
    // step are loaded one step ahead, so their latency hides behind the walk.
    uint32_t nin[CPL], nout[CPL];
    auto prefetch = [&](int tn) {
        if (DIMS != 2 || tn >= te) return;
        const int ti = clampi(tn + r, 0, L - 1), to = clampi(tn - r - 1, 0, L - 1);
        const T* rin = reinterpret_cast<const T*>(a.src + (size_t)ti * a.s_row);
        const T* rout = reinterpret_cast<const T*>(a.src + (size_t)to * a.s_row);
#pragma unroll
        for (int j = 0; j < CPL; ++j) {
            const int cx = tid + NT * j;
            if (cx < NC) {
                const int gx = clampi(x0 - r + cx, 0, a.W - 1);
                nin[j] = __ldg(rin + gx);
                if (!use_ring) nout[j] = __ldg(rout + gx);
            }
        }
    };
    prefetch(ts + 1);
    oc.lap(CNT_CYC_INIT);

    // cost model (per block): one shared prefix of a node vs direct n-column sums
    const int prefix_cost = ((NC + NT - 1) / NT) * (CW == 1 ? 31 : 24) + 700;  // incl. two barriers
    const int vpc = DIMS == 3 ? n * n : n;  // values per column record
    const int grp = max(1, 255 / vpc);        // records summed as packed bytes per expansion
    const int direct_cost = n * (CW == 1 ? 24 : 14);
    uint32_t pass_id = 0;

    for (int t = ts; t < te; ++t) {
        const uint32_t stampv = (uint32_t)(t - ts + 1);
        if (t > ts) {
            const int to = clampi(t - r - 1, 0, L - 1);
            const int ti = clampi(t + r, 0, L - 1);
            if (DIMS == 2 && CW == 1) {
                T* rin = use_ring ? ring + (size_t)ring_idx(t + r, M) * NC : nullptr;
                const T* rout = use_ring ? ring + (size_t)ring_idx(t - r - 1, M) * NC : nullptr;
                // root level: each of the thread's column records is read,
                // changed by the leaving and entering values, and written back;
                // all loads are issued before any store
                LevelMasks lm;
                lm.l0 = m.lmask[0];
                lm.l1 = m.lmask[1];
                lm.l2 = m.lmask[2];
                lm.deep = m.ndeep != 0;
                uint32_t vo[CPL], vi[CPL];
                uint4 rec[CPL];
#pragma unroll
                for (int j = 0; j < CPL; ++j) {
                    const int cx = tid + NT * j;
                    if (cx < NC) {
                        vi[j] = nin[j];
                        vo[j] = use_ring ? (uint32_t)rout[cx] : nout[j];
                        rec[j] = reinterpret_cast<const uint4*>(slots)[cx];
                    }
                }
#pragma unroll
                for (int j = 0; j < CPL; ++j) {
                    const int cx = tid + NT * j;
                    if (cx < NC) {
                        if (use_ring) rin[cx] = (T)vi[j];
                        uint32_t dw[4] = {0, 0, 0, 0};
                        const int co = coarse_of(m, vo[j]), ci = coarse_of(m, vi[j]);
                        delta_add<1>(dw, co, -1);
                        delta_add<1>(dw, ci, +1);
                        rec[j].x += dw[0]; rec[j].y += dw[1]; rec[j].z += dw[2]; rec[j].w += dw[3];
                        reinterpret_cast<uint4*>(slots)[cx] = rec[j];
                        if (vo[j] != vi[j]) pair_update(m, lm, slots, NC, cx, vo[j], co, vi[j], ci);
                    }
                }
            } else if (to != ti) {
                // n leaving and n entering values per column (3D slab); the
                // root deltas are accumulated in registers and applied once
                for (int cx = tid; cx < NC; cx += NT) {
                    const int gx = clampi(x0 - r + cx, 0, a.W - 1);
                    uint32_t dw[4 * CW];
#pragma unroll
                    for (int k = 0; k < 4 * CW; ++k) dw[k] = 0;
                    for (int i = 0; i < g.layer; i += 4) {
                        uint32_t vo[4], vi[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int ii = min(i + k, g.layer - 1);
                            vo[k] = geo_ld<T>(g, to, ii, gx);
                            vi[k] = geo_ld<T>(g, ti, ii, gx);
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            if (i + k < g.layer && vo[k] != vi[k]) {
                                const int co = coarse_of(m, vo[k]), ci = coarse_of(m, vi[k]);
                                delta_add<CW>(dw, co, -1);
                                delta_add<CW>(dw, ci, +1);
                                deep_update<CW>(m, slots, NC, cx, vo[k], co, -1);
                                deep_update<CW>(m, slots, NC, cx, vi[k], ci, +1);
                            }
                    }
                    uint32_t* rw = reinterpret_cast<uint32_t*>(slots + (size_t)cx * 16 * CW);
#pragma unroll
                    for (int k = 0; k < 4 * CW; ++k) rw[k] += dw[k];
                }
            }
            prefetch(t + 1);
            __syncthreads();
        }
        oc.lap(CNT_CYC_COLUMNS);
        oc.add(CNT_ROWS, 1);

        // ---- level walk for the TW outputs at walk position t ----
        uint32_t K[PPL], pre[PPL], val[PPL];
        int cbin[PPL], slot[PPL], dig[PPL];
        bool pend[PPL], todo[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            K[k] = a.K;
            pre[k] = 0;
            val[k] = 0;
            cbin[k] = 0;
            pend[k] = x0 + tid + NT * k < a.W;
        }
        // level 0: the root (slot 0) serves every output of the row, so it
        // needs no lookup; one prefix over the row's columns
        {
            const int hi0 = min(TW, a.W - x0) - 1;
            block_prefix<CW>(m, slots, pfx, NC, 0, 0, hi0 + 2 * r);
            oc.add(CNT_ROUNDS, 1);
            oc.add(CNT_PREFIXES, 1);
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                if (!pend[k]) continue;
                const int xl = tid + NT * k;
                const uint4 a0 = pfx[xl], a1 = pfx[NC + 1 + xl], b0 = pfx[xl + n], b1 = pfx[NC + 1 + xl + n];
                uint32_t w[8] = {b0.x - a0.x, b0.y - a0.y, b0.z - a0.z, b0.w - a0.w,
                                 b1.x - a1.x, b1.y - a1.y, b1.z - a1.z, b1.w - a1.w};
                const int c = select16(w, K[k]);
                cbin[k] = c;
                if ((int)m.D[c] <= a.drop_bits) {
                    val[k] = m.e[c];
                    pend[k] = false;
                }
            }
            oc.add(CNT_LEVELS, 1);
        }
        oc.lap(CNT_CYC_WINDOW);

        // One round: pin the resident nodes of the outputs still to do, record
        // which slots they use and over which columns, request the missing
        // ones; the last warp clears the round buffer after next.
        int nres = 0;
        auto resolve = [&](int level, Meta::Round& rb) {
            nres = 0;
            bool hit[PPL];
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                slot[k] = -1;
                hit[k] = false;
                if (todo[k]) {
                    const int xl = tid + NT * k;
                    int s = slot_lookup(m, level, cbin[k], pre[k]);
                    if (s >= 0 && !span_ok(m, s, xl, r)) s = -1;  // resident, but not over this window
                    slot[k] = s;
                    if (s >= 0) {
                        m.pin[s] = pass_id;
                        hit[k] = true;
                        ++nres;
                    } else {
                        request_node(m, rb, node_key(level, cbin[k], pre[k]), max(xl - SPAN_MARGIN, 0),
                                     min(xl + 2 * r + SPAN_MARGIN, NC - 1));
                    }
                }
            }
            note_used<PPL>(rb, slot, hit, tid, NT);
            if (warp == BLOCK_WARPS - 1) round_clear(m.rs[(pass_id + 1) % 3]);
        };
        bool anyp = false;
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            todo[k] = pend[k];
            anyp |= pend[k];
        }
        // the first round of level 1 is resolved before the barrier that
        // closes level 0 (its prefix scratch is free once that barrier passes)
        ++pass_id;
        resolve(1, m.rs[pass_id % 3]);
        bool more = __syncthreads_or(anyp);
        oc.lap(CNT_CYC_RESOLVE);
        for (int level = 1; more && level < 6; ++level) {
            for (int guard = 0;; ++guard) {
                if (guard > 0) {  // a previous round of this level left outputs unresolved
                    bool anyt = false;
#pragma unroll
                    for (int k = 0; k < PPL; ++k) anyt |= todo[k];
                    if (!__syncthreads_or(anyt)) break;
                    if (guard > TW + 1) {  // cannot happen: every round settles >= 1 node
                        if (tid == 0) set_error(a.err, DEV_SLOT_OVERFLOW);
                        break;
                    }
                    ++pass_id;
                    resolve(level, m.rs[pass_id % 3]);
                    __syncthreads();
                    oc.lap(CNT_CYC_RESOLVE);
                }
                Meta::Round& rb = m.rs[pass_id % 3];
                oc.add(CNT_ROUNDS, 1);
                const uint32_t nreq = rb.nreq;
                if (nreq) {
                    // warp 0 gives unpinned slots (least recently used first)
                    // to the requested nodes; the block builds them
                    if (warp == 0) {
                        // A request for a resident node (its span was too
                        // narrow) widens that slot in place: only the new
                        // columns are built.  Otherwise the least recently
                        // used unpinned slot is taken and built over the span.
                        const uint32_t nr = min(nreq, (uint32_t)REQ_MAX);
                        uint32_t nb = 0, off = 0;
                        bool deep_changed = false;
                        for (uint32_t i = 0; i < nr && nb + 2 <= (uint32_t)MAX_SLOTS; ++i) {
                            const uint32_t key = m.req[i];
                            const int h = m.req_h[i];
                            int lo = m.preq_lo[h], hi = m.preq_hi[h];
                            int slot_w = slot_lookup(m, key);
                            // (the deep-node hash is refreshed after the loop: a slot
                            // reassigned earlier in this loop may still be listed)
                            if (slot_w >= 0 && m.key[slot_w] != key) slot_w = -1;
                            int part_lo[2] = {lo, 0}, part_hi[2] = {hi, -1};
                            if (slot_w >= 0) {
                                const int olo = m.clo[slot_w], ohi = m.chi[slot_w];
                                // the union must stay contiguous: build from the new
                                // edge up to the old span on each side (gaps included)
                                part_lo[0] = lo;
                                part_hi[0] = olo - 1;
                                part_lo[1] = ohi + 1;
                                part_hi[1] = hi;
                                lo = min(lo, olo);
                                hi = max(hi, ohi);
                            } else {
                                uint32_t cand = 0xFFFFFFFFu;
                                if (lane > 0 && lane < S && m.pin[lane] != pass_id)
                                    cand = (m.stamp[lane] << 5) | (uint32_t)lane;
                                cand = __reduce_min_sync(0xffffffffu, cand);
                                if (cand == 0xFFFFFFFFu) break;  // every slot is in use this round
                                slot_w = (int)(cand & 31u);
                                if (lane == 0) deep_changed |= slot_set_key(m, slot_w, key);
                            }
                            if (lane == 0) {
                                m.pin[slot_w] = pass_id;
                                m.stamp[slot_w] = stampv;
                                m.clo[slot_w] = (int16_t)lo;
                                m.chi[slot_w] = (int16_t)hi;
                                for (int q = 0; q < 2; ++q) {
                                    if (part_hi[q] < part_lo[q]) continue;
                                    m.build_slot[nb] = (uint32_t)slot_w;
                                    m.build_key[nb] = key;
                                    m.build_lo[nb] = (int16_t)part_lo[q];
                                    m.build_hi[nb] = (int16_t)part_hi[q];
                                    m.build_off[nb] = off;
                                    off += (uint32_t)((part_hi[q] >> 1) - (part_lo[q] >> 1) + 1);
                                    ++nb;
                                }
                            }
                            nb = __shfl_sync(0xffffffffu, nb, 0);
                            off = __shfl_sync(0xffffffffu, off, 0);
                            __syncwarp();
                        }
                        slot_tables_refresh(m, S, __shfl_sync(0xffffffffu, (int)deep_changed, 0) != 0);
                        for (int i = lane; i < PREQ_SIZE; i += 32) {
                            m.preq[i] = KEY_NONE;
                            m.preq_lo[i] = 0x7FFFFFFF;
                            m.preq_hi[i] = -1;
                        }
                        if (lane == 0) {
                            m.nbuild = nb;
                            m.ninst += nb;
                            m.build_off[nb] = off;
                        }
                    }
                    __syncthreads();
                    oc.lap(CNT_CYC_ALLOC);
                    build_slots<T, CW, DIMS>(a, g, m, slots, NC, x0, t, ring);
                    oc.add(CNT_INSTALLS, m.nbuild);
                    bool got[PPL];
#pragma unroll
                    for (int k = 0; k < PPL; ++k) {
                        got[k] = false;
                        if (todo[k] && slot[k] < 0) {
                            const int s2 = slot_lookup(m, level, cbin[k], pre[k]);
                            if (s2 >= 0 && m.pin[s2] == pass_id && span_ok(m, s2, tid + NT * k, r)) {
                                slot[k] = s2;
                                got[k] = true;
                                ++nres;
                            }
                        }
                    }
                    note_used<PPL>(rb, slot, got, tid, NT);
                    __syncthreads();  // new records built, all spans recorded
                }
                if (PPL > 1) {
                    const unsigned wmax = __reduce_max_sync(0xffffffffu, (unsigned)nres);
                    if (wmax && lane == 0) atomicMax(&rb.maxres, wmax);
                }
                oc.lap(CNT_CYC_INSTALL);
                // window counts of the resolved outputs, then one descent step
                bool res[PPL];
#pragma unroll
                for (int k = 0; k < PPL; ++k) res[k] = todo[k] && slot[k] >= 0;
                const uint32_t used = rb.used;
                const int groups = __popc(used);
                // With one output per thread every thread with a resolved output
                // has exactly one, so the decision needs no barrier; otherwise
                // maxres is complete only after one (the prefix path needs none).
                bool direct = false;
                if (PPL == 1) {
                    direct = groups > 0 && direct_cost < groups * prefix_cost;
                } else if (n * (CW == 1 ? 24 : 14) < groups * prefix_cost) {
                    __syncthreads();
                    direct = (int)rb.maxres * direct_cost < groups * prefix_cost;
                }
                oc.add(direct ? CNT_DIRECT_ROUNDS : CNT_PREFIXES, direct ? 1 : groups);
                if (direct) {
#pragma unroll
                    for (int k = 0; k < PPL; ++k) {
                        if (!res[k]) continue;
                        const int xl = tid + NT * k;
                        const unsigned char* base = slots + (size_t)slot[k] * NC * 16 * CW;
                        uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                        if (GRP && CW == 1 && grp >= 8) {
                            // 8-bit counters: a column holds vpc values, so up to 255 / vpc
                            // records add as packed bytes without overflow; expand once per
                            // group (small windows: at least 8 records per group)
                            for (int cx = xl; cx < xl + n;) {
                                const int ce = min(cx + grp, xl + n);
                                uint4 b = make_uint4(0, 0, 0, 0);
                                for (; cx < ce; ++cx) {
                                    const uint4 q = *reinterpret_cast<const uint4*>(base + (size_t)cx * 16);
                                    b.x += q.x; b.y += q.y; b.z += q.z; b.w += q.w;
                                }
                                acc_add(w, b);
                            }
                        } else {
                            for (int cx = xl; cx < xl + n; ++cx) rec_add<CW>(w, base + (size_t)cx * 16 * CW);
                        }
                        dig[k] = select16(w, K[k]);
                    }
                } else {
                    uint32_t rem = used;
                    while (rem) {
                        const int s = __ffs(rem) - 1;
                        rem &= rem - 1;
                        const int lo = rb.span_lo[s], hi = rb.span_hi[s];
                        block_prefix<CW>(m, slots, pfx, NC, s, lo, hi + 2 * r);
#pragma unroll
                        for (int k = 0; k < PPL; ++k) {
                            if (!(res[k] && slot[k] == s)) continue;
                            const int xl = tid + NT * k;
                            const int ea = xl - lo, eb = xl - lo + n;
                            const uint4 a0 = pfx[ea], a1 = pfx[NC + 1 + ea], b0 = pfx[eb], b1 = pfx[NC + 1 + eb];
                            uint32_t w[8] = {b0.x - a0.x, b0.y - a0.y, b0.z - a0.z, b0.w - a0.w,
                                             b1.x - a1.x, b1.y - a1.y, b1.z - a1.z, b1.w - a1.w};
                            dig[k] = select16(w, K[k]);
                        }
                        if (rem) __syncthreads();  // the scratch is reused by the next node
                    }
                }
#pragma unroll
                for (int k = 0; k < PPL; ++k)
                    if (res[k]) {
                        m.stamp[slot[k]] = stampv;
                        todo[k] = false;
                    }
                oc.lap(CNT_CYC_WINDOW);
                if (!nreq) break;  // nothing was missing: every output of this level is settled
                __syncthreads();   // end of a round with installs: the next round may rebuild slots
            }
            oc.add(CNT_LEVELS, 1);
            // advance every output one level down its path
            anyp = false;
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                if (!pend[k]) continue;
                const int Dc = (int)m.D[cbin[k]];
                const int top = Dc - 4 * (level - 1);
                const int b = min(4, top);
                pre[k] = (pre[k] << b) | (uint32_t)dig[k];
                const int left = top - b;
                if (left <= a.drop_bits) {
                    val[k] = m.e[cbin[k]] + (pre[k] << left);
                    pend[k] = false;
                }
                todo[k] = pend[k];
                anyp |= pend[k];
            }
            oc.lap(CNT_CYC_ADVANCE);
            // the next level's first round is resolved before the barrier that
            // closes this level (every thread is then done with the scratch)
            ++pass_id;
            resolve(level + 1, m.rs[pass_id % 3]);
            more = __syncthreads_or(anyp);
            oc.lap(CNT_CYC_RESOLVE);
        }
        // ---- store the outputs of walk position t ----
        T* drow = reinterpret_cast<T*>(drow0 + (size_t)t * dstep);
        const uint32_t mask = a.drop_bits > 0 ? ~((1u << a.drop_bits) - 1u) : 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int x = x0 + tid + NT * k;
            if (x < a.W) drow[x] = (T)(val[k] & mask);
        }
        oc.lap(CNT_CYC_ADVANCE);
    }
    oc.add(CNT_TILES, 1);
    oc.add(CNT_CYC_TOTAL, (unsigned long long)(clock64() - t_tile0));
    if (tid == 0) {
        oc.flush(tile);
        oc.tile(tile, ns_tile0);
        if (a.stats) atomicAdd(a.stats, m.ninst);  // thread 0 is the only writer of m.ninst
    }
}

}  // namespace hrm

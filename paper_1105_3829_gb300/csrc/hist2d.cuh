// hist2d.cuh -- hierarchical recursive running median, 2D tile body.
//
// One warp filters one tile: TW = 32*PPL output columns of a strip of rows,
// walking down the strip (Section III, "column IOTs" slid vertically and the
// window assembled from them horizontally).
//
// Per warp, in shared memory:
//   * column histograms ("column IOTs") for the TW + 2r columns the tile's
//     windows touch, at the 16-interval top level (the root node, always
//     resident) and for a small LRU cache of deeper nodes ("slots").  A slot
//     holds, for every column, the 16 child counts of one tree node.  Counts
//     are bytes (a column holds n <= 255 values).
//   * Moving down one row removes the leaving pixel and inserts the entering
//     pixel of every column into every resident node on its path (Section
//     III-B, add_value / remove_value: one +-1 per level).
//   * The window counts of a node are sums of its column counts over the n
//     columns of each output's window (Section III: window IOT =
//     sum of column IOTs).  They are formed on demand, only for the nodes the
//     walk actually visits (Section III, on-demand update).  When many outputs
//     share a node, one prefix sum over the tile's columns serves all of them
//     (the parallel form of the window recursion "+entering column -leaving
//     column"); for small windows each output sums its n columns directly.
//   * get_order_statistic (Section III) descends level by level: the window
//     counts of the 16 children of the current node are searched with a
//     binary descent for the child holding rank K, K is reduced by the counts
//     to its left, and the walk continues in that child.  The value reached at
//     the leaves is exactly the K-th smallest value of the window.
//   * A node needed for the first time (a non-elementary update in the
//     paper's terms) is built from the n staged input rows of every column.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "hist_common.cuh"

namespace hrm {

struct Hist2DJob {
    const unsigned char* src;
    size_t sp;
    unsigned char* dst;
    size_t dp;
    int W, H, r;
    int sh;          // strip height (rows per tile)
    int tiles_x;     // tiles per row of tiles
    int ntiles;
    uint32_t K;      // 1-based target rank
    int nslots;      // slots per warp including the root
    const LevelDesc* desc;  // nullptr: uniform with fixed_shift
    int fixed_shift;
    int drop_bits;   // reduced precision: stop once <= drop_bits bits remain (0 = exact)
    int elem;        // 1 or 2 (batch kernel dispatch)
    int ppl;         // pixels per lane (batch kernel dispatch)
    unsigned* err;   // device error word (may be null)
};

__host__ __device__ inline size_t hist2d_smem_bytes(int tw, int r, int nslots) {
    int nc = tw + 2 * r;
    return (size_t)META_BYTES + (size_t)(nc + 1) * 32 + (size_t)nslots * nc * 16;
}

template <typename T>
__device__ __forceinline__ uint32_t ld2(const Hist2DJob& a, int y, int gx) {
    return (uint32_t)__ldg(reinterpret_cast<const T*>(a.src + (size_t)y * a.sp) + gx);
}

// Build slot s for node `key` at output row y from the n input rows of every column.
template <typename T>
__device__ void build_slot2d(const Hist2DJob& a, const Meta& m, unsigned char* slots, int NC,
                             int x0, int y, int s, uint32_t key) {
    const int lane = threadIdx.x & 31;
    const int r = a.r;
    const int level = (int)(key >> 20);
    const int c = (int)((key >> 16) & 15);
    const uint32_t pre = key & 0xFFFFu;
    uint32_t lo = 0, hi = 0xFFFFFFFFu;
    int dshift = 0;
    if (level > 0) {
        int top = (int)m.D[c] - 4 * (level - 1);
        int b = min(4, top);
        lo = m.e[c] + (pre << top);
        hi = min(lo + (1u << top), m.e[c + 1]);
        dshift = top - b;
    }
    for (int cx = lane; cx < NC; cx += 32) {
        const int gx = clampi(x0 - r + cx, 0, a.W - 1);
        uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#pragma unroll 4
        for (int yy = y - r; yy <= y + r; ++yy) {
            uint32_t v = ld2<T>(a, clampi(yy, 0, a.H - 1), gx);
            int d;
            if (level == 0) {
                d = coarse_of(m, v);
            } else {
                if (v < lo || v >= hi) continue;
                d = (int)((v - lo) >> dshift);
            }
            reg_bump(c0, c1, c2, c3, d);
        }
        *reinterpret_cast<uint4*>(slots + ((size_t)s * NC + cx) * 16) = make_uint4(c0, c1, c2, c3);
    }
}

// Insert (delta = +1) or remove (-1) value v of column cx in every resident node on its path.
__device__ __forceinline__ void column_update(const Meta& m, unsigned char* slots, int NC, int cx,
                                              uint32_t v, int delta) {
    const int c = coarse_of(m, v);
    bump(reinterpret_cast<uint32_t*>(slots + (size_t)cx * 16), c, delta);
    if (!((m.lmask[0] >> c) & 1u)) return;
    const uint32_t u = v - m.e[c];
    const int D = (int)m.D[c];
    for (int level = 1; 4 * (level - 1) < D; ++level) {
        if (!((m.lmask[level] >> c) & 1u)) continue;
        const int top = D - 4 * (level - 1);
        const int s = slot_lookup(m, node_key(level, c, u >> top));
        if (s < 0) continue;
        const int b = min(4, top);
        const int d = (int)((u >> (top - b)) & ((1u << b) - 1u));
        bump(reinterpret_cast<uint32_t*>(slots + ((size_t)s * NC + cx) * 16), d, delta);
    }
}

// Inclusive prefix over columns [lo, hi] of slot s into pfx[1 .. m], pfx[0] = 0.
__device__ __forceinline__ void slot_prefix(const unsigned char* slots, uint4* pfx, int NC, int s,
                                            int lo, int hi) {
    const int lane = threadIdx.x & 31;
    const int mcols = hi - lo + 1;
    const int q = (mcols + 31) >> 5;
    const int c_begin = lo + lane * q;
    const int c_end = min(c_begin + q, hi + 1);
    uint32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const uint4* col = reinterpret_cast<const uint4*>(slots) + (size_t)s * NC;
    for (int cx = c_begin; cx < c_end; ++cx) {
        acc_add(acc, col[cx]);
        uint4* p = pfx + 2 * (cx - lo + 1);
        p[0] = make_uint4(acc[0], acc[1], acc[2], acc[3]);
        p[1] = make_uint4(acc[4], acc[5], acc[6], acc[7]);
    }
    // exclusive scan of the chunk totals across lanes
    uint32_t inc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) inc[k] = acc[k];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            uint32_t t = __shfl_up_sync(0xffffffffu, inc[k], off);
            if (lane >= off) inc[k] += t;
        }
    }
    uint32_t carry[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) carry[k] = inc[k] - acc[k];
    for (int cx = c_begin; cx < c_end; ++cx) {
        uint4* p = pfx + 2 * (cx - lo + 1);
        uint4 u0 = p[0], u1 = p[1];
        u0.x += carry[0]; u0.y += carry[1]; u0.z += carry[2]; u0.w += carry[3];
        u1.x += carry[4]; u1.y += carry[5]; u1.z += carry[6]; u1.w += carry[7];
        p[0] = u0;
        p[1] = u1;
    }
    if (lane == 0) {
        pfx[0] = make_uint4(0, 0, 0, 0);
        pfx[1] = make_uint4(0, 0, 0, 0);
    }
    __syncwarp();
}

template <typename T, int PPL>
__device__ void hist2d_tile(const Hist2DJob& a, int tile, unsigned char* sm) {
    constexpr int TW = 32 * PPL;
    const int lane = threadIdx.x & 31;
    const int r = a.r;
    const int n = 2 * r + 1;
    const int NC = TW + 2 * r;
    const int S = a.nslots;
    const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int x0 = tx * TW;
    const int ys = ty * a.sh;
    const int ye = min(ys + a.sh, a.H);
    if (ys >= a.H || x0 >= a.W) return;

    Meta& m = *reinterpret_cast<Meta*>(sm);
    uint4* pfx = reinterpret_cast<uint4*>(sm + META_BYTES);
    unsigned char* slots = sm + META_BYTES + (size_t)(NC + 1) * 32;

    load_levels(m, a.desc, a.fixed_shift);
    if (lane < MAX_SLOTS) {
        m.key[lane] = lane == 0 ? 0u : KEY_NONE;
        m.stamp[lane] = lane == 0 ? 0xFFFFFFFFu : 0u;
        m.pin[lane] = 0;
    }
    __syncwarp();
    rehash(m, S);
    build_slot2d<T>(a, m, slots, NC, x0, ys, 0, 0u);
    __syncwarp();

    // direct vs shared-prefix cost model (warp instructions, see header comment)
    const int prefix_cost = ((NC + 31) >> 5) * 31 + 120;
    uint32_t pass_id = 0;

    for (int y = ys; y < ye; ++y) {
        const uint32_t rowstamp = (uint32_t)(y - ys + 1);
        if (y > ys) {
            const int yo = clampi(y - r - 1, 0, a.H - 1);
            const int yi = clampi(y + r, 0, a.H - 1);
            if (yo != yi) {
                for (int cx = lane; cx < NC; cx += 32) {
                    const int gx = clampi(x0 - r + cx, 0, a.W - 1);
                    const uint32_t vo = ld2<T>(a, yo, gx);
                    const uint32_t vi = ld2<T>(a, yi, gx);
                    if (vo != vi) {
                        column_update(m, slots, NC, cx, vo, -1);
                        column_update(m, slots, NC, cx, vi, +1);
                    }
                }
            }
            __syncwarp();
        }

        // ---- level walk for the TW outputs of row y ----
        uint32_t K[PPL], pre[PPL], val[PPL];
        int cbin[PPL];
        bool pend[PPL];
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            K[k] = a.K;
            pre[k] = 0;
            val[k] = 0;
            cbin[k] = 0;
            pend[k] = x0 + lane + 32 * k < a.W;
        }
        for (int level = 0; level < 6; ++level) {
            bool anyp = false;
#pragma unroll
            for (int k = 0; k < PPL; ++k) anyp |= pend[k];
            if (!__any_sync(0xffffffffu, anyp)) break;

            uint32_t key[PPL];
            int slot[PPL], dig[PPL];
            bool todo[PPL];
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                key[k] = level == 0 ? 0u : node_key(level, cbin[k], pre[k]);
                todo[k] = pend[k];
                dig[k] = 0;
            }
            for (int guard = 0;; ++guard) {
                bool anyt = false;
#pragma unroll
                for (int k = 0; k < PPL; ++k) anyt |= todo[k];
                if (!__any_sync(0xffffffffu, anyt)) break;
                if (guard > 32 * PPL + 1) {  // cannot happen: every round settles >= 1 node
                    if (lane == 0) set_error(a.err, DEV_SLOT_OVERFLOW);
                    break;
                }
                ++pass_id;
                // 1) resident nodes
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    slot[k] = -1;
                    if (todo[k]) {
                        slot[k] = level == 0 ? 0 : slot_lookup(m, key[k]);
                        if (slot[k] > 0) m.pin[slot[k]] = pass_id;
                    }
                }
                __syncwarp();
                // 2) install missing nodes while unpinned slots remain
                for (;;) {
                    int mk = -1;
#pragma unroll
                    for (int k = PPL - 1; k >= 0; --k)
                        if (todo[k] && slot[k] < 0) mk = k;
                    const unsigned miss = __ballot_sync(0xffffffffu, mk >= 0);
                    if (!miss) break;
                    const int leader = __ffs(miss) - 1;
                    uint32_t mykey = 0;
#pragma unroll
                    for (int k = 0; k < PPL; ++k)
                        if (k == mk) mykey = key[k];
                    const uint32_t nk = __shfl_sync(0xffffffffu, mykey, leader);
                    uint32_t cand = 0xFFFFFFFFu;
                    if (lane > 0 && lane < S && m.pin[lane] != pass_id)
                        cand = (m.stamp[lane] << 5) | (uint32_t)lane;
                    cand = __reduce_min_sync(0xffffffffu, cand);
                    if (cand == 0xFFFFFFFFu) break;  // every slot is in use this round
                    const int victim = (int)(cand & 31u);
                    __syncwarp();
                    if (lane == 0) {
                        m.key[victim] = nk;
                        m.pin[victim] = pass_id;
                        m.stamp[victim] = rowstamp;
                    }
                    __syncwarp();
                    rehash(m, S);
                    build_slot2d<T>(a, m, slots, NC, x0, y, victim, nk);
#pragma unroll
                    for (int k = 0; k < PPL; ++k)
                        if (todo[k] && slot[k] < 0 && key[k] == nk) slot[k] = victim;
                    __syncwarp();
                }
                // 3) window counts of the resolved outputs, then one descent step
                bool res[PPL];
                uint32_t used = 0;
                int nres = 0;
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    res[k] = todo[k] && slot[k] >= 0;
                    if (res[k]) {
                        used |= 1u << slot[k];
                        ++nres;
                    }
                }
                used = __reduce_or_sync(0xffffffffu, used);
                const int maxres = (int)__reduce_max_sync(0xffffffffu, (unsigned)nres);
                const int groups = __popc(used);
                const bool direct = level > 0 && maxres * n * 17 < groups * prefix_cost;
                if (direct) {
#pragma unroll
                    for (int k = 0; k < PPL; ++k) {
                        if (!res[k]) continue;
                        const int xl = lane + 32 * k;
                        const uint4* col = reinterpret_cast<const uint4*>(slots) + (size_t)slot[k] * NC;
                        uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                        for (int cx = xl; cx < xl + n; ++cx) acc_add(w, col[cx]);
                        dig[k] = select16(w, K[k]);
                    }
                } else {
                    uint32_t rem = used;
                    while (rem) {
                        const int s = __ffs(rem) - 1;
                        rem &= rem - 1;
                        int lo = 1 << 30, hi = -1;
#pragma unroll
                        for (int k = 0; k < PPL; ++k)
                            if (res[k] && slot[k] == s) {
                                lo = min(lo, lane + 32 * k);
                                hi = max(hi, lane + 32 * k);
                            }
                        lo = (int)__reduce_min_sync(0xffffffffu, (unsigned)lo);
                        hi = (int)__reduce_max_sync(0xffffffffu, (unsigned)(hi + 1)) - 1;
                        slot_prefix(slots, pfx, NC, s, lo, hi + 2 * r);
#pragma unroll
                        for (int k = 0; k < PPL; ++k) {
                            if (!(res[k] && slot[k] == s)) continue;
                            const int xl = lane + 32 * k;
                            const uint4* pa = pfx + 2 * (xl - lo);
                            const uint4* pb = pfx + 2 * (xl - lo + n);
                            uint4 a0 = pa[0], a1 = pa[1], b0 = pb[0], b1 = pb[1];
                            uint32_t w[8] = {b0.x - a0.x, b0.y - a0.y, b0.z - a0.z, b0.w - a0.w,
                                             b1.x - a1.x, b1.y - a1.y, b1.z - a1.z, b1.w - a1.w};
                            dig[k] = select16(w, K[k]);
                        }
                        __syncwarp();
                    }
                }
#pragma unroll
                for (int k = 0; k < PPL; ++k)
                    if (res[k]) {
                        if (slot[k] > 0) m.stamp[slot[k]] = rowstamp;
                        todo[k] = false;
                    }
                __syncwarp();
            }
            // advance every output one level down its path
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                if (!pend[k]) continue;
                if (level == 0) {
                    cbin[k] = dig[k];
                    const int D = (int)m.D[dig[k]];
                    if (D <= a.drop_bits) {
                        val[k] = m.e[dig[k]];
                        pend[k] = false;
                    }
                } else {
                    const int D = (int)m.D[cbin[k]];
                    const int top = D - 4 * (level - 1);
                    const int b = min(4, top);
                    pre[k] = (pre[k] << b) | (uint32_t)dig[k];
                    const int left = top - b;
                    if (left <= a.drop_bits) {
                        val[k] = m.e[cbin[k]] + (pre[k] << left);
                        pend[k] = false;
                    }
                }
            }
        }
        // ---- store row y ----
        T* drow = reinterpret_cast<T*>(a.dst + (size_t)y * a.dp);
        const uint32_t mask = a.drop_bits > 0 ? ~((1u << a.drop_bits) - 1u) : 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int x = x0 + lane + 32 * k;
            if (x < a.W) drow[x] = (T)(val[k] & mask);
        }
    }
}

}  // namespace hrm

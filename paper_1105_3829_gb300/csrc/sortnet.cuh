// sortnet.cuh -- exact median for radius 1 and 2 (3x3, 5x5) by register
// selection networks.
//
// For windows this small the paper itself notes that direct selection is
// competitive (Section IV: Quickselect loses to the tree method only for
// windows larger than 4x4).  On the GPU the direct form is a fixed network of
// min/max operations in registers:
//   * every lane owns 8 consecutive columns and slides down a run of rows;
//   * each column's vertical n-tuple is sorted once and shared by the n
//     horizontally neighbouring outputs (neighbour lanes exchange their edge
//     columns with warp shuffles);
//   * two adjacent columns travel together as a packed uint16 pair, so every
//     min/max (native min.u16x2 / max.u16x2) serves two outputs.
// r = 1: median of 9 from three sorted columns is
//        med3(max of the lows, med3 of the middles, min of the highs).
// r = 2: the 5x5 block with sorted columns is row-sorted, 12 of its entries
//        are provably off-median, and the 7th smallest of the remaining 13 is
//        the median; the networks are Batcher odd-even merge sorts generated
//        at compile time and pruned to the outputs actually used.
// r = 3..5: the same pruning for the general k x k block (k = 2r+1), with
//        one column pair per lane and the neighbouring columns fetched by
//        shuffles one rank-row at a time (register footprint ~ the
//        candidate count: 29, 47, 73 for k = 7, 9, 11); the candidates of
//        each rank-row form a sorted run, and the runs are merged pairwise
//        down to the selected position.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "hrm_common.cuh"

namespace hrm {

// ---------------------------------------------------------------------------
// Compile-time Batcher odd-even merge sort comparator lists for n <= 128
// (generated for the next power of two; comparators touching an index >= n
// are dropped, which is the same as padding with +infinity).
struct Net {
    int n = 0;
    unsigned char a[1536] = {};
    unsigned char b[1536] = {};
};

constexpr Net make_net(int N) {
    Net net{};
    int P = 1;
    while (P < N) P <<= 1;
    for (int p = 1; p < P; p <<= 1)
        for (int k = p; k >= 1; k >>= 1)
            for (int j = k % p; j + k < P; j += 2 * k)
                for (int i = 0; i < k; ++i)
                    if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) {
                        int lo = i + j, hi = i + j + k;
                        if (hi < N) {
                            net.a[net.n] = (unsigned char)lo;
                            net.b[net.n] = (unsigned char)hi;
                            ++net.n;
                        }
                    }
    return net;
}

template <int N>
struct NetOf {
    static constexpr Net net = make_net(N);
};

// Sort v[0..N) ascending (per 16-bit half) with the Batcher network.
template <int N>
__device__ __forceinline__ void sortnet(uint32_t (&v)[N]) {
    constexpr Net net = NetOf<N>::net;
#pragma unroll
    for (int c = 0; c < net.n; ++c) {
        const int i = net.a[c], j = net.b[c];
        uint32_t lo = vmin2(v[i], v[j]);
        uint32_t hi = vmax2(v[i], v[j]);
        v[i] = lo;
        v[j] = hi;
    }
}

// ---------------------------------------------------------------------------
// Row loads: 8 consecutive columns starting at x as 4 packed uint16 pairs.
template <typename T>
__device__ __forceinline__ void load8(const unsigned char* src, size_t sp, int W, int y, int x,
                                      uint32_t (&p)[4]) {
    const unsigned char* row = src + (size_t)y * sp;
    if (x + 7 < W) {
        const T* ptr = reinterpret_cast<const T*>(row) + x;
        if (sizeof(T) == 2 && (reinterpret_cast<uintptr_t>(ptr) & 15) == 0) {
            uint4 q = __ldg(reinterpret_cast<const uint4*>(ptr));
            p[0] = q.x; p[1] = q.y; p[2] = q.z; p[3] = q.w;
            return;
        }
        if (sizeof(T) == 1 && (reinterpret_cast<uintptr_t>(ptr) & 7) == 0) {
            uint2 q = __ldg(reinterpret_cast<const uint2*>(ptr));
            p[0] = lo_pair(q.x); p[1] = hi_pair(q.x);
            p[2] = lo_pair(q.y); p[3] = hi_pair(q.y);
            return;
        }
    }
    const T* r = reinterpret_cast<const T*>(row);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t a = __ldg(r + min(x + 2 * k, W - 1));
        uint32_t b = __ldg(r + min(x + 2 * k + 1, W - 1));
        p[k] = a | (b << 16);
    }
}

template <typename T>
__device__ __forceinline__ uint32_t load1(const unsigned char* src, size_t sp, int W, int y, int x) {
    x = clampi(x, 0, W - 1);
    return (uint32_t)__ldg(reinterpret_cast<const T*>(src + (size_t)y * sp) + x);
}

template <typename T>
__device__ __forceinline__ void store8(unsigned char* dst, size_t dp, int W, int y, int x,
                                       const uint32_t (&o)[4]) {
    unsigned char* row = dst + (size_t)y * dp;
    if (x + 7 < W) {
        T* ptr = reinterpret_cast<T*>(row) + x;
        if (sizeof(T) == 2 && (reinterpret_cast<uintptr_t>(ptr) & 15) == 0) {
            *reinterpret_cast<uint4*>(ptr) = make_uint4(o[0], o[1], o[2], o[3]);
            return;
        }
        if (sizeof(T) == 1 && (reinterpret_cast<uintptr_t>(ptr) & 7) == 0) {
            *reinterpret_cast<uint2*>(ptr) =
                make_uint2(__byte_perm(o[0], o[1], 0x6420), __byte_perm(o[2], o[3], 0x6420));
            return;
        }
    }
    T* r = reinterpret_cast<T*>(row);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (x + 2 * k < W) r[x + 2 * k] = (T)(o[k] & 0xFFFFu);
        if (x + 2 * k + 1 < W) r[x + 2 * k + 1] = (T)(o[k] >> 16);
    }
}

// (hi half of a, lo half of b): the pair shifted by one column.
__device__ __forceinline__ uint32_t shift1(uint32_t a, uint32_t b) { return __byte_perm(a, b, 0x5432); }

__device__ __forceinline__ uint32_t med3(uint32_t a, uint32_t b, uint32_t c) {
    return vmax2(vmin2(a, b), vmin2(vmax2(a, b), c));
}

// ---------------------------------------------------------------------------
// r = 1
// One warp: 256 columns starting at tile_x*256, rows [tile_y*rpw, +rpw).
template <typename T>
__device__ void sortnet3x3_tile(const unsigned char* __restrict__ src, size_t sp,
                                unsigned char* __restrict__ dst, size_t dp, int W, int H,
                                int rows_per_warp, int tile_x, int tile_y) {
    const int lane = threadIdx.x & 31;
    const int x = tile_x * 256 + lane * 8;
    const int y0 = tile_y * rows_per_warp;
    if (y0 >= H || tile_x * 256 >= W) return;
    const int y1 = min(y0 + rows_per_warp, H);

    uint32_t a[4], b[4], c[4];
    uint32_t ea, eb, ec;  // halo column (lane 0: x-1, lane 31: x+8), duplicated in both halves
    const int hx = lane == 0 ? x - 1 : x + 8;
    load8<T>(src, sp, W, clampi(y0 - 1, 0, H - 1), x, a);
    load8<T>(src, sp, W, y0, x, b);
    ea = load1<T>(src, sp, W, clampi(y0 - 1, 0, H - 1), hx) * 0x10001u;
    eb = load1<T>(src, sp, W, y0, hx) * 0x10001u;
    for (int y = y0; y < y1; ++y) {
        const int yn = min(y + 1, H - 1);
        load8<T>(src, sp, W, yn, x, c);
        ec = load1<T>(src, sp, W, yn, hx) * 0x10001u;
        uint32_t lo[4], mi[4], hi[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t t1 = vmin2(a[k], b[k]), t2 = vmax2(a[k], b[k]);
            lo[k] = vmin2(t1, c[k]);
            uint32_t t3 = vmax2(t1, c[k]);
            mi[k] = vmin2(t2, t3);
            hi[k] = vmax2(t2, t3);
        }
        uint32_t elo, emi, ehi;
        {
            uint32_t t1 = vmin2(ea, eb), t2 = vmax2(ea, eb);
            elo = vmin2(t1, ec);
            uint32_t t3 = vmax2(t1, ec);
            emi = vmin2(t2, t3);
            ehi = vmax2(t2, t3);
        }
        // left neighbour pair (columns x-2, x-1) and right (x+8, x+9)
        uint32_t llo = __shfl_up_sync(0xffffffffu, lo[3], 1);
        uint32_t lmi = __shfl_up_sync(0xffffffffu, mi[3], 1);
        uint32_t lhi = __shfl_up_sync(0xffffffffu, hi[3], 1);
        uint32_t rlo = __shfl_down_sync(0xffffffffu, lo[0], 1);
        uint32_t rmi = __shfl_down_sync(0xffffffffu, mi[0], 1);
        uint32_t rhi = __shfl_down_sync(0xffffffffu, hi[0], 1);
        if (lane == 0) { llo = elo; lmi = emi; lhi = ehi; }
        if (lane == 31) { rlo = elo; rmi = emi; rhi = ehi; }
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t plo = k == 0 ? llo : lo[k - 1], pmi = k == 0 ? lmi : mi[k - 1], phi = k == 0 ? lhi : hi[k - 1];
            uint32_t nlo = k == 3 ? rlo : lo[k + 1], nmi = k == 3 ? rmi : mi[k + 1], nhi = k == 3 ? rhi : hi[k + 1];
            uint32_t Llo = shift1(plo, lo[k]), Lmi = shift1(pmi, mi[k]), Lhi = shift1(phi, hi[k]);
            uint32_t Rlo = shift1(lo[k], nlo), Rmi = shift1(mi[k], nmi), Rhi = shift1(hi[k], nhi);
            uint32_t A = vmax2(vmax2(Llo, lo[k]), Rlo);
            uint32_t B = med3(Lmi, mi[k], Rmi);
            uint32_t C = vmin2(vmin2(Lhi, hi[k]), Rhi);
            o[k] = med3(A, B, C);
        }
        store8<T>(dst, dp, W, y, x, o);
#pragma unroll
        for (int k = 0; k < 4; ++k) { a[k] = b[k]; b[k] = c[k]; }
        ea = eb;
        eb = ec;
    }
}

// ---------------------------------------------------------------------------
// r = 2.  Positions (i = rank within a column, j = column after row sorting)
// of the 5x5 block that can still hold the median: (i+1)(j+1) <= 13 and
// (5-i)(5-j) <= 13.  Six entries are provably below it, so the median is the
// 7th smallest (index 6) of these 13 candidates.
__device__ __forceinline__ uint32_t median25_sorted_cols(uint32_t (&m)[5][5]) {
    // m[j][i]: column j, rank i (columns already sorted ascending).
    // Sort each rank-row across the five columns.
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        uint32_t r[5] = {m[0][i], m[1][i], m[2][i], m[3][i], m[4][i]};
        sortnet<5>(r);
#pragma unroll
        for (int j = 0; j < 5; ++j) m[j][i] = r[j];
    }
    uint32_t cand[13];
    int q = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j)
            if ((i + 1) * (j + 1) <= 13 && (5 - i) * (5 - j) <= 13) cand[q++] = m[j][i];
    sortnet<13>(cand);
    return cand[6];
}

template <typename T>
__device__ void sortnet5x5_tile(const unsigned char* __restrict__ src, size_t sp,
                                unsigned char* __restrict__ dst, size_t dp, int W, int H,
                                int rows_per_warp, int tile_x, int tile_y) {
    const int lane = threadIdx.x & 31;
    const int x = tile_x * 256 + lane * 8;
    const int y0 = tile_y * rows_per_warp;
    if (y0 >= H || tile_x * 256 >= W) return;
    const int y1 = min(y0 + rows_per_warp, H);

    // rows y-2..y+2 of the lane's 8 columns, plus a halo pair: lane 0 holds
    // columns (x-2, x-1), lane 31 holds (x+8, x+9).
    uint32_t rw[5][4], he[5];
    const int hx = lane == 0 ? x - 2 : x + 8;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        int yy = clampi(y0 - 2 + t, 0, H - 1);
        load8<T>(src, sp, W, yy, x, rw[t]);
        he[t] = load1<T>(src, sp, W, yy, hx) | (load1<T>(src, sp, W, yy, hx + 1) << 16);
    }
    for (int y = y0; y < y1; ++y) {
        const int yn = min(y + 2, H - 1);
        load8<T>(src, sp, W, yn, x, rw[4]);
        he[4] = load1<T>(src, sp, W, yn, hx) | (load1<T>(src, sp, W, yn, hx + 1) << 16);
        // sort each column pair vertically
        uint32_t s[4][5], hs[5];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t v[5] = {rw[0][k], rw[1][k], rw[2][k], rw[3][k], rw[4][k]};
            sortnet<5>(v);
#pragma unroll
            for (int t = 0; t < 5; ++t) s[k][t] = v[t];
        }
        {
            uint32_t v[5] = {he[0], he[1], he[2], he[3], he[4]};
            sortnet<5>(v);
#pragma unroll
            for (int t = 0; t < 5; ++t) hs[t] = v[t];
        }
        uint32_t lp[5], rp[5];  // pair (x-2, x-1) and (x+8, x+9) as sorted 5-tuples
#pragma unroll
        for (int t = 0; t < 5; ++t) {
            lp[t] = __shfl_up_sync(0xffffffffu, s[3][t], 1);
            rp[t] = __shfl_down_sync(0xffffffffu, s[0][t], 1);
            if (lane == 0) lp[t] = hs[t];
            if (lane == 31) rp[t] = hs[t];
        }
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t m[5][5];
#pragma unroll
            for (int t = 0; t < 5; ++t) {
                uint32_t P = k == 0 ? lp[t] : s[k - 1][t];  // columns 2k-2, 2k-1
                uint32_t C = s[k][t];                        // 2k, 2k+1
                uint32_t N = k == 3 ? rp[t] : s[k + 1][t];  // 2k+2, 2k+3
                m[0][t] = P;
                m[1][t] = shift1(P, C);
                m[2][t] = C;
                m[3][t] = shift1(C, N);
                m[4][t] = N;
            }
            o[k] = median25_sorted_cols(m);
        }
        store8<T>(dst, dp, W, y, x, o);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
#pragma unroll
            for (int k = 0; k < 4; ++k) rw[t][k] = rw[t + 1][k];
            he[t] = he[t + 1];
        }
    }
}

// ---------------------------------------------------------------------------
// r = 3..5 (k = 2r+1).  After every column of the k x k block is sorted and
// then every rank-row is sorted across the k columns, rows and columns are
// both sorted, so entry (i, j) has at least (i+1)(j+1) entries at or below it
// and at least (k-i)(k-j) at or above it.  With M = (k^2+1)/2, entries with
// (i+1)(j+1) > M lie above the median and entries with (k-i)(k-j) > M below
// it; the remaining candidates of rank-row i are the run j in [jlo(i), jhi(i)]
// and the median is the (M - #below)-th smallest candidate.
template <int R>
struct Wide {
    static constexpr int K = 2 * R + 1;
    static constexpr int M = (K * K + 1) / 2;
    static constexpr int HL = (R + 1) / 2;     // neighbour pairs needed on each side
    static constexpr int OUTL = 32 - 2 * HL;   // lanes of a warp that produce outputs
    __host__ __device__ static constexpr int jlo(int i) {
        int j = 0;
        while (j < K && (K - i) * (K - j) > M) ++j;
        return j;
    }
    __host__ __device__ static constexpr int jhi(int i) {
        int j = K - 1;
        while (j >= 0 && (i + 1) * (j + 1) > M) --j;
        return j;
    }
    static constexpr int ncand() {
        int c = 0;
        for (int i = 0; i < K; ++i)
            if (jhi(i) >= jlo(i)) c += jhi(i) - jlo(i) + 1;
        return c;
    }
    static constexpr int nbelow() {
        int c = 0;
        for (int i = 0; i < K; ++i)
            for (int j = 0; j < K; ++j)
                if ((K - i) * (K - j) > M) ++c;
        return c;
    }
    static constexpr int NCAND = ncand();
    static constexpr int SEL = M - nbelow() - 1;  // 0-based index among the sorted candidates
};

// Selecting the answer among the candidates: the candidates of rank-row i
// are already a sorted run, so instead of sorting all of them the runs are
// merged pairwise, shortest first, with Batcher's odd-even merge (valid for
// any two lengths); the compiler then drops every comparator that does not
// reach the selected position (about 35 % fewer min/max than a pruned sort
// of all candidates for k = 11).
struct SelNet {
    int n = 0;                          // comparators: min -> a[c], max -> b[c]
    unsigned char a[1024] = {};
    unsigned char b[1024] = {};
    int sel = 0;                        // candidate slot that ends at the selected rank
};

constexpr void oe_merge(SelNet& net, const unsigned char* A, int m, const unsigned char* B, int n,
                        unsigned char* out) {
    if (m == 0) {
        for (int i = 0; i < n; ++i) out[i] = B[i];
        return;
    }
    if (n == 0) {
        for (int i = 0; i < m; ++i) out[i] = A[i];
        return;
    }
    if (m == 1 && n == 1) {
        net.a[net.n] = A[0];
        net.b[net.n] = B[0];
        ++net.n;
        out[0] = A[0];
        out[1] = B[0];
        return;
    }
    unsigned char ae[64] = {}, ao[64] = {}, be[64] = {}, bo[64] = {};
    int mae = 0, mao = 0, nbe = 0, nbo = 0;
    for (int i = 0; i < m; ++i) {
        if (i % 2 == 0) ae[mae++] = A[i];
        else ao[mao++] = A[i];
    }
    for (int i = 0; i < n; ++i) {
        if (i % 2 == 0) be[nbe++] = B[i];
        else bo[nbo++] = B[i];
    }
    unsigned char v[128] = {}, w[128] = {};
    oe_merge(net, ae, mae, be, nbe, v);  // even-indexed elements
    oe_merge(net, ao, mao, bo, nbo, w);  // odd-indexed elements
    const int nv = mae + nbe, nw = mao + nbo;
    int k = 0;
    out[k++] = v[0];
    for (int i = 0; i < nw; ++i) {
        if (i + 1 < nv) {
            net.a[net.n] = w[i];
            net.b[net.n] = v[i + 1];
            ++net.n;
            out[k++] = w[i];
            out[k++] = v[i + 1];
        } else {
            out[k++] = w[i];
        }
    }
    for (int i = nw + 1; i < nv; ++i) out[k++] = v[i];
}

template <int R>
constexpr SelNet make_selnet() {
    using P = Wide<R>;
    SelNet net{};
    unsigned char lists[2 * P::K + 1][128] = {};
    int len[2 * P::K + 1] = {};
    int nl = 0, idx = 0;
    for (int i = 0; i < P::K; ++i) {
        const int L = P::jhi(i) - P::jlo(i) + 1;
        if (L <= 0) continue;
        for (int j = 0; j < L; ++j) lists[nl][j] = (unsigned char)idx++;
        len[nl++] = L;
    }
    while (nl > 1) {
        int p = 0;
        for (int i = 1; i < nl; ++i)
            if (len[i] < len[p]) p = i;
        int q = p == 0 ? 1 : 0;
        for (int i = 0; i < nl; ++i)
            if (i != p && len[i] < len[q]) q = i;
        unsigned char out[128] = {};
        oe_merge(net, lists[p], len[p], lists[q], len[q], out);
        const int lm = len[p] + len[q];
        for (int j = 0; j < lm; ++j) lists[p][j] = out[j];
        len[p] = lm;
        for (int j = 0; j < len[nl - 1]; ++j) lists[q][j] = lists[nl - 1][j];  // last list into q's place
        len[q] = len[nl - 1];
        --nl;
    }
    net.sel = lists[0][P::SEL];
    return net;
}

template <int R>
struct SelOf {
    static constexpr SelNet net = make_selnet<R>();
};

// Two horizontally adjacent values of row y starting at even column c (any
// c; clamped), as a packed pair.
template <typename T>
__device__ __forceinline__ uint32_t loadpair(const unsigned char* src, size_t sp, int W, int y, int c) {
    const T* row = reinterpret_cast<const T*>(src + (size_t)y * sp);
    if (c >= 0 && c + 1 < W) {
        if (sizeof(T) == 2 && (reinterpret_cast<uintptr_t>(row + c) & 3) == 0)
            return __ldg(reinterpret_cast<const uint32_t*>(row + c));
        if (sizeof(T) == 1 && (reinterpret_cast<uintptr_t>(row + c) & 1) == 0) {
            const uint32_t v = __ldg(reinterpret_cast<const unsigned short*>(row + c));
            return (v & 0xFFu) | ((v >> 8) << 16);
        }
    }
    const uint32_t a = __ldg(row + clampi(c, 0, W - 1));
    const uint32_t b = __ldg(row + clampi(c + 1, 0, W - 1));
    return a | (b << 16);
}

template <typename T>
__device__ __forceinline__ void storepair(unsigned char* dst, size_t dp, int W, int y, int c, uint32_t v) {
    T* row = reinterpret_cast<T*>(dst + (size_t)y * dp);
    if (c + 1 < W) {
        if (sizeof(T) == 2 && (reinterpret_cast<uintptr_t>(row + c) & 3) == 0) {
            *reinterpret_cast<uint32_t*>(row + c) = v;
            return;
        }
        if (sizeof(T) == 1 && (reinterpret_cast<uintptr_t>(row + c) & 1) == 0) {
            *reinterpret_cast<unsigned short*>(row + c) = (unsigned short)((v & 0xFFu) | ((v >> 8) & 0xFF00u));
            return;
        }
    }
    if (c < W) row[c] = (T)(v & 0xFFFFu);
    if (c + 1 < W) row[c + 1] = (T)(v >> 16);
}

// One warp: pairs tile_x*OUTL - HL ... (one aligned column pair per lane; the
// HL lanes at each edge only supply neighbours), rows [tile_y*rpw, +rpw).
template <typename T, int R>
__device__ void sortnet_wide_tile(const unsigned char* __restrict__ src, size_t sp,
                                  unsigned char* __restrict__ dst, size_t dp, int W, int H,
                                  int rows_per_warp, int tile_x, int tile_y) {
    using P = Wide<R>;
    constexpr int K = P::K, HL = P::HL;
    const int lane = threadIdx.x & 31;
    const int c = 2 * (tile_x * P::OUTL + lane - HL);  // first column of the lane's pair
    const int y0 = tile_y * rows_per_warp;
    if (y0 >= H || 2 * tile_x * P::OUTL >= W) return;  // uniform across the warp
    const int y1 = min(y0 + rows_per_warp, H);
    const bool out_lane = lane >= HL && lane < 32 - HL && c < W;

    uint32_t raw[K];  // rows y-R .. y+R of the lane's pair
#pragma unroll
    for (int t = 0; t < K - 1; ++t) raw[t] = loadpair<T>(src, sp, W, clampi(y0 - R + t, 0, H - 1), c);
    for (int y = y0; y < y1; ++y) {
        raw[K - 1] = loadpair<T>(src, sp, W, min(y + R, H - 1), c);
        uint32_t col[K];
#pragma unroll
        for (int t = 0; t < K; ++t) col[t] = raw[t];
        sortnet<K>(col);
        uint32_t cand[P::NCAND];
        int q = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            // rank i of the aligned pairs p-HL .. p+HL
            uint32_t A[2 * HL + 1];
            A[HL] = col[i];
#pragma unroll
            for (int d = 1; d <= HL; ++d) {
                A[HL - d] = __shfl_up_sync(0xffffffffu, col[i], d);
                A[HL + d] = __shfl_down_sync(0xffffffffu, col[i], d);
            }
            // the k packed columns starting at c-R, c-R+1, ..., c+R
            uint32_t row[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int s = j - R + 2 * HL;  // column offset from pair p-HL (>= 0)
                row[j] = (s & 1) ? shift1(A[s >> 1], A[(s >> 1) + 1]) : A[s >> 1];
            }
            sortnet<K>(row);
#pragma unroll
            for (int j = P::jlo(i); j <= P::jhi(i); ++j) cand[q++] = row[j];
        }
        constexpr SelNet net = SelOf<R>::net;
#pragma unroll
        for (int q2 = 0; q2 < net.n; ++q2) {
            const int i = net.a[q2], j = net.b[q2];
            const uint32_t lo = vmin2(cand[i], cand[j]);
            const uint32_t hi = vmax2(cand[i], cand[j]);
            cand[i] = lo;
            cand[j] = hi;
        }
        if (out_lane) storepair<T>(dst, dp, W, y, c, cand[net.sel]);
#pragma unroll
        for (int t = 0; t < K - 1; ++t) raw[t] = raw[t + 1];
    }
}

// ---------------------------------------------------------------------------
// 3D, r = 1 (3x3x3).  Per (x, y') column the z-triple (z-1, z, z+1) is sorted
// once; the 27 window values form a 3 x 9 matrix (rank within the z-triple x
// the 9 (x, y) columns) with sorted columns.  Sorting each rank-row across the
// 9 columns keeps the columns sorted; entry (i, j) then has >= (i+1)(j+1)
// values at or below it and >= (3-i)(9-j) at or above it.  For rank 14 of 27
// the 13 entries with (i+1)(j+1) <= 14 and (3-i)(9-j) <= 14 remain, 7 entries
// lie provably below, so the median is the 7th smallest candidate.
__device__ __forceinline__ uint32_t median27_sorted_cols(uint32_t (&m)[9][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        uint32_t r[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) r[j] = m[j][i];
        sortnet<9>(r);
#pragma unroll
        for (int j = 0; j < 9; ++j) m[j][i] = r[j];
    }
    uint32_t cand[13];
    int q = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 9; ++j)
            if ((i + 1) * (j + 1) <= 14 && (3 - i) * (9 - j) <= 14) cand[q++] = m[j][i];
    sortnet<13>(cand);
    return cand[6];
}

template <typename T>
__device__ __forceinline__ void load8_3d(const unsigned char* src, size_t sp, size_t ss, int W, int H, int D,
                                        int y, int z, int x, uint32_t (&p)[4]) {
    load8<T>(src + (size_t)clampi(z, 0, D - 1) * ss, sp, W, clampi(y, 0, H - 1), x, p);
}

template <typename T>
__device__ __forceinline__ uint32_t load1_3d(const unsigned char* src, size_t sp, size_t ss, int W, int H, int D,
                                            int y, int z, int x) {
    return load1<T>(src + (size_t)clampi(z, 0, D - 1) * ss, sp, W, clampi(y, 0, H - 1), x);
}

// One warp: 256 columns starting at tile_x*256 of row y, slices [z0, z0+zn).
template <typename T>
__device__ void sortnet3d_tile(const unsigned char* __restrict__ src, size_t sp, size_t ss,
                               unsigned char* __restrict__ dst, size_t dp, size_t ds, int W, int H, int D,
                               int zn, int tile_x, int y, int tile_z) {
    const int lane = threadIdx.x & 31;
    const int x = tile_x * 256 + lane * 8;
    const int z0 = tile_z * zn;
    if (z0 >= D || y >= H || tile_x * 256 >= W) return;
    const int z1 = min(z0 + zn, D);
    const int hx = lane == 0 ? x - 1 : x + 8;
    // v[t][row][k]: slice z-1+t, row y-1+row, pair k; e[t][row]: halo column (duplicated)
    uint32_t v[3][3][4], e[3][3];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            load8_3d<T>(src, sp, ss, W, H, D, y - 1 + q, z0 - 1 + t, x, v[t][q]);
            e[t][q] = load1_3d<T>(src, sp, ss, W, H, D, y - 1 + q, z0 - 1 + t, hx) * 0x10001u;
        }
    for (int z = z0; z < z1; ++z) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            load8_3d<T>(src, sp, ss, W, H, D, y - 1 + q, z + 1, x, v[2][q]);
            e[2][q] = load1_3d<T>(src, sp, ss, W, H, D, y - 1 + q, z + 1, hx) * 0x10001u;
        }
        // sorted z-triples of the lane's columns and of its halo column
        uint32_t sl[3][4][3], sh[3][3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t a = v[0][q][k], b = v[1][q][k], c = v[2][q][k];
                uint32_t t1 = vmin2(a, b), t2 = vmax2(a, b);
                sl[q][k][0] = vmin2(t1, c);
                uint32_t t3 = vmax2(t1, c);
                sl[q][k][1] = vmin2(t2, t3);
                sl[q][k][2] = vmax2(t2, t3);
            }
            uint32_t a = e[0][q], b = e[1][q], c = e[2][q];
            uint32_t t1 = vmin2(a, b), t2 = vmax2(a, b);
            sh[q][0] = vmin2(t1, c);
            uint32_t t3 = vmax2(t1, c);
            sh[q][1] = vmin2(t2, t3);
            sh[q][2] = vmax2(t2, t3);
        }
        uint32_t lp[3][3], rp[3][3];  // neighbour pairs (x-2, x-1) and (x+8, x+9)
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                lp[q][i] = __shfl_up_sync(0xffffffffu, sl[q][3][i], 1);
                rp[q][i] = __shfl_down_sync(0xffffffffu, sl[q][0][i], 1);
                if (lane == 0) lp[q][i] = sh[q][i];
                if (lane == 31) rp[q][i] = sh[q][i];
            }
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t m[9][3];
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const uint32_t P = k == 0 ? lp[q][i] : sl[q][k - 1][i];
                    const uint32_t C = sl[q][k][i];
                    const uint32_t N = k == 3 ? rp[q][i] : sl[q][k + 1][i];
                    m[3 * q + 0][i] = shift1(P, C);
                    m[3 * q + 1][i] = C;
                    m[3 * q + 2][i] = shift1(C, N);
                }
            o[k] = median27_sorted_cols(m);
        }
        store8<T>(dst + (size_t)z * ds, dp, W, y, x, o);
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v[0][q][k] = v[1][q][k];
                v[1][q][k] = v[2][q][k];
            }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            e[0][q] = e[1][q];
            e[1][q] = e[2][q];
        }
    }
}

}  // namespace hrm

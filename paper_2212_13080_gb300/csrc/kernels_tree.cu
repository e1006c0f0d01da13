// Binning, split, stable sort by finest cell, recombination of split charges
// and the FP64 energy reduction.
#include <algorithm>
#include <type_traits>

#include "fmm_internal.cuh"
#include "launch.cuh"
#include "lagrange.cuh"

namespace fmm {

// ---------------------------------------------------------------------------
// §2.2 step 1: the canonical single-precision map of a coordinate to its
// finest cell.  u = fl32(fl32(x - x0) / fl32(L)) (wrapped in the periodic form),
// c = min(floor(u 2^depth), 2^depth - 1), t = u 2^depth - c (exact).
// Every operation is an explicitly rounded intrinsic: no contraction.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bin_axis(const Geom &g, float x, int a, float &t, int &c,
                                         int &st) {
    float u = __fdiv_rn(__fsub_rn(x, g.x0[a]), g.Lf);
    if (!isfinite(u)) {
        st |= ST_NONFINITE;
        u = 0.0f;
    }
    if (g.periodic) {
        u = __fsub_rn(u, floorf(u));
        if (u >= 1.0f) u = 0.0f;
    } else if (!(u >= 0.0f && u < 1.0f)) {
        st |= ST_OUT_OF_BOX;
        u = 0.0f;
    }
    float v = __fmul_rn(u, (float)g.S);
    int ci = (int)floorf(v);
    if (ci > g.S - 1) ci = g.S - 1;
    t = __fsub_rn(v, (float)ci);
    c = ci;
}

// Split decision of one axis (§2.3; walls too in the periodic form, §4.2).
// mode 0: not split (1 entry); 1: split below the cell (plane between c-1 and
// c); 2: split above (plane between c and c+1).
struct AxisInfo {
    int mode, cl, cu, m;
    float t;
};

__device__ __forceinline__ AxisInfo split_axis_info(const Geom &g, int c, float t) {
    AxisInfo A;
    A.t = t;
    A.mode = 0;
    A.cl = A.cu = c;
    A.m = 1;
    if (!g.continuous) return A;
    bool lower = (g.periodic || c > 0) && t < g.dtf;
    bool upper = (g.periodic || c < g.S - 1) && t > g.dthi;
    if (lower) {
        A.mode = 1;
        A.cl = c - 1;
        A.cu = c;
    } else if (upper) {
        A.mode = 2;
        A.cl = c;
        A.cu = c + 1;
    } else {
        return A;
    }
    if (g.periodic) {
        A.cl = (A.cl + g.S) % g.S;
        A.cu = A.cu % g.S;
    }
    A.m = g.p + (g.p & 1);  // odd p: the middle node becomes two half charges
    return A;
}

// Entry e of a split axis: cell, local coordinate, weight, d weight / du.
// Segment nodes s_k = -1 + 2k/(p-1) (length 2d centred on the plane); the
// weights are the one-dimensional replacement onto them, g_k((sigma+1)/2),
// sigma = signed distance from the plane in units of d.
template <typename real>
__device__ __forceinline__ void split_entry(const Geom &g, const Coef<real> &C, const AxisInfo &A,
                                            int e, int &cell, real &t, real &w, real &dw) {
    if (A.mode == 0) {
        cell = A.cl;
        t = (real)A.t;
        w = 1;
        dw = 0;
        return;
    }
    const int p = g.p;
    const real dt = (real)g.dtf;
    real sigma = (A.mode == 1) ? (real)A.t / dt : ((real)A.t - real(1)) / dt;
    real x = (sigma + real(1)) * real(0.5);
    int k, side;  // side 0: lower cell, 1: upper cell
    real half = 1;
    if (p & 1) {
        int mid = (p - 1) / 2;
        if (e < mid) {
            k = e;
            side = 0;
        } else if (e == mid) {
            k = mid;
            side = 0;
            half = real(0.5);
        } else if (e == mid + 1) {
            k = mid;
            side = 1;
            half = real(0.5);
        } else {
            k = e - 1;
            side = 1;
        }
    } else {
        k = e;
        side = (2 * k < p - 1) ? 0 : 1;
    }
    real gk, dgk;
    lag_one(C, p, k, x, gk, dgk);
    w = half * gk;
    dw = half * dgk * (real(0.5) / dt) * (real)g.S;
    real s = (real)(2 * k) / (real)(p - 1) - real(1);
    if (half != real(1)) {
        t = side ? real(0) : real(1);
    } else {
        t = side ? s * dt : real(1) + s * dt;
    }
    cell = side ? A.cu : A.cl;
}

// Charges of particle i (continuous form) and its split axes (bit a: axis a).
__device__ __forceinline__ int split_count_one(const Geom &g, const float *__restrict__ pos, int i,
                                               unsigned char &ax, int &st) {
    int m = 1;
    ax = 0;
    for (int a = 0; a < 3; a++) {
        float t;
        int c;
        bin_axis(g, pos[3 * i + a], a, t, c, st);
        AxisInfo A = split_axis_info(g, c, t);
        m *= A.m;
        if (A.mode) ax |= (unsigned char)(1 << a);
    }
    return m;
}

// Emits the charges, one thread per charge (no divergence on split
// particles): charge e is entry k = e - offset[i] of particle i, the tensor
// product of its axes with x fastest.  Writes the Morton key, (t, q_eff),
// (W, dW/du) and origin, and counts the charges of every finest cell; the
// count before this charge's increment is its rank among the cell's charges
// in arrival order (e_rank), the slot the sort scatters it to.  The plain form
// emits every particle (n_eff = n); the continuous form's n_eff was set by the
// scan of the charge counts.
template <typename real>
struct KEmit {
    static constexpr int BS = 0, MINB = 0;
    Geom g;
    Coef<real> C;
    int n;
    const float *__restrict__ pos;
    const float *__restrict__ q;
    const int *__restrict__ offset;
    uint32_t *__restrict__ e_key;
    typename Vec4<real>::T *__restrict__ e_pt;
    typename Vec4<real>::T *__restrict__ e_wd;
    int *__restrict__ e_origin;
    int *__restrict__ e_rank;
    int *__restrict__ leaf_count;
    WsHeader *hdr;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        int st = 0;
        const int ne = offset ? hdr->n_eff : n;
        if (!offset && bid_ == 0 && threadIdx.x == 0) hdr->n_eff = n;
        for (int e = bid_ * blockDim.x + threadIdx.x; e < ne; e += nblk_ * blockDim.x) {
            const int i = offset ? e_origin[e] : e;
            int k = offset ? e - offset[i] : 0;
            AxisInfo A[3];
            for (int a = 0; a < 3; a++) {
                float t;
                int c;
                bin_axis(g, pos[3 * i + a], a, t, c, st);
                A[a] = split_axis_info(g, c, t);
            }
            const int ex = k % A[0].m;
            k /= A[0].m;
            const int ey = k % A[1].m, ez = k / A[1].m;
            int cx, cy, cz;
            real tx, ty, tz, wx, wy, wz, dwx, dwy, dwz;
            split_entry(g, C, A[0], ex, cx, tx, wx, dwx);
            split_entry(g, C, A[1], ey, cy, ty, wy, dwy);
            split_entry(g, C, A[2], ez, cz, tz, wz, dwz);
            const real W = wx * wy * wz;
            const uint32_t key = morton_encode(cx, cy, cz);
            e_key[e] = key;
            typename Vec4<real>::T v;
            v.x = tx;
            v.y = ty;
            v.z = tz;
            v.w = (real)q[i] * W;
            e_pt[e] = v;
            if (e_wd) {
                typename Vec4<real>::T d;
                d.x = W;
                d.y = dwx * wy * wz;
                d.z = wx * dwy * wz;
                d.w = wx * wy * dwz;
                e_wd[e] = d;
            }
            if (!offset) e_origin[e] = i;
            e_rank[e] = atomicAdd(&leaf_count[key], 1);
        }
        if (st) atomicOr(&hdr->status, st);
    }
};
template <typename real>
__global__ void k_emit(const __grid_constant__ KEmit<real> k) {
    k.run(blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 (three passes: block sums, scan of block sums,
// block-local scan plus prefix); out has m+1 entries, out[m] = total.  The
// continuous form's charge counts are computed by the first pass itself, and
// its last pass also marks the particle of every emitted charge.  Up to
// SCAN1_MAX entries (the finest cells to depth 5) are scanned by one CTA in
// one launch.  The last pass and the one-CTA scan read and write a warp's
// entries 128 at a time (int4 per lane).
// ---------------------------------------------------------------------------
#define SCAN_BS 256
#define SCAN_IPT 8
#define SCAN_TILE (SCAN_BS * SCAN_IPT)
#define SCAN1_BS 1024
#define SCAN1_IPT 32
#define SCAN1_MAX (SCAN1_BS * SCAN1_IPT)

__device__ __forceinline__ int block_excl_scan(int v, int *sh, int &total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    int pre = (wid > 0 ? sh[wid - 1] : 0) + x - v;
    __syncthreads();
    return pre;
}

struct KScanReduce {
    static constexpr int BS = 0, MINB = 0;
    const int *__restrict__ in;
    int m;
    int *__restrict__ bsum;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        __shared__ int sh[32];
        int base = bid_ * SCAN_TILE;
        int s = 0;
        for (int k = 0; k < SCAN_IPT; k++) {
            int i = base + k * SCAN_BS + threadIdx.x;
            if (i < m) s += in[i];
        }
        int tot;
        block_excl_scan(s, sh, tot);
        if (threadIdx.x == 0) bsum[bid_] = tot;
    }
};
__global__ void k_scan_reduce(const __grid_constant__ KScanReduce k) {
    k.run(blockIdx.x, gridDim.x);
}

// first pass over the particles (continuous form): charges per particle and
// split axes (§2.3), written out and summed per block
struct KSplitCount {
    static constexpr int BS = 0, MINB = 0;
    Geom g;
    int n;
    const float *__restrict__ pos;
    int *__restrict__ count;
    unsigned char *__restrict__ axes;
    int *__restrict__ bsum;
    WsHeader *hdr;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        __shared__ int sh[32];
        const int base = bid_ * SCAN_TILE;
        int s = 0, st = 0;
        for (int k = 0; k < SCAN_IPT; k++) {
            const int i = base + k * SCAN_BS + threadIdx.x;
            if (i < n) {
                unsigned char ax;
                const int m = split_count_one(g, pos, i, ax, st);
                count[i] = m;
                axes[i] = ax;
                s += m;
            }
        }
        int tot;
        block_excl_scan(s, sh, tot);
        if (threadIdx.x == 0) bsum[bid_] = tot;
        if (st) atomicOr(&hdr->status, st);
    }
};
__global__ void k_split_count_reduce(const __grid_constant__ KSplitCount k) {
    k.run(blockIdx.x, gridDim.x);
}

struct KScanBlocks {
    static constexpr int BS = 0, MINB = 0;
    int *bsum;
    int nb;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        __shared__ int sh[32];
        int carry = 0;
        for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
            int i = b0 + threadIdx.x;
            int v = i < nb ? bsum[i] : 0;
            int tot;
            int pre = block_excl_scan(v, sh, tot);
            if (i < nb) bsum[i] = carry + pre;
            carry += tot;
        }
        if (threadIdx.x == 0) bsum[nb] = carry;
    }
};
__global__ void k_scan_blocks(const __grid_constant__ KScanBlocks k) {
    k.run(blockIdx.x, gridDim.x);
}

// Exclusive scan of a CTA's tile of 128 * IT entries per warp from base: warp
// w owns [base + 128 IT w, base + 128 IT (w + 1)), read 128 entries at a time
// (one int4 per lane: coalesced).  v[it] gets the lane's four entries of chunk
// it, pre[it] the exclusive prefix (within the tile) of the first of them;
// total the tile's sum.
template <int IT>
__device__ __forceinline__ void tile_scan(const int *__restrict__ in, int base, int m, int4 (&v)[IT],
                                          int (&pre)[IT], int *sh, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int run = 0;
#pragma unroll
    for (int it = 0; it < IT; it++) {
        const int i = base + (warp * IT + it) * 128 + 4 * lane;
        int4 x;
        if (i + 4 <= m) {
            x = *reinterpret_cast<const int4 *>(in + i);
        } else {
            x.x = i < m ? in[i] : 0;
            x.y = i + 1 < m ? in[i + 1] : 0;
            x.z = i + 2 < m ? in[i + 2] : 0;
            x.w = i + 3 < m ? in[i + 3] : 0;
        }
        v[it] = x;
        const int s = x.x + x.y + x.z + x.w;
        int inc = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        pre[it] = run + inc - s;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    // the warps' totals: only lane 31 contributes, so every lane of warp w
    // receives the sum over the warps before w
    const int wpre = block_excl_scan(lane == 31 ? run : 0, sh, total);
#pragma unroll
    for (int it = 0; it < IT; it++) pre[it] += wpre;
}

// writes the exclusive prefixes of the lane's four entries of chunk it
__device__ __forceinline__ void tile_store(int *__restrict__ out, int i, int m, int p, int4 x) {
    const int4 r = make_int4(p, p + x.x, p + x.x + x.y, p + x.x + x.y + x.z);
    if (i + 4 <= m) {
        *reinterpret_cast<int4 *>(out + i) = r;
    } else {
        if (i < m) out[i] = r.x;
        if (i + 1 < m) out[i + 1] = r.y;
        if (i + 2 < m) out[i + 2] = r.z;
    }
}

// MARK (charges per particle): the emitted charges are those of the particles
// whose charges end at or before cap, a prefix since the offsets increase; the
// particle of each of them goes to e_origin, and n_eff (their number) to the
// header, by the particle where the prefix ends (with the overflow status) or,
// when every particle fits, by the last block.
template <bool MARK>
__device__ __forceinline__ void mark_one(int i, int m, int pre, int cnt, int cap, int *__restrict__ e_origin,
                                         WsHeader *hdr) {
    if (!MARK || i >= m) return;
    const int end = pre + cnt;
    if (end <= cap) {
        for (int j = pre; j < end; j++) e_origin[j] = i;
    } else if (pre <= cap) {
        hdr->n_eff = pre;
        atomicOr(&hdr->status, ST_SPLIT_OVERFLOW);
    }
}

template <bool MARK>
struct KScanApply {
    static constexpr int BS = SCAN_BS, MINB = 0;  // bounds on the block size only
    const int *__restrict__ in;
    int m;
    const int *__restrict__ bsum;
    int *__restrict__ out;
    int cap;
    int *__restrict__ e_origin;
    WsHeader *hdr;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        __shared__ int sh[32];
        constexpr int IT = SCAN_TILE / SCAN_BS / 4;
        const int base = bid_ * SCAN_TILE;
        int4 v[IT];
        int pre[IT];
        int tot;
        tile_scan<IT>(in, base, m, v, pre, sh, tot);
        const int carry = bsum[bid_];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int it = 0; it < IT; it++) {
            const int i = base + (warp * IT + it) * 128 + 4 * lane;
            const int p = pre[it] + carry;
            tile_store(out, i, m, p, v[it]);
            mark_one<MARK>(i, m, p, v[it].x, cap, e_origin, hdr);
            mark_one<MARK>(i + 1, m, p + v[it].x, v[it].y, cap, e_origin, hdr);
            mark_one<MARK>(i + 2, m, p + v[it].x + v[it].y, v[it].z, cap, e_origin, hdr);
            mark_one<MARK>(i + 3, m, p + v[it].x + v[it].y + v[it].z, v[it].w, cap, e_origin, hdr);
        }
        if (bid_ == nblk_ - 1 && threadIdx.x == 0) {
            const int total = bsum[nblk_];
            out[m] = total;
            if (MARK && total <= cap) hdr->n_eff = total;
        }
    }
};
template <bool MARK>
__global__ void __launch_bounds__(KScanApply<MARK>::BS) k_scan_apply(const __grid_constant__ KScanApply<MARK> k) {
    k.run(blockIdx.x, gridDim.x);
}

// m <= SCAN1_MAX: the whole array is one tile of the CTA
struct KScanOne {
    static constexpr int BS = SCAN1_BS, MINB = 0;  // bounds on the block size only
    const int *__restrict__ in;
    int m;
    int *__restrict__ out;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        __shared__ int sh[32];
        constexpr int IT = SCAN1_MAX / SCAN1_BS / 4;
        int4 v[IT];
        int pre[IT];
        int tot;
        tile_scan<IT>(in, 0, m, v, pre, sh, tot);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int it = 0; it < IT; it++) tile_store(out, (warp * IT + it) * 128 + 4 * lane, m, pre[it], v[it]);
        if (threadIdx.x == 0) out[m] = tot;
    }
};
__global__ void __launch_bounds__(KScanOne::BS) k_scan_one(const __grid_constant__ KScanOne k) {
    k.run(blockIdx.x, gridDim.x);
}

int launch_scan(const int *in, int *out, int m, int *tmp, cudaStream_t st, Tracer &tr) {
    if (m <= SCAN1_MAX) {
        launch_k(tr, FMM_TAG(S_SCAN_ONE, 0), k_scan_one, KScanOne{in, m, out}, 1, SCAN1_BS, 0, st);
        return 1;
    }
    int nb = (m + SCAN_TILE - 1) / SCAN_TILE;
    launch_k(tr, FMM_TAG(S_SCAN_REDUCE, 0), k_scan_reduce, KScanReduce{in, m, tmp}, nb, SCAN_BS, 0, st);
    launch_k(tr, FMM_TAG(S_SCAN_BLOCKS, 0), k_scan_blocks, KScanBlocks{tmp, nb}, 1, 1024, 0, st);
    launch_k(tr, FMM_TAG(S_SCAN_APPLY, 0), k_scan_apply<false>,
             KScanApply<false>{in, m, tmp, out, 0, nullptr, nullptr}, nb, SCAN_BS, 0, st);
    return 3;
}

template <typename real>
void launch_bin_emit(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                     int n, const float *pos, const float *q, cudaStream_t st, Tracer &tr) {
    const int *offset = nullptr;
    tr.begin(FMM_STAGE_BIN, st);
    if (g.continuous) {
        // charges per particle, their offsets, the particle of every emitted charge
        const int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
        launch_k(tr, FMM_TAG(S_SPLIT_COUNT, 0), k_split_count_reduce,
                 KSplitCount{g, n, pos, P.count, P.axes, P.scan_tmp, P.hdr}, nb, SCAN_BS, 0, st);
        launch_k(tr, FMM_TAG(S_SCAN_BLOCKS_E, 0), k_scan_blocks, KScanBlocks{P.scan_tmp, nb}, 1, 1024, 0, st);
        launch_k(tr, FMM_TAG(S_SCAN_APPLY_E, 0), k_scan_apply<true>,
                 KScanApply<true>{P.count, n, P.scan_tmp, P.offset, (int)W.cap, P.e_origin, P.hdr}, nb, SCAN_BS, 0,
                 st);
        tr.count(3);
        offset = P.offset;
    }
    int64_t ne_max = offset ? W.cap : n;
    int nbe = (int)((ne_max + 255) / 256);
    if (nbe < 1) nbe = 1;
    if (nbe > 152 * 64) nbe = 152 * 64;
    launch_k(tr, FMM_TAG(S_EMIT, 0), k_emit<real>,
             KEmit<real>{g, C, n, pos, q, offset, P.e_key, P.e_pt, g.continuous ? P.e_wd : nullptr, P.e_origin,
                         P.e_rank, P.leaf_count, P.hdr},
             nbe, 256, 0, st);
    tr.count();
    tr.end();
}

// ---------------------------------------------------------------------------
// stable counting sort by finest cell: scatter to the slot of each charge's
// arrival rank in its cell, then order each cell's segment by emitted index
// (= particle order), then gather.
// ---------------------------------------------------------------------------
struct KScatter {
    static constexpr int BS = 0, MINB = 0;
    const WsHeader *hdr;
    const uint32_t *__restrict__ e_key;
    const int *__restrict__ e_rank;
    const int *__restrict__ leaf_start;
    int *__restrict__ tmp;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        int ne = hdr->n_eff;
        for (int e = bid_ * blockDim.x + threadIdx.x; e < ne; e += nblk_ * blockDim.x)
            tmp[leaf_start[e_key[e]] + e_rank[e]] = e;
    }
};
__global__ void k_scatter(const __grid_constant__ KScatter k) {
    k.run(blockIdx.x, gridDim.x);
}

// one warp per finest cell: rank every element of the cell's segment among
// the segment (emission indices, all distinct), and move it to its sorted
// slot: charge, origin and perm (slot -> emitted index).  Up to 64 elements
// are ranked in registers (two per lane, compared through shuffles).
template <typename real>
struct KLeafGather {
    static constexpr int BS = 0, MINB = 0;
    int ncell;
    const int *__restrict__ leaf_start;
    const int *__restrict__ tmp;
    const typename Vec4<real>::T *__restrict__ e_pt;
    const int *__restrict__ e_origin;
    typename Vec4<real>::T *__restrict__ s_pt;
    int *__restrict__ s_origin;
    int *__restrict__ perm;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        int lane = threadIdx.x & 31;
        int warp = (bid_ * blockDim.x + threadIdx.x) >> 5;
        int nwarps = (nblk_ * blockDim.x) >> 5;
        for (int c = warp; c < ncell; c += nwarps) {
            int s0 = leaf_start[c], s1 = leaf_start[c + 1];
            int cnt = s1 - s0;
            if (cnt == 0) continue;
            if (cnt <= 64) {
                const int v0 = lane < cnt ? tmp[s0 + lane] : 0x7fffffff;
                const int v1 = lane + 32 < cnt ? tmp[s0 + 32 + lane] : 0x7fffffff;
                int r0 = 0, r1 = 0;
                const int c0 = cnt < 32 ? cnt : 32;
                for (int j = 0; j < c0; j++) {
                    const int w = __shfl_sync(0xffffffffu, v0, j);
                    r0 += (w < v0);
                    r1 += (w < v1);
                }
                for (int j = 0; j < cnt - 32; j++) {
                    const int w = __shfl_sync(0xffffffffu, v1, j);
                    r0 += (w < v0);
                    r1 += (w < v1);
                }
                if (lane < cnt) {
                    const int slot = s0 + r0;
                    perm[slot] = v0;
                    s_pt[slot] = e_pt[v0];
                    s_origin[slot] = e_origin[v0];
                }
                if (lane + 32 < cnt) {
                    const int slot = s0 + r1;
                    perm[slot] = v1;
                    s_pt[slot] = e_pt[v1];
                    s_origin[slot] = e_origin[v1];
                }
            } else {
                for (int i = lane; i < cnt; i += 32) {
                    int v = tmp[s0 + i];
                    int r = 0;
                    for (int j = 0; j < cnt; j++) r += (tmp[s0 + j] < v);
                    const int slot = s0 + r;
                    perm[slot] = v;
                    s_pt[slot] = e_pt[v];
                    s_origin[slot] = e_origin[v];
                }
            }
        }
    }
};
template <typename real>
__global__ void k_leaf_gather(const __grid_constant__ KLeafGather<real> k) {
    k.run(blockIdx.x, gridDim.x);
}

template <typename real>
void launch_sort(const Geom &g, const Ptrs<real> &P, const WsLayout &W, int n, cudaStream_t st,
                 Tracer &tr) {
    int ncell = (int)W.ncell;
    tr.begin(FMM_STAGE_SORT, st);
    tr.count(launch_scan(P.leaf_count, P.leaf_start, ncell, P.scan_tmp, st, tr));
    int nbp = (int)((W.cap + 255) / 256);
    if (nbp < 1) nbp = 1;
    if (nbp > 152 * 64) nbp = 152 * 64;
    launch_k(tr, FMM_TAG(S_SCATTER, 0), k_scatter, KScatter{P.hdr, P.e_key, P.e_rank, P.leaf_start, P.tmp}, nbp,
             256, 0, st);
    int nbl = (ncell * 32 + 255) / 256;
    if (nbl > 152 * 64) nbl = 152 * 64;
    launch_k(tr, FMM_TAG(S_LEAF_GATHER, 0), k_leaf_gather<real>,
             KLeafGather<real>{ncell, P.leaf_start, P.tmp, P.e_pt, P.e_origin, P.s_pt, P.s_origin, P.perm}, nbl, 256,
             0, st);
    tr.count(2);
    tr.end();
}

// ---------------------------------------------------------------------------
// Adjoint forces of split particles, difference form (§2.3).  Along a split
// axis the adjoint force is -q sum_k (dW_k/dx) phi(s_k); the weights sum to
// one, so their derivatives sum to zero and the same force is
// -q sum_k (dW_k/dx) D_k with D_k = phi(s_k) - phi(r) for any reference point
// r.  dW/dx ~ 1/(2d) amplifies independent errors of the phi(s_k): FP32
// rounding of each charge's near- and far-field sums, and (for even p) the
// single-precision rounding of the charges' positions (the nodes plane +
// d(-1 + 2k/(p-1)) are not binary fractions).  This kernel forms the D_k
// directly, for split particles only, r = the particle's first charge (the
// node plane - d of every split axis, exact in single precision), s_k the
// exact node (a single-precision pair).
//
// One split axis a (nearly every split particle): the charges differ from r
// by delta_k along a only.  The neighbour cells form three slabs along a:
// u = -1 (seen by r and the charges below the plane), u = 0..1 (seen by all),
// u = 2 (seen by the charges above).  For a source farther than 16 max|delta|
// from r, 1/|s_k - x| = sum_n delta_k^n c_n(mu) / rho^(n+1) (Legendre; for
// 1/r^2 the Chebyshev U_n and one more power), rho = |x - r|, mu its cosine
// with the axis, so every slab reduces to seven moments M_n = sum q c_n /
// rho^(n+1), n = 0..6, independent of the charges (h^7 < 4e-9 is dropped);
// the few sources closer than that to r take direct terms per charge.  Then
// D_k = sum_{n>=1} delta_k^n (M_n(middle) + M_n(the other slab its side sees))
// + direct terms, and above the plane + M_0(u = 2) - M_0(u = -1).  Far field:
// g(s_k) . L - g(r) . L = (W_a(s_k) - W_a(r)) W_b W_c . L of the lower cell
// (below), or (W_a(s_k) - e_0) W_b W_c . L_upper + X with X = g(plane) .
// L_upper - g(r) . L_lower (above): the weight differences are small and
// exact to their own rounding, so these sums run in single precision, and
// only X (with the two M_0, which cancel against it) in double precision.
// Several split axes (a fraction of a percent): direct terms, chunks of CH
// charges per task, near-field part q (1/|s_k - x| - 1/|r - x|) = -q n /
// (r0 rk (r0 + rk)) with n = delta . (delta - 2 (x - r)) where both see the
// source, plain terms where one does, far field in double precision.
// Same-particle and coincident charges are skipped as in the near field.
// Persistent warps take one task each: the chunks of the several-axis
// particles first (the longest), then one task per one-axis particle.
// POW: the pair function 1/r (1) or 1/r^2 (2).
// ---------------------------------------------------------------------------

// Entry e of split axis A: the side (0 lower, 1 upper cell of the plane; 0
// for an axis that is not split), the exact node as a single-precision pair
// t = th + tl (error-free transformations: the quotient 2k/(p-1) with its
// remainder, TwoSum for the shifts; dt is a power of two), and the
// single-precision coordinate the emission computed (the expression of
// split_entry), which the near field compares for coincidence.
__device__ __forceinline__ void split_entry_df(const Geom &g, const AxisInfo &A, int e, int &side, float &th,
                                               float &tl, float &tf) {
    if (A.mode == 0) {
        side = 0;
        th = tf = A.t;
        tl = 0.0f;
        return;
    }
    const int p = g.p;
    int k;
    bool half = false;
    if (p & 1) {
        const int mid = (p - 1) / 2;
        if (e < mid) {
            k = e;
            side = 0;
        } else if (e == mid) {
            k = mid;
            side = 0;
            half = true;
        } else if (e == mid + 1) {
            k = mid;
            side = 1;
            half = true;
        } else {
            k = e - 1;
            side = 1;
        }
    } else {
        k = e;
        side = (2 * k < p - 1) ? 0 : 1;
    }
    const float dtf = g.dtf;
    const float sf = (float)(2 * k) / (float)(p - 1) - 1.0f;
    tf = half ? (side ? 0.0f : 1.0f) : (side ? sf * dtf : 1.0f + sf * dtf);
    if (half) {
        th = side ? 0.0f : 1.0f;
        tl = 0.0f;
        return;
    }
    const float num = (float)(2 * k), den = (float)(p - 1);
    const float qh = __fdiv_rn(num, den), ql = __fdiv_rn(fmaf(-qh, den, num), den);  // 2k/(p-1)
    const float sh = __fsub_rn(qh, 1.0f), bb = __fsub_rn(sh, qh);                      // s = q - 1
    const float sl = __fadd_rn(__fadd_rn(__fsub_rn(qh, __fsub_rn(sh, bb)), __fsub_rn(-1.0f, bb)), ql);
    const float ah = __fmul_rn(sh, dtf), al = __fmul_rn(sl, dtf);                    // s dt (exact)
    if (side) {
        th = __fadd_rn(ah, al);
        tl = __fsub_rn(al, __fsub_rn(th, ah));
    } else {  // 1 + s dt
        const float t1 = __fadd_rn(1.0f, ah), b2 = __fsub_rn(t1, 1.0f);
        const float e2 = __fadd_rn(__fadd_rn(__fsub_rn(1.0f, __fsub_rn(t1, b2)), __fsub_rn(ah, b2)), al);
        th = __fadd_rn(t1, e2);
        tl = __fsub_rn(e2, __fsub_rn(th, t1));
    }
}

// x - s along one axis, the source x at coordinate v of a cell `shift` cells
// from the charge's cell, the charge at t = th + tl of its own cell: each case
// subtracts in the frame where the nearby operands are exact (Sterbenz)
__device__ __forceinline__ float sd_axis_diff(float v, int shift, float th, float tl) {
    const float d = shift == 1 ? v - (th - 1.0f) : (shift == -1 ? (v - 1.0f) - th : (v + (float)shift) - th);
    return d - tl;
}

#define SD_WARPS 4  // warps per CTA

// The split particles as tasks.  slist[0] = the number split along one axis,
// listed from slist[2] up; slist[1] = the number split along two or three,
// listed from slist[n + 1] down (each particle is one or the other, so the
// two never meet).  m1 = the charges of a particle split along one axis.
struct KSplitList {
    static constexpr int BS = 0, MINB = 0;
    int n;
    int m1;
    const int *__restrict__ count;
    const int *__restrict__ offset;
    const WsHeader *hdr;
    int *__restrict__ slist;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        const int i = bid_ * blockDim.x + threadIdx.x, lane = threadIdx.x & 31;
        const bool mine = i < n && count[i] > 1 && offset[i] + count[i] <= hdr->n_eff;
        const bool one = mine && count[i] <= m1;
        const unsigned b1 = __ballot_sync(0xffffffffu, one), bm = __ballot_sync(0xffffffffu, mine && !one);
        int base1 = 0, basem = 0;
        if (lane == 0 && b1) base1 = atomicAdd(&slist[0], __popc(b1));
        if (lane == 0 && bm) basem = atomicAdd(&slist[1], __popc(bm));
        base1 = __shfl_sync(0xffffffffu, base1, 0);
        basem = __shfl_sync(0xffffffffu, basem, 0);
        const unsigned below = (1u << lane) - 1u;
        if (one)
            slist[2 + base1 + __popc(b1 & below)] = i;
        else if (mine)
            slist[n + 1 - (basem + __popc(bm & below))] = i;
    }
};
__global__ void k_split_list(const __grid_constant__ KSplitList k) {
    k.run(blockIdx.x, gridDim.x);
}

#define SD_NM 7                 // series terms n = 0..6
#define SD_NMOM (3 * SD_NM)     // moments of the three slabs

// (h, l) += (bh, bl) in single-precision pair arithmetic (TwoSum of the high
// parts, the low parts and the error added to the low part)
__device__ __forceinline__ void sd_two_sum(float &h, float &l, float bh, float bl) {
    const float s = h + bh, v = s - h, e = (h - (s - v)) + (bh - v), t = e + l + bl;
    h = s + t;
    l = t - (h - s);
}
#define SD_KMAX (FMM_MAXP + 1)  // charges of a particle split along one axis, at most

// q (1/|s_k - x|^POW - 1/|r - x|^POW) for a source x seen by r (inR) and/or by
// the charge s_k (its cells: side bits sdk); d0 = x - r, r02 = |d0|^2, ri0 =
// 1/|d0| (0 where x = r).  kk: s_k - r (3), s_k as th (3) + tl (3), and the
// single-precision coordinate the emission computed (3).
template <int POW>
__device__ __forceinline__ float sd_pair_term(const float4 &v, int ux, int uy, int uz, float d0x, float d0y,
                                              float d0z, float r02, float ri0, bool inR, const float *kk,
                                              int sdk) {
    const int sx = sdk & 1, sy = (sdk >> 1) & 1, sz = sdk >> 2;
    const bool inK = ux >= sx - 1 && ux <= sx + 1 && uy >= sy - 1 && uy <= sy + 1 && uz >= sz - 1 && uz <= sz + 1;
    // x - s_k directly, accurate also when x is close to s_k
    const float dkx = sd_axis_diff(v.x, ux - sx, kk[3], kk[6]), dky = sd_axis_diff(v.y, uy - sy, kk[4], kk[7]),
                dkz = sd_axis_diff(v.z, uz - sz, kk[5], kk[8]);
    const float rk2 = dkx * dkx + dky * dky + dkz * dkz;
    // coincident with the emitted charge (the single-precision positions the
    // near field compares): skipped as there.  Only a charge within a few ulps
    // of s_k can be.
    bool zk = false;
    if (rk2 < 1e-12f)
        zk = sd_axis_diff(v.x, ux - sx, kk[9], 0.0f) == 0.0f && sd_axis_diff(v.y, uy - sy, kk[10], 0.0f) == 0.0f &&
             sd_axis_diff(v.z, uz - sz, kk[11], 0.0f) == 0.0f;
    const float rik = (rk2 > 0.0f && !zk) ? rsqrtf(rk2) : 0.0f;
    float term = 0.0f;
    if (inK && inR && rik > 0.0f && ri0 > 0.0f) {
        // |s_k - x|^2 - |r - x|^2 = delta . (delta - 2 (x - r)): a small number
        // with a small relative error
        const float nm = kk[0] * (kk[0] - 2.0f * d0x) + kk[1] * (kk[1] - 2.0f * d0y) + kk[2] * (kk[2] - 2.0f * d0z);
        if (POW == 2)
            term = -v.w * nm * (ri0 * ri0) * (rik * rik);
        else
            term = -v.w * nm * ri0 * rik * __fdividef(1.0f, r02 * ri0 + rk2 * rik);
    } else {
        if (inK) term += POW == 2 ? v.w * rik * rik : v.w * rik;
        if (inR) term -= POW == 2 ? v.w * ri0 * ri0 : v.w * ri0;
    }
    return term;
}

// The direct terms of one source x of the middle slab (seen by r and every
// charge) close to r, added to gs[k] for the m charges: rare, kept out of line.
template <int POW>
__device__ __noinline__ void sd_direct_terms(const float4 v, int ux, int uy, int uz, float d0x, float d0y, float d0z,
                                             float r02, float ri0, int m, const float *kq, const int *ks, float *gs) {
    for (int k = 0; k < m; k++)
        atomicAdd(&gs[k], sd_pair_term<POW>(v, ux, uy, uz, d0x, d0y, d0z, r02, ri0, true, kq + 12 * k, ks[k]));
}

// Series terms of one source for a point s = r + h |x - r| e_a on the split
// axis a: 1/|s - x|^POW = sum_n h^n c_n(mu) / |x - r|^POW, mu = (x - r)_a /
// |x - r| (the generating functions of the Legendre polynomials P_n for 1/r
// and of the Chebyshev polynomials U_n of the second kind for 1/r^2).  With h
// = delta / rho: t_n = q c_n(mu) / rho^(n + POW), and 1/|s - x|^POW = sum_n
// delta^n t_n / q.  da = (x - r)_a, ri = 1/rho.
template <int POW>
__device__ __forceinline__ void sd_series_terms(float q, float da, float ri, float (&t)[SD_NM]) {
    const float mu = da * ri;
    float c[SD_NM];
    c[0] = 1.0f;
    c[1] = POW == 2 ? 2.0f * mu : mu;
#pragma unroll
    for (int k = 2; k < SD_NM; k++)
        c[k] = POW == 2 ? fmaf(2.0f * mu, c[k - 1], -c[k - 2])
                        : fmaf((float)(2 * k - 1) / (float)k * mu, c[k - 1], -(float)(k - 1) / (float)k * c[k - 2]);
    float gq = POW == 2 ? q * ri * ri : q * ri;
#pragma unroll
    for (int k = 0; k < SD_NM; k++) {
        t[k] = gq * c[k];
        gq *= ri;
    }
}

// Direct terms of a source of an outer slab closer to r than the series
// allows (only with split widths well above the default): u = -1 (set 0): the
// charges below the plane see it with r, a difference term each (r's plain
// term stays in the slab's M_0); u = 2 (set 2): the charges above the plane
// alone see it, a plain term each, in double precision.
template <int POW>
__device__ __noinline__ void sd_direct_outer(const float4 v, int ux, int uy, int uz, float d0x, float d0y, float d0z,
                                             float r02, float ri0, int set, int a1, int m, const float *kq,
                                             const int *ks, float *gs, double *gsd) {
    for (int k = 0; k < m; k++) {
        const int sk = ks[k];
        const bool upk = (sk >> a1) & 1;
        if (set == 0 && !upk) {
            atomicAdd(&gs[k], sd_pair_term<POW>(v, ux, uy, uz, d0x, d0y, d0z, r02, ri0, true, kq + 12 * k, sk));
        } else if (set == 2 && upk) {
            const float *kk = kq + 12 * k;
            const int sh[3] = {ux - (sk & 1), uy - ((sk >> 1) & 1), uz - (sk >> 2)};
            const float vv[3] = {v.x, v.y, v.z};
            double r2 = 0.0;
            for (int a = 0; a < 3; a++) {
                const double d = ((double)vv[a] + (double)sh[a]) - ((double)kk[3 + a] + (double)kk[6 + a]);
                r2 += d * d;
            }
            if (r2 > 0.0) atomicAdd(&gsd[k], POW == 2 ? (double)v.w / r2 : (double)v.w / sqrt(r2));
        }
    }
}

// The offset u (each in -1..2) of cell c of the neighbour table whose axis o2
// varies slowest, then o1, then o0 (extents n0, n1).
__device__ __forceinline__ void sd_cell_offset(int c, int o0, int o1, int n0, int n1, int &ux, int &uy, int &uz) {
    const int a = c % n0 - 1, b = (c / n0) % n1 - 1, d = c / (n0 * n1) - 1;
    ux = o0 == 0 ? a : (o1 == 0 ? b : d);
    uy = o0 == 1 ? a : (o1 == 1 ? b : d);
    uz = o0 == 2 ? a : (o1 == 2 ? b : d);
}

template <int POW, int CH>
struct KSplitDelta {
    static constexpr int BS = 32 * SD_WARPS, MINB = 5;
    Geom g;
    Coef<double> Cd;
    int n;
    const float *__restrict__ pos;
    const int *__restrict__ count;
    const int *__restrict__ offset;
    const int *__restrict__ leaf_start;
    const float4 *__restrict__ s_pt;
    const int *__restrict__ s_origin;
    const float *__restrict__ loc_leaf;
    float *__restrict__ delta;
    const int *__restrict__ slist;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        // double-precision weights: every distinct coordinate of the particle's
        // charges (axis a, entry e) for a particle split along several axes; the
        // per-axis rows and weight differences for one split axis (carved below)
        __shared__ double wsm[SD_WARPS][3][FMM_MAXP + 1][FMM_MAXP];
        __shared__ int csm[SD_WARPS][64 + 65 + 64];        // neighbour cells: first slot, count prefix, offset
        __shared__ float ksm[SD_WARPS][SD_KMAX * 12];      // the charges (one split axis) or one chunk of them
        __shared__ int ssm[SD_WARPS][SD_KMAX];             // their sides (bit a: the upper cell of axis a)
        __shared__ float gsm[SD_WARPS][SD_KMAX];           // near-source terms per charge (one split axis)
        __shared__ double gsd[SD_WARPS][SD_KMAX];          // plain near-source terms per charge (outer slab)
        __shared__ float msm[SD_WARPS][2][SD_NMOM];        // the moments (high, low) per slab and order
        __shared__ float csum[SD_WARPS][2][CH][32];        // per-lane compensated sums per charge (several axes)
        const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
        const int S = g.S, p = g.p, p3 = g.p3;
        constexpr int PM = CH;  // p <= PM: the launch picks CH = 4, 6 or 8 by p
        const int n1 = slist[0], nmul = slist[1];
        const int m1 = p + (p & 1);
        const int nchm = (m1 * m1 * m1 + CH - 1) / CH;  // chunks of a particle split along several axes, at most
        const long long ntask = (long long)nmul * nchm + n1;
        // persistent warps over the tasks: the chunks of the particles split along
        // several axes (the longest) first, then one task per particle split along one
        for (long long tk = bid_ * SD_WARPS + wl; tk < ntask; tk += (long long)nblk_ * SD_WARPS) {
            int i, c0 = 0;
            if (tk < (long long)nmul * nchm) {
                i = slist[n + 1 - (int)(tk / nchm)];
                c0 = (int)(tk % nchm) * CH;
                if (c0 >= count[i]) continue;  // warp-uniform: past this particle's charges
            } else {
                i = slist[2 + (int)(tk - (long long)nmul * nchm)];
            }
            // the particle's axes: binned cell, split geometry, base = the lower cell
            // of each split axis (unwrapped), the binned cell otherwise
            AxisInfo A[3];
            int base[3], sp[3];
            float R[3];  // the reference point (first charge) in the base frame
#pragma unroll
            for (int a = 0; a < 3; a++) {
                int st = 0, c;
                float t;
                bin_axis(g, pos[3 * i + a], a, t, c, st);
                A[a] = split_axis_info(g, c, t);
                sp[a] = A[a].mode != 0;
                base[a] = A[a].mode == 1 ? c - 1 : c;
                R[a] = sp[a] ? 1.0f - g.dtf : t;  // node plane - d: exact in single precision
            }
            const int m = A[0].m * A[1].m * A[2].m, e0 = offset[i];
            const int a1 = sp[0] + sp[1] + sp[2] == 1 ? (sp[0] ? 0 : (sp[1] ? 1 : 2)) : -1;  // the one split axis
            // the neighbour table: the cells adjacent to any of the particle's cells,
            // resolved once by all lanes (first sorted slot, prefix of the charge
            // counts, offset u from the base cell packed 3 x 4 bits); with one split
            // axis it varies slowest, so that its slabs u = -1, 0..1, 2 are
            // contiguous (cells 0..8, 9..26, 27..35)
            int o0 = 0, o1 = 1;
            if (a1 == 0) {
                o0 = 1;
                o1 = 2;
            } else if (a1 == 1) {
                o1 = 2;
            }
            const int nd0 = 3 + sp[o0], nd1 = 3 + sp[o1];
            const int nc = (3 + sp[0]) * (3 + sp[1]) * (3 + sp[2]);
            int *cst = csm[wl], *cpre = cst + 64, *cpk = cpre + 65;
            {
                int cnt_lane[2] = {0, 0};
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int c = lane + 32 * h;
                    if (c < nc) {
                        int ux, uy, uz;
                        sd_cell_offset(c, o0, o1, nd0, nd1, ux, uy, uz);
                        int gx = base[0] + ux, gy = base[1] + uy, gz = base[2] + uz;
                        bool in = true;
                        if (g.periodic) {
                            gx = (gx + S) % S;
                            gy = (gy + S) % S;
                            gz = (gz + S) % S;
                        } else {
                            in = gx >= 0 && gy >= 0 && gz >= 0 && gx < S && gy < S && gz < S;
                        }
                        int a0 = 0, cc = 0;
                        if (in) {
                            const uint32_t key = morton_encode(gx, gy, gz);
                            a0 = leaf_start[key];
                            cc = leaf_start[key + 1] - a0;
                        }
                        cst[c] = a0;
                        cpk[c] = (ux + 1) | ((uy + 1) << 4) | ((uz + 1) << 8);
                        cnt_lane[h] = cc;
                    }
                }
                // prefix of the counts over the (up to 64) cells
                int inc0 = cnt_lane[0], inc1 = cnt_lane[1];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y0 = __shfl_up_sync(0xffffffffu, inc0, o), y1 = __shfl_up_sync(0xffffffffu, inc1, o);
                    if (lane >= o) {
                        inc0 += y0;
                        inc1 += y1;
                    }
                }
                const int tot0 = __shfl_sync(0xffffffffu, inc0, 31);
                if (lane < nc) cpre[lane + 1] = inc0;
                if (lane + 32 < nc) cpre[lane + 33] = tot0 + inc1;
                if (lane == 0) cpre[0] = 0;
            }
            const float Sp = POW == 2 ? (float)S * (float)S : (float)S;  // cell units to unit-box units
            if (a1 >= 0) {
                // ---- one split axis a1: the m <= SD_KMAX charges in one pass ----
                const int ob = o0, oc = o1;  // the other two axes
                // W_a1 at r (lower cell), W_ob and W_oc at the particle; per charge
                // W_a1(s_k) - W_a1 at its cell's point: r below the plane, the plane
                // itself above (t = 0 of the upper cell, the first node: weights e_0)
                double *wr = &wsm[wl][0][0][0];
                double *wb = wr + FMM_MAXP, *wc = wb + FMM_MAXP;
                float *dw = reinterpret_cast<float *>(wc + FMM_MAXP);
                float *kq = ksm[wl], *gs = gsm[wl];
                int *ks = ssm[wl];
                int sidek = 0;
                double t = 0.0;  // lane k < m: charge k along a1; 16: r along a1; 17, 18: the other axes
                if (lane < m) {  // charge k = lane: entry k of a1, entry 0 of the other axes
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        int side;
                        float th, tl, tfk;
                        split_entry_df(g, A[a], a == a1 ? lane : 0, side, th, tl, tfk);
                        // s_k - r: th - r exact (Sterbenz) below the plane, r = 1 - dt
                        const float dd = !sp[a] ? 0.0f : (side ? __fadd_rn(th, g.dtf) : __fsub_rn(th, R[a]));
                        kq[lane * 12 + a] = dd + tl;
                        kq[lane * 12 + 3 + a] = th;
                        kq[lane * 12 + 6 + a] = tl;
                        kq[lane * 12 + 9 + a] = tfk;
                        sidek |= side << a;
                        if (a == a1) t = (double)th + (double)tl;
                    }
                    ks[lane] = sidek;
                    gs[lane] = 0.0f;
                    gsd[wl][lane] = 0.0;
                } else if (lane >= 16 && lane < 19) {
                    const int a = lane == 17 ? ob : (lane == 18 ? oc : a1);
                    int side;
                    float th, tl, tfk;
                    split_entry_df(g, A[a], 0, side, th, tl, tfk);
                    t = (double)th + (double)tl;
                }
                {
                    double w[PM];
                    lag_weights<double, PM>(Cd, p, t, w);  // one pass for all lanes
                    if (lane >= 16 && lane < 19) {
                        double *dst = lane == 16 ? wr : (lane == 17 ? wb : wc);
#pragma unroll
                        for (int k = 0; k < PM; k++)
                            if (k < p) dst[k] = w[k];
                    }
                    __syncwarp();
                    if (lane < m) {
                        const bool upk = (sidek >> a1) & 1;
#pragma unroll
                        for (int k = 0; k < PM; k++)
                            if (k < p) dw[lane * FMM_MAXP + k] = (float)(w[k] - (upk ? (k == 0 ? 1.0 : 0.0) : wr[k]));
                    }
                }
                __syncwarp();
                // far field along the lines of a1 (one per node pair of ob, oc):
                // charge k: (W_a1(s_k) - W_a1(its cell's point)) W_ob W_oc . L of its
                // cell in single precision (the difference is small and carries its
                // own rounding only); X = g(plane) . L_upper - g(r) . L_lower in
                // double precision, the same for every upper charge (g(plane) is
                // e_0 along a1)
                const int sa = a1 == 0 ? 1 : (a1 == 1 ? p : p * p);
                const int sb = ob == 0 ? 1 : (ob == 1 ? p : p * p), sc = oc == 0 ? 1 : (oc == 1 ? p : p * p);
                const int64_t cl = loc_cell(g.depth, (base[0] + S) % S, (base[1] + S) % S, (base[2] + S) % S);
                const int64_t cu = loc_cell(g.depth, (base[0] + (a1 == 0) + S) % S, (base[1] + (a1 == 1) + S) % S,
                                            (base[2] + (a1 == 2) + S) % S);
                float fk[PM];  // m <= p + (p & 1) <= PM charges
#pragma unroll
                for (int k = 0; k < PM; k++) fk[k] = 0.0f;
                double X = 0.0;
                for (int ln = lane; ln < p * p; ln += 32) {
                    const int jb = ln % p, jc = ln / p;
                    const float *Ll = loc_leaf + cl * p3 + jb * sb + jc * sc, *Lu = loc_leaf + cu * p3 + jb * sb + jc * sc;
                    float L0[PM], L1[PM];
                    double xs = 0.0;
#pragma unroll
                    for (int a = 0; a < PM; a++) {
                        L0[a] = a < p ? Ll[a * sa] : 0.0f;
                        L1[a] = a < p ? Lu[a * sa] : 0.0f;
                        if (a < p) xs -= wr[a] * (double)L0[a];
                    }
                    const double wbc = wb[jb] * wc[jc];
                    X += wbc * (xs + (double)L1[0]);
                    const float fbc = (float)wbc;
#pragma unroll
                    for (int k = 0; k < PM; k++) {
                        if (k < m) {
                            const bool upk = (ks[k] >> a1) & 1;
                            const float *d = dw + k * FMM_MAXP;
                            float s = 0.0f;
#pragma unroll
                            for (int a = 0; a < PM; a++)
                                if (a < p) s = fmaf(d[a], upk ? L1[a] : L0[a], s);
                            fk[k] = fmaf(fbc, s, fk[k]);
                        }
                    }
                }
                float myf = 0.0f;
#pragma unroll
                for (int k = 0; k < PM; k++) {
                    if (k < m) {
                        float v = fk[k];
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (lane == k) myf = v;
                    }
                }
                for (int o = 16; o > 0; o >>= 1) X += __shfl_xor_sync(0xffffffffu, X, o);
                // near field, three slabs of the table along a1: u = -1 (seen by r and
                // the lower charges), 0..1 (seen by all), 2 (seen by the upper
                // charges).  Sources closer to r than 16 max|delta|: direct terms per
                // charge (gs; with the default split width only middle-slab sources
                // are that close); all others: series moments, which truncated after
                // h^6 leave h^7 < 4e-9 of each term (8 h^7 for 1/r^2)
                float far2 = 0.0f;
#pragma unroll
                for (int k = 0; k < PM; k++)
                    if (k < m) far2 = fmaxf(far2, 256.0f * kq[k * 12 + a1] * kq[k * 12 + a1]);
                bool outer_direct = false;
#pragma unroll 1
                for (int set = 0; set < 3; set++) {
                    const int cb = set == 0 ? 0 : (set == 1 ? 9 : 27), ce = set == 0 ? 9 : (set == 1 ? 27 : 36);
                    const int fe = cpre[ce];
                    // one source: its series terms t (zero where it is skipped or taken
                    // directly; r's plain term of the slab u = -1 is kept in its M_0 for
                    // every source; direct sources of the outer slabs are taken after
                    // the three slabs)
                    auto source = [&](const float4 &v, int pk, bool ok, float(&t)[SD_NM]) {
                        const int ux = (pk & 15) - 1, uy = ((pk >> 4) & 15) - 1, uz = (pk >> 8) - 1;
                        // x - r (the reference is exact in single precision, side 0)
                        const float d0x = sd_axis_diff(v.x, ux, R[0], 0.0f), d0y = sd_axis_diff(v.y, uy, R[1], 0.0f),
                                    d0z = sd_axis_diff(v.z, uz, R[2], 0.0f);
                        const float r02 = d0x * d0x + d0y * d0y + d0z * d0z;
                        const float ri0 = r02 > 0.0f ? rsqrtf(r02) : 0.0f;
                        const bool direct = r02 <= far2;
                        if (ok && direct) {
                            if (set == 1)
                                sd_direct_terms<POW>(v, ux, uy, uz, d0x, d0y, d0z, r02, ri0, m, kq, ks, gs);
                            else
                                outer_direct = true;  // taken after the slabs
                        }
                        sd_series_terms<POW>(ok && !direct ? v.w : 0.0f, a1 == 0 ? d0x : (a1 == 1 ? d0y : d0z), ri0, t);
                        if (set == 0 && ok && direct) t[0] = POW == 2 ? v.w * ri0 * ri0 : v.w * ri0;
                    };
                    float acc[SD_NM], cmp[SD_NM];
#pragma unroll
                    for (int k = 0; k < SD_NM; k++) acc[k] = cmp[k] = 0.0f;
                    // two sources per lane and step (f and f + 32), loaded together
                    int c = cb, c2 = cb;
                    for (int f = cpre[cb] + lane; f < fe; f += 64) {
                        while (cpre[c + 1] <= f) c++;
                        const int f2 = f + 32;
                        const bool ok2 = f2 < fe;
                        if (ok2) {
                            c2 = max(c2, c);
                            while (cpre[c2 + 1] <= f2) c2++;
                        }
                        const int j = cst[c] + (f - cpre[c]);
                        const int j2 = ok2 ? cst[c2] + (f2 - cpre[c2]) : j;
                        const int og1 = s_origin[j], og2 = s_origin[j2];
                        const float4 v1 = s_pt[j], v2 = s_pt[j2];
                        float t1[SD_NM], t2[SD_NM];
                        source(v1, cpk[c], og1 != i, t1);
                        source(v2, cpk[c2], ok2 && og2 != i, t2);
#pragma unroll
                        for (int k = 0; k < SD_NM; k++) {  // compensated sums
                            const float y = (t1[k] + t2[k]) - cmp[k], tt = acc[k] + y;
                            cmp[k] = (tt - acc[k]) - y;
                            acc[k] = tt;
                        }
                    }
                    // over the lanes: the moments n >= 1 in single precision (each lane's
                    // compensated sum rounded once); n = 0 (used where the two points see
                    // different slabs, and cancelling there) as pairs
                    float h0 = acc[0], l0 = -cmp[0];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
                        sd_two_sum(h0, l0, __shfl_xor_sync(0xffffffffu, h0, o), __shfl_xor_sync(0xffffffffu, l0, o));
#pragma unroll
                    for (int k = 1; k < SD_NM; k++) {
                        float v = acc[k] - cmp[k];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        acc[k] = v;
                    }
                    if (lane == 0) {
                        msm[wl][0][set * SD_NM] = h0;
                        msm[wl][1][set * SD_NM] = l0;
#pragma unroll
                        for (int k = 1; k < SD_NM; k++) {
                            msm[wl][0][set * SD_NM + k] = acc[k];
                            msm[wl][1][set * SD_NM + k] = 0.0f;
                        }
                    }
                }
                if (__any_sync(0xffffffffu, outer_direct)) {
                    // sources of the outer slabs closer to r than the series allows (split
                    // widths well above the default): their direct terms
                    for (int set = 0; set < 3; set += 2) {
                        const int fb = cpre[set == 0 ? 0 : 27], fe = cpre[set == 0 ? 9 : 36];
                        int c = set == 0 ? 0 : 27;
                        for (int f = fb + lane; f < fe; f += 32) {
                            while (cpre[c + 1] <= f) c++;
                            const int j = cst[c] + (f - cpre[c]);
                            if (s_origin[j] == i) continue;
                            const float4 v = s_pt[j];
                            const int pk = cpk[c], ux = (pk & 15) - 1, uy = ((pk >> 4) & 15) - 1, uz = (pk >> 8) - 1;
                            const float d0x = sd_axis_diff(v.x, ux, R[0], 0.0f), d0y = sd_axis_diff(v.y, uy, R[1], 0.0f),
                                        d0z = sd_axis_diff(v.z, uz, R[2], 0.0f);
                            const float r02 = d0x * d0x + d0y * d0y + d0z * d0z;
                            if (r02 > far2) continue;
                            const float ri0 = r02 > 0.0f ? rsqrtf(r02) : 0.0f;
                            sd_direct_outer<POW>(v, ux, uy, uz, d0x, d0y, d0z, r02, ri0, set, a1, m, kq, ks, gs, gsd[wl]);
                        }
                    }
                }
                __syncwarp();
                if (lane < m) {
                    // D_k = sum_{n>=1} delta^n (M_n of the middle slab + of the slab only
                    // this side sees besides it) + direct terms + far difference; an upper
                    // charge adds M_0(u = 2) - M_0(u = -1) + X, which cancel to a small
                    // number: that sum in double precision
                    const float dk = kq[lane * 12 + a1];
                    const bool up = (sidek >> a1) & 1;
                    const float *MH = msm[wl][0], *ML = msm[wl][1];
                    const int o = up ? 2 * SD_NM : 0;  // the other slab: u = 2 above the plane, u = -1 below
                    float s = 0.0f;
#pragma unroll
                    for (int k = SD_NM - 1; k >= 1; k--)
                        s = (s + ((MH[SD_NM + k] + ML[SD_NM + k]) + (MH[o + k] + ML[o + k]))) * dk;
                    const double zs = (up ? (double)Sp * (((double)MH[2 * SD_NM] + (double)ML[2 * SD_NM]) -
                                                          ((double)MH[0] + (double)ML[0])) + X
                                          : 0.0) +
                                      (double)Sp * gsd[wl][lane];
                    delta[e0 + lane] = (float)((double)(Sp * (s + gs[lane]) + myf) + zs);
                }
            } else {
                // ---- several split axes: charges c0 .. c0 + CH - 1, direct terms ----
                double(*W)[FMM_MAXP + 1][FMM_MAXP] = wsm[wl];
                {  // weights: lane = a * 8 + e computes entry e of axis a
                    const int a = lane >> 3, e = lane & 7;
                    if (a < 3 && e < A[a].m) {
                        int side;
                        float th, tl, tfl;
                        split_entry_df(g, A[a], e, side, th, tl, tfl);
                        double w[PM];
                        lag_weights<double, PM>(Cd, p, (double)th + (double)tl, w);
#pragma unroll
                        for (int k = 0; k < PM; k++)
                            if (k < p) W[a][e][k] = w[k];
                    }
                }
                __syncwarp();
                double far0 = 0.0;  // far field at the reference point (entry 0 of every axis)
                {
                    const int64_t cr = loc_cell(g.depth, (base[0] + S) % S, (base[1] + S) % S, (base[2] + S) % S);
                    for (int o = lane; o < p3; o += 32)
                        far0 += W[0][0][o % p] * W[1][0][(o / p) % p] * W[2][0][o / (p * p)] * (double)loc_leaf[cr * p3 + o];
                }
                for (int o = 16; o > 0; o >>= 1) far0 += __shfl_xor_sync(0xffffffffu, far0, o);
                float *kq = ksm[wl];  // per charge of the chunk: s_k - r (3), th (3), tl (3), tf (3)
                int *ks = ssm[wl];    // and its sides
                double fdk = 0.0;     // lane k: the far-field difference of charge c0 + k
#pragma unroll 1
                for (int k = 0; k < CH; k++) {
                    int le = min(c0 + k, m - 1);
                    const int ex = le % A[0].m;
                    le /= A[0].m;
                    const int e3[3] = {ex, le % A[1].m, le / A[1].m};
                    int side[3];
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        float th, tl, tfk;
                        split_entry_df(g, A[a], e3[a], side[a], th, tl, tfk);
                        if (lane == k) {
                            const float dd = !sp[a] ? 0.0f : (side[a] ? __fadd_rn(th, g.dtf) : __fsub_rn(th, R[a]));
                            kq[k * 12 + a] = dd + tl;
                            kq[k * 12 + 3 + a] = th;
                            kq[k * 12 + 6 + a] = tl;
                            kq[k * 12 + 9 + a] = tfk;
                            ks[k] = side[0] | (side[1] << 1) | (side[2] << 2);
                        }
                    }
                    const int64_t ck = loc_cell(g.depth, (base[0] + side[0] + S) % S, (base[1] + side[1] + S) % S,
                                                (base[2] + side[2] + S) % S);
                    double f = 0.0;
                    for (int o = lane; o < p3; o += 32)
                        f += W[0][e3[0]][o % p] * W[1][e3[1]][(o / p) % p] * W[2][e3[2]][o / (p * p)] *
                             (double)loc_leaf[ck * p3 + o];
                    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
                    if (lane == k) fdk = f - far0;
                    csum[wl][0][k][lane] = 0.0f;  // this lane's compensated sums for the charge
                    csum[wl][1][k][lane] = 0.0f;
                }
                __syncwarp();
                // two sources per lane and step (f and f + 32), loaded together
                const int nsrc = cpre[nc];
                int c = 0, c2 = 0;
                for (int f = lane; f < nsrc; f += 64) {
                    while (cpre[c + 1] <= f) c++;
                    const int f2 = f + 32;
                    const bool ok2 = f2 < nsrc;
                    if (ok2) {
                        c2 = max(c2, c);
                        while (cpre[c2 + 1] <= f2) c2++;
                    }
                    const int j = cst[c] + (f - cpre[c]);
                    const int j2 = ok2 ? cst[c2] + (f2 - cpre[c2]) : j;
                    const int og1 = s_origin[j], og2 = s_origin[j2];
                    const float4 v1 = s_pt[j], v2 = s_pt[j2];
#pragma unroll 1
                    for (int h = 0; h < 2; h++) {
                        if (h == 0 ? og1 == i : (!ok2 || og2 == i)) continue;
                        const float4 v = h == 0 ? v1 : v2;
                        const int pk = cpk[h == 0 ? c : c2], ux = (pk & 15) - 1, uy = ((pk >> 4) & 15) - 1,
                                  uz = (pk >> 8) - 1;
                        const bool inR = ux <= 1 && uy <= 1 && uz <= 1;
                        const float d0x = sd_axis_diff(v.x, ux, R[0], 0.0f), d0y = sd_axis_diff(v.y, uy, R[1], 0.0f),
                                    d0z = sd_axis_diff(v.z, uz, R[2], 0.0f);
                        const float r02 = d0x * d0x + d0y * d0y + d0z * d0z;
                        const float ri0 = r02 > 0.0f ? rsqrtf(r02) : 0.0f;
#pragma unroll 1
                        for (int k = 0; k < CH; k++) {
                            const float term = sd_pair_term<POW>(v, ux, uy, uz, d0x, d0y, d0z, r02, ri0, inR, kq + k * 12, ks[k]);
                            const float ak = csum[wl][0][k][lane], ck = csum[wl][1][k][lane];
                            const float y = term - ck, tt = ak + y;  // compensated sum
                            csum[wl][1][k][lane] = (tt - ak) - y;
                            csum[wl][0][k][lane] = tt;
                        }
                    }
                }
                double vk = 0.0;
#pragma unroll 1
                for (int k = 0; k < CH; k++) {
                    double v = (double)csum[wl][0][k][lane] - (double)csum[wl][1][k][lane];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == k) vk = v;
                }
                if (lane < CH && c0 + lane < m) delta[e0 + c0 + lane] = (float)((double)Sp * vk + fdk);
            }
            __syncwarp();  // the tables are rewritten by the next task
        }
    }
};
template <int POW, int CH>
__global__ void __launch_bounds__(KSplitDelta<POW, CH>::BS, KSplitDelta<POW, CH>::MINB) k_split_delta(const __grid_constant__ KSplitDelta<POW, CH> k) {
    k.run(blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// recombination of the split charges into their particles (§2.3), scaling to
// physical units, and the FP64 energy E = 1/2 sum_i q_i phi_i.
//   phi_i = sum_k W_k phi(s_k)
//   adjoint force, axis not split: sum_k F(s_k); split axis: -q_i sum_k dW_k/du phi(s_k)
//   paper force: sum_k F(s_k) on every axis
// out_e holds (phi, F) per emitted charge in unit-box units: the charges of
// particle i are read in a row, [offset[i], offset[i+1]) (i itself in the
// plain form).
// backward: grad_pos = -F * gE, grad_q = phi * gE.
// ---------------------------------------------------------------------------
#define UNSPLIT_BS 256

// Error-free transformations (Dekker, Knuth): a*b = p + fma_exact_err(a, b, p)
// exactly; pair_add adds (bh, bl) to the pair (ah, al) with the rounding error
// of the high parts carried in the low part.  In double precision these are
// ordinary double operations.
__device__ __forceinline__ float fma_exact_err(float a, float b, float p) { return fmaf(a, b, -p); }
__device__ __forceinline__ double fma_exact_err(double a, double b, double p) { return fma(a, b, -p); }
template <typename real>
__device__ __forceinline__ void pair_add(real &ah, real &al, real bh, real bl) {
    const real s = ah + bh;
    const real v = s - ah;
    const real e = (ah - (s - v)) + (bh - v);
    const real t = e + al + bl;
    ah = s + t;
    al = t - (ah - s);
}

template <typename real>
struct KUnsplit {
    static constexpr int BS = 0, MINB = 0;
    Geom g;
    const WsHeader *hdr;
    int n;
    const float *__restrict__ q;
    const int *__restrict__ offset;
    const int *__restrict__ count;
    const unsigned char *__restrict__ axes;
    const typename Vec4<real>::T *__restrict__ e_wd;
    const typename Vec4<real>::T *__restrict__ out_e;
    const float *__restrict__ delta;
    real *__restrict__ potential;
    real *__restrict__ forces;
    real *__restrict__ epart;
    const double *__restrict__ grad_energy;
    real *__restrict__ grad_q;
    int backward;
    real sphi;
    real sF;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        // sphi = 1/L and sF = 1/L^2 come from the host: no FP64 arithmetic per thread
        __shared__ real sh[UNSPLIT_BS / 32][2];
        double gE = backward ? *grad_energy : 0.0;
        real ehi = 0, elo = 0;
        int i = bid_ * blockDim.x + threadIdx.x;
        if (i < n) {
            real phi, Fx, Fy, Fz;
            if (!offset) {
                typename Vec4<real>::T o = out_e[i];
                phi = o.x;
                Fx = o.y;
                Fy = o.z;
                Fz = o.w;
            } else {
                int e0 = offset[i], m = count[i];
                if (e0 + m > hdr->n_eff) m = 0;  // not emitted (split overflow; status is set)
                phi = 0;
                real Sx = 0, Sy = 0, Sz = 0, Nx = 0, Ny = 0, Nz = 0;
                for (int e = e0; e < e0 + m; e++) {
                    typename Vec4<real>::T o = out_e[e];
                    typename Vec4<real>::T d = e_wd[e];
                    phi += d.x * o.x;
                    Sx += o.y;
                    Sy += o.z;
                    Sz += o.w;
                    // split axes: the weights' derivatives against phi(s_k), or
                    // against the differences phi(s_k) - phi(r) where they were formed
                    const real D = (delta && m > 1) ? (real)delta[e] : o.x;
                    Nx += d.y * D;
                    Ny += d.z * D;
                    Nz += d.w * D;
                }
                // paper and force-kernel forces: the sum of the split charges' forces
                unsigned ax = g.force_mode != FMM_FORCE_ADJOINT ? 0u : axes[i];
                real qi = (real)q[i];
                Fx = (ax & 1) ? -qi * Nx : Sx;
                Fy = (ax & 2) ? -qi * Ny : Sy;
                Fz = (ax & 4) ? -qi * Nz : Sz;
            }
            phi *= sphi;
            Fx *= sF;
            Fy *= sF;
            Fz *= sF;
            if (!backward) {
                if (potential) potential[i] = phi;
                if (forces) {
                    forces[3 * i] = Fx;
                    forces[3 * i + 1] = Fy;
                    forces[3 * i + 2] = Fz;
                }
                ehi = (real)q[i] * phi;  // q phi exactly as ehi + elo (single precision)
                elo = fma_exact_err((real)q[i], phi, ehi);
            } else {
                if (forces) {
                    forces[3 * i] = (real)(-(double)Fx * gE);
                    forces[3 * i + 1] = (real)(-(double)Fy * gE);
                    forces[3 * i + 2] = (real)(-(double)Fz * gE);
                }
                if (grad_q) grad_q[i] = (real)((double)phi * gE);
            }
        }
        if (epart) {
            // deterministic block reduction of sum q phi: exact products, then
            // compensated pair sums over the warp and over the warps in order; the
            // block's sum stays a (hi, lo) pair of the working precision: no FP64
            // arithmetic here (a slow pipe on this part, which the per-block
            // conversions and adds kept busy)
            for (int o = 16; o > 0; o >>= 1) {
                const real bh = __shfl_down_sync(0xffffffffu, ehi, o);
                const real bl = __shfl_down_sync(0xffffffffu, elo, o);
                pair_add(ehi, elo, bh, bl);
            }
            if ((threadIdx.x & 31) == 0) {
                sh[threadIdx.x >> 5][0] = ehi;
                sh[threadIdx.x >> 5][1] = elo;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                real h = sh[0][0], l = sh[0][1];
                for (int w = 1; w < UNSPLIT_BS / 32; w++) pair_add(h, l, sh[w][0], sh[w][1]);
                epart[2 * bid_] = h;
                epart[2 * bid_ + 1] = l;
            }
        }
    }
};
template <typename real>
__global__ void k_unsplit(const __grid_constant__ KUnsplit<real> k) {
    k.run(blockIdx.x, gridDim.x);
}

// total energy from the blocks' (hi, lo) pairs: strided per-thread pair sums,
// warp trees, then the warps' pairs in order (fixed order: deterministic);
// E = (hi + lo) / 2 in FP64 once
template <typename real>
struct KEnergyFinal {
    static constexpr int BS = 0, MINB = 0;
    const real *__restrict__ epart;
    int nb;
    double *energy;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        __shared__ real sh[32][2];
        real h = 0, l = 0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) pair_add(h, l, epart[2 * b], epart[2 * b + 1]);
        for (int o = 16; o > 0; o >>= 1) {
            const real bh = __shfl_down_sync(0xffffffffu, h, o);
            const real bl = __shfl_down_sync(0xffffffffu, l, o);
            pair_add(h, l, bh, bl);
        }
        if ((threadIdx.x & 31) == 0) {
            sh[threadIdx.x >> 5][0] = h;
            sh[threadIdx.x >> 5][1] = l;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            real th = sh[0][0], tl = sh[0][1];
            for (int w = 1; w < (int)(blockDim.x >> 5); w++) pair_add(th, tl, sh[w][0], sh[w][1]);
            *energy = 0.5 * ((double)th + (double)tl);
        }
    }
};
template <typename real>
__global__ void k_energy_final(const __grid_constant__ KEnergyFinal<real> k) {
    k.run(blockIdx.x, gridDim.x);
}

struct KZeroEnergy {
    static constexpr int BS = 0, MINB = 0;
    double *energy;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {     *energy = 0.0;     }
};
__global__ void k_zero_energy(const __grid_constant__ KZeroEnergy k) {
    k.run(blockIdx.x, gridDim.x);
}

template <typename real>
void launch_unsplit(const Geom &g, const Ptrs<real> &P, const WsLayout &W, int n, const float *q,
                    real *potential, double *energy, real *forces, const double *grad_energy,
                    real *grad_q, bool backward, cudaStream_t st, Tracer &tr) {
    tr.begin(FMM_STAGE_UNSPLIT, st);
    if (n == 0) {
        if (energy && !backward) {
            launch_k(tr, FMM_TAG(S_ZERO_ENERGY, 0), k_zero_energy, KZeroEnergy{energy}, 1, 1, 0, st);
            tr.count();
        }
        tr.end();
        return;
    }
    int nb = (n + UNSPLIT_BS - 1) / UNSPLIT_BS;
    real *ep = (!backward && energy) ? reinterpret_cast<real *>(P.epart) : nullptr;  // [nb][2]
    // unit box -> box of edge L: potentials of 1/r^k scale by L^-k, forces by L^-(k+1)
    const double iL = 1.0 / g.L, sphi = g.power == 2 ? iL * iL : iL;
    launch_k(tr, FMM_TAG(S_UNSPLIT, 0), k_unsplit<real>,
             KUnsplit<real>{g, P.hdr, n, q, g.continuous ? P.offset : nullptr, P.count, P.axes,
                            g.continuous ? P.e_wd : nullptr, P.out_e,
                            (std::is_same<real, float>::value && g.continuous && g.force_mode == FMM_FORCE_ADJOINT)
                                ? P.delta
                                : nullptr,
                            potential, forces, ep, grad_energy, grad_q, backward ? 1 : 0, (real)sphi,
                            (real)(sphi * iL)},
             nb, UNSPLIT_BS, 0, st);
    tr.count();
    if (ep) {
        launch_k(tr, FMM_TAG(S_ENERGY_FINAL, 0), k_energy_final<real>, KEnergyFinal<real>{ep, nb, energy}, 1, 1024,
                 0, st);
        tr.count();
    }
    tr.end();
}

void launch_split_delta(const Geom &g, const Coef<double> &Cd, const Ptrs<float> &P, const WsLayout &W, int n,
                        const float *pos, cudaStream_t st, Tracer &tr) {
    if (n <= 0) return;
    tr.begin(FMM_STAGE_UNSPLIT, st);
    zero_words(tr, FMM_TAG(S_ZERO_SLIST, 0), P.slist, 8, st);
    launch_k(tr, FMM_TAG(S_SPLIT_LIST, 0), k_split_list,
             KSplitList{n, g.p + (g.p & 1), P.count, P.offset, P.hdr, P.slist}, (n + 255) / 256, 256, 0, st);
    tr.count();
    // persistent: five CTAs per SM, fewer for small systems (a few percent of
    // the particles are split; the loop takes any number of tasks)
    const int nb = (int)std::min<int64_t>(152 * 5, std::max<int64_t>(1, ((int64_t)n + 63) / 64));
    const float *leaf = reinterpret_cast<const float *>(P.loc) + W.loc_level[g.depth];
    // charges per pass of a particle split along several axes
    const int ch = g.p <= 4 ? 4 : (g.p <= 6 ? 6 : 8);
#define SD_LAUNCH(POW, CH)                                                                                  \
    launch_k(tr, FMM_TAG(S_SPLIT_DELTA, 0), k_split_delta<POW, CH>,                                             \
             KSplitDelta<POW, CH>{g, Cd, n, pos, P.count, P.offset, P.leaf_start, P.s_pt, P.s_origin, leaf, P.delta, \
                                  P.slist},                                                                     \
             nb, 32 * SD_WARPS, 0, st)
    if (g.power == 2) {
        if (ch == 4) SD_LAUNCH(2, 4); else if (ch == 6) SD_LAUNCH(2, 6); else SD_LAUNCH(2, 8);
    } else {
        if (ch == 4) SD_LAUNCH(1, 4); else if (ch == 6) SD_LAUNCH(1, 6); else SD_LAUNCH(1, 8);
    }
#undef SD_LAUNCH
    tr.count();
    tr.end();
}

#define INST(real)                                                                               \
    template void launch_bin_emit<real>(const Geom &, const Coef<real> &, const Ptrs<real> &,     \
                                        const WsLayout &, int, const float *, const float *,      \
                                        cudaStream_t, Tracer &);                                  \
    template void launch_sort<real>(const Geom &, const Ptrs<real> &, const WsLayout &, int,      \
                                    cudaStream_t, Tracer &);                                      \
    template void launch_unsplit<real>(const Geom &, const Ptrs<real> &, const WsLayout &, int,   \
                                       const float *, real *, double *, real *, const double *,   \
                                       real *, bool, cudaStream_t, Tracer &);
INST(float)
INST(double)

}  // namespace fmm

// Binning, split, stable sort by finest cell, recombination of split charges
// and the FP64 energy reduction.
#include <type_traits>

#include "fmm_internal.cuh"
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
__global__ void k_emit(Geom g, Coef<real> C, int n, const float *__restrict__ pos,
                       const float *__restrict__ q, const int *__restrict__ offset,
                       uint32_t *__restrict__ e_key, typename Vec4<real>::T *__restrict__ e_pt,
                       typename Vec4<real>::T *__restrict__ e_wd, int *__restrict__ e_origin,
                       int *__restrict__ e_rank, int *__restrict__ leaf_count, WsHeader *hdr) {
    int st = 0;
    const int ne = offset ? hdr->n_eff : n;
    if (!offset && blockIdx.x == 0 && threadIdx.x == 0) hdr->n_eff = n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
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

__global__ void k_scan_reduce(const int *__restrict__ in, int m, int *__restrict__ bsum) {
    __shared__ int sh[32];
    int base = blockIdx.x * SCAN_TILE;
    int s = 0;
    for (int k = 0; k < SCAN_IPT; k++) {
        int i = base + k * SCAN_BS + threadIdx.x;
        if (i < m) s += in[i];
    }
    int tot;
    block_excl_scan(s, sh, tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// first pass over the particles (continuous form): charges per particle and
// split axes (§2.3), written out and summed per block
__global__ void k_split_count_reduce(Geom g, int n, const float *__restrict__ pos, int *__restrict__ count,
                                     unsigned char *__restrict__ axes, int *__restrict__ bsum,
                                     WsHeader *hdr) {
    __shared__ int sh[32];
    const int base = blockIdx.x * SCAN_TILE;
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
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
    if (st) atomicOr(&hdr->status, st);
}

__global__ void k_scan_blocks(int *bsum, int nb) {
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
__global__ void __launch_bounds__(SCAN_BS) k_scan_apply(const int *__restrict__ in, int m, const int *__restrict__ bsum,
                                                        int *__restrict__ out, int cap, int *__restrict__ e_origin,
                                                        WsHeader *hdr) {
    __shared__ int sh[32];
    constexpr int IT = SCAN_TILE / SCAN_BS / 4;
    const int base = blockIdx.x * SCAN_TILE;
    int4 v[IT];
    int pre[IT];
    int tot;
    tile_scan<IT>(in, base, m, v, pre, sh, tot);
    const int carry = bsum[blockIdx.x];
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
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        const int total = bsum[gridDim.x];
        out[m] = total;
        if (MARK && total <= cap) hdr->n_eff = total;
    }
}

// m <= SCAN1_MAX: the whole array is one tile of the CTA
__global__ void __launch_bounds__(SCAN1_BS) k_scan_one(const int *__restrict__ in, int m, int *__restrict__ out) {
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

int launch_scan(const int *in, int *out, int m, int *tmp, cudaStream_t st) {
    if (m <= SCAN1_MAX) {
        k_scan_one<<<1, SCAN1_BS, 0, st>>>(in, m, out);
        return 1;
    }
    int nb = (m + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_reduce<<<nb, SCAN_BS, 0, st>>>(in, m, tmp);
    k_scan_blocks<<<1, 1024, 0, st>>>(tmp, nb);
    k_scan_apply<false><<<nb, SCAN_BS, 0, st>>>(in, m, tmp, out, 0, nullptr, nullptr);
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
        k_split_count_reduce<<<nb, SCAN_BS, 0, st>>>(g, n, pos, P.count, P.axes, P.scan_tmp, P.hdr);
        k_scan_blocks<<<1, 1024, 0, st>>>(P.scan_tmp, nb);
        k_scan_apply<true><<<nb, SCAN_BS, 0, st>>>(P.count, n, P.scan_tmp, P.offset, (int)W.cap, P.e_origin,
                                                   P.hdr);
        tr.count(3);
        offset = P.offset;
    }
    int64_t ne_max = offset ? W.cap : n;
    int nbe = (int)((ne_max + 255) / 256);
    if (nbe < 1) nbe = 1;
    if (nbe > 152 * 64) nbe = 152 * 64;
    k_emit<real><<<nbe, 256, 0, st>>>(g, C, n, pos, q, offset, P.e_key, P.e_pt,
                                      g.continuous ? P.e_wd : nullptr, P.e_origin, P.e_rank,
                                      P.leaf_count, P.hdr);
    tr.count();
    tr.end();
}

// ---------------------------------------------------------------------------
// stable counting sort by finest cell: scatter to the slot of each charge's
// arrival rank in its cell, then order each cell's segment by emitted index
// (= particle order), then gather.
// ---------------------------------------------------------------------------
__global__ void k_scatter(const WsHeader *hdr, const uint32_t *__restrict__ e_key,
                          const int *__restrict__ e_rank, const int *__restrict__ leaf_start,
                          int *__restrict__ tmp) {
    int ne = hdr->n_eff;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x)
        tmp[leaf_start[e_key[e]] + e_rank[e]] = e;
}

// one warp per finest cell: rank every element of the cell's segment among
// the segment (emission indices, all distinct), and move it to its sorted
// slot: charge, origin and perm (slot -> emitted index).  Up to 64 elements
// are ranked in registers (two per lane, compared through shuffles).
template <typename real>
__global__ void k_leaf_gather(int ncell, const int *__restrict__ leaf_start, const int *__restrict__ tmp,
                              const typename Vec4<real>::T *__restrict__ e_pt,
                              const int *__restrict__ e_origin, typename Vec4<real>::T *__restrict__ s_pt,
                              int *__restrict__ s_origin, int *__restrict__ perm) {
    int lane = threadIdx.x & 31;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int nwarps = (gridDim.x * blockDim.x) >> 5;
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

template <typename real>
void launch_sort(const Geom &g, const Ptrs<real> &P, const WsLayout &W, int n, cudaStream_t st,
                 Tracer &tr) {
    int ncell = (int)W.ncell;
    tr.begin(FMM_STAGE_SORT, st);
    tr.count(launch_scan(P.leaf_count, P.leaf_start, ncell, P.scan_tmp, st));
    int nbp = (int)((W.cap + 255) / 256);
    if (nbp < 1) nbp = 1;
    if (nbp > 152 * 64) nbp = 152 * 64;
    k_scatter<<<nbp, 256, 0, st>>>(P.hdr, P.e_key, P.e_rank, P.leaf_start, P.tmp);
    int nbl = (ncell * 32 + 255) / 256;
    if (nbl > 152 * 64) nbl = 152 * 64;
    k_leaf_gather<real><<<nbl, 256, 0, st>>>(ncell, P.leaf_start, P.tmp, P.e_pt, P.e_origin, P.s_pt,
                                             P.s_origin, P.perm);
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
// directly, for split particles only: r is the particle's first charge (the
// node plane - d of every split axis, exact in single precision), s_k the
// exact node (double precision); the near-field part sums, over the sources
// both points see, q (1/|s_k - x| - 1/|r - x|) = -q n / (r0 rk (r0 + rk)) with
// n = |s_k - x|^2 - |r - x|^2 = delta . (delta - 2 (x - r)), delta = s_k - r
// (a small number with a small relative error), and the plain terms of the
// sources only one of them sees (cells adjacent to one of the two cells the
// segment crosses); the far-field part is the difference of the two points'
// functionals g(t) . L of their own cells, each evaluated in double precision.
// Same-particle and coincident charges are skipped as in the near field.
// One warp per split particle; each warp takes 32 consecutive particles.
// POW: the pair function 1/r (1) or 1/r^2 (2).
// ---------------------------------------------------------------------------

// exact node of entry e of split axis A: the side (0 lower, 1 upper cell of
// the plane; 0 for an axis that is not split) and the cell-local coordinate
__device__ __forceinline__ void split_entry_exact(const Geom &g, const AxisInfo &A, int e, int &side,
                                                  double &t, float &tf) {
    if (A.mode == 0) {
        side = 0;
        t = (double)A.t;
        tf = A.t;
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
    const double dt = (double)g.dtf, s = (double)(2 * k) / (double)(p - 1) - 1.0;
    t = half ? (side ? 0.0 : 1.0) : (side ? s * dt : 1.0 + s * dt);
    // the emitted charge's single-precision coordinate: the expression of split_entry
    const float sf = (float)(2 * k) / (float)(p - 1) - 1.0f, dtf = g.dtf;
    tf = half ? (side ? 0.0f : 1.0f) : (side ? sf * dtf : 1.0f + sf * dtf);
}

// x - s along one axis, the source x at coordinate v of a cell `shift` cells
// from the charge's cell, the charge at t = th + tl of its own cell: each case
// subtracts in the frame where the nearby operands are exact (Sterbenz)
__device__ __forceinline__ float sd_axis_diff(float v, int shift, float th, float tl) {
    const float d = shift == 1 ? v - (th - 1.0f) : (shift == -1 ? (v - 1.0f) - th : (v + (float)shift) - th);
    return d - tl;
}

#define SD_WARPS 8  // warps per CTA

template <int POW, int CH>
__global__ void __launch_bounds__(32 * SD_WARPS) k_split_delta(Geom g, Coef<double> Cd, int n, const float *__restrict__ pos,
                                                           const int *__restrict__ count, const int *__restrict__ offset,
                                                           const int *__restrict__ leaf_start,
                                                           const float4 *__restrict__ s_pt, const int *__restrict__ s_origin,
                                                           const float *__restrict__ loc_leaf, float *__restrict__ delta,
                                                           const WsHeader *hdr) {
    // double-precision weights of every distinct coordinate of the particle's
    // charges: axis a, entry e (the reference point is entry 0 of every axis)
    __shared__ double wsm[SD_WARPS][3][FMM_MAXP + 1][FMM_MAXP];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int i0 = (blockIdx.x * SD_WARPS + wl) * 32;
    if (i0 >= n) return;
    const int S = g.S, p = g.p, p3 = g.p3;
    const int n_eff = hdr->n_eff;
    const int mine = i0 + lane < n && count[i0 + lane] > 1 && offset[i0 + lane] + count[i0 + lane] <= n_eff;
    unsigned todo = __ballot_sync(0xffffffffu, mine);
    double (*W)[FMM_MAXP + 1][FMM_MAXP] = wsm[wl];
    while (todo) {
        const int i = i0 + __ffs(todo) - 1;
        todo &= todo - 1;
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
        // weights: lane = a * 8 + e computes entry e of axis a
        {
            const int a = lane >> 3, e = lane & 7;
            if (a < 3 && e < A[a].m) {
                int side;
                double t;
                float tfl;
                split_entry_exact(g, A[a], e, side, t, tfl);
                double w[FMM_MAXP];
                lag_weights<double>(Cd, p, t, w);
#pragma unroll
                for (int k = 0; k < FMM_MAXP; k++) W[a][e][k] = w[k];
            }
        }
        __syncwarp();
        double far0 = 0.0;  // far field at the reference point (entry 0 of every axis)
        {
            const int64_t cr = loc_cell(g.depth, (base[0] + S) % S, (base[1] + S) % S, (base[2] + S) % S);
            for (int o = lane; o < p3; o += 32)
                far0 += W[0][0][o % p] * W[1][0][(o / p) % p] * W[2][0][o / (p * p)] * (double)loc_leaf[cr * p3 + o];
        }
        for (int c0 = 0; c0 < m; c0 += CH) {
            // the chunk's charges: entries, sides (bit a: upper cell of axis a),
            // offset from the reference point, far-field difference
            float dl[CH][3], th[CH][3], tl[CH][3], tf[CH][3];
            int sd[CH];
            double fd[CH];
#pragma unroll
            for (int k = 0; k < CH; k++) {
                int le = min(c0 + k, m - 1);
                const int ex = le % A[0].m;
                le /= A[0].m;
                const int e3[3] = {ex, le % A[1].m, le / A[1].m};
                int side[3];
                double tk[3];
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    split_entry_exact(g, A[a], e3[a], side[a], tk[a], tf[k][a]);
                    dl[k][a] = (float)(((double)side[a] + tk[a]) - (double)R[a]);
                    th[k][a] = (float)tk[a];
                    tl[k][a] = (float)(tk[a] - (double)th[k][a]);
                }
                sd[k] = side[0] | (side[1] << 1) | (side[2] << 2);
                const int64_t ck = loc_cell(g.depth, (base[0] + side[0] + S) % S, (base[1] + side[1] + S) % S,
                                            (base[2] + side[2] + S) % S);
                double f = 0.0;
                for (int o = lane; o < p3; o += 32)
                    f += W[0][e3[0]][o % p] * W[1][e3[1]][(o / p) % p] * W[2][e3[2]][o / (p * p)] *
                         (double)loc_leaf[ck * p3 + o];
                fd[k] = f - far0;
            }
            // near field: the cells adjacent to any of the particle's cells
            float acc[CH], cmp[CH];
#pragma unroll
            for (int k = 0; k < CH; k++) acc[k] = cmp[k] = 0.0f;
            for (int uz = -1; uz <= 1 + sp[2]; uz++)
                for (int uy = -1; uy <= 1 + sp[1]; uy++)
                    for (int ux = -1; ux <= 1 + sp[0]; ux++) {
                        int gx = base[0] + ux, gy = base[1] + uy, gz = base[2] + uz;
                        if (g.periodic) {
                            gx = (gx + S) % S;
                            gy = (gy + S) % S;
                            gz = (gz + S) % S;
                        } else if (gx < 0 || gy < 0 || gz < 0 || gx >= S || gy >= S || gz >= S) {
                            continue;
                        }
                        const uint32_t key = morton_encode(gx, gy, gz);
                        const int ja = leaf_start[key], jb = leaf_start[key + 1];
                        const bool inR = ux <= 1 && uy <= 1 && uz <= 1;
                        for (int j = ja + lane; j < jb; j += 32) {
                            if (s_origin[j] == i) continue;
                            const float4 v = s_pt[j];
                            // x - r (the reference is exact in single precision, side 0)
                            const float d0x = sd_axis_diff(v.x, ux, R[0], 0.0f), d0y = sd_axis_diff(v.y, uy, R[1], 0.0f),
                                        d0z = sd_axis_diff(v.z, uz, R[2], 0.0f);
                            const float r02 = d0x * d0x + d0y * d0y + d0z * d0z;
#pragma unroll
                            for (int k = 0; k < CH; k++) {
                                const int sx = sd[k] & 1, sy = (sd[k] >> 1) & 1, sz = sd[k] >> 2;
                                const bool inK = ux >= sx - 1 && ux <= sx + 1 && uy >= sy - 1 && uy <= sy + 1 &&
                                                 uz >= sz - 1 && uz <= sz + 1;
                                // x - s_k directly, accurate also when x is close to s_k
                                const float dkx = sd_axis_diff(v.x, ux - sx, th[k][0], tl[k][0]),
                                            dky = sd_axis_diff(v.y, uy - sy, th[k][1], tl[k][1]),
                                            dkz = sd_axis_diff(v.z, uz - sz, th[k][2], tl[k][2]);
                                // coincident with the emitted charge (the single-precision
                                // positions the near field compares): skipped as there
                                const bool zk = sd_axis_diff(v.x, ux - sx, tf[k][0], 0.0f) == 0.0f &&
                                                sd_axis_diff(v.y, uy - sy, tf[k][1], 0.0f) == 0.0f &&
                                                sd_axis_diff(v.z, uz - sz, tf[k][2], 0.0f) == 0.0f;
                                // |s_k - x|^2 - |r - x|^2 = delta . (delta - 2 (x - r))
                                const float nm = dl[k][0] * (dl[k][0] - 2.0f * d0x) + dl[k][1] * (dl[k][1] - 2.0f * d0y) +
                                                 dl[k][2] * (dl[k][2] - 2.0f * d0z);
                                const float rk2 = dkx * dkx + dky * dky + dkz * dkz;
                                float term = 0.0f;
                                if (inK && inR && !zk && r02 > 0.0f && rk2 > 0.0f) {
                                    if (POW == 2) {
                                        term = -v.w * nm / (r02 * rk2);
                                    } else {
                                        const float r0 = sqrtf(r02), rk = sqrtf(rk2);
                                        term = -v.w * nm / (r0 * rk * (r0 + rk));
                                    }
                                } else {
                                    if (inK && !zk && rk2 > 0.0f) term += POW == 2 ? v.w / rk2 : v.w / sqrtf(rk2);
                                    if (inR && r02 > 0.0f) term -= POW == 2 ? v.w / r02 : v.w / sqrtf(r02);
                                }
                                const float y = term - cmp[k], tt = acc[k] + y;  // compensated sum
                                cmp[k] = (tt - acc[k]) - y;
                                acc[k] = tt;
                            }
                        }
                    }
            const double Sp = POW == 2 ? (double)S * S : (double)S;
#pragma unroll
            for (int k = 0; k < CH; k++) {
                double v = (double)acc[k] - (double)cmp[k];
                double f = fd[k];
                for (int o = 16; o > 0; o >>= 1) {
                    v += __shfl_xor_sync(0xffffffffu, v, o);
                    f += __shfl_xor_sync(0xffffffffu, f, o);
                }
                if (lane == 0 && c0 + k < m) delta[e0 + c0 + k] = (float)(Sp * v + f);
            }
        }
        __syncwarp();  // the weights table is rewritten for the next particle
    }
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
__global__ void k_unsplit(Geom g, const WsHeader *hdr, int n, const float *__restrict__ q,
                          const int *__restrict__ offset,
                          const int *__restrict__ count, const unsigned char *__restrict__ axes,
                          const typename Vec4<real>::T *__restrict__ e_wd,
                          const typename Vec4<real>::T *__restrict__ out_e, const float *__restrict__ delta,
                          real *__restrict__ potential, real *__restrict__ forces, real *__restrict__ epart,
                          const double *__restrict__ grad_energy, real *__restrict__ grad_q,
                          int backward, real sphi, real sF) {
    // sphi = 1/L and sF = 1/L^2 come from the host: no FP64 arithmetic per thread
    __shared__ real sh[UNSPLIT_BS / 32][2];
    double gE = backward ? *grad_energy : 0.0;
    real ehi = 0, elo = 0;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
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
            epart[2 * blockIdx.x] = h;
            epart[2 * blockIdx.x + 1] = l;
        }
    }
}

// total energy from the blocks' (hi, lo) pairs: strided per-thread pair sums,
// warp trees, then the warps' pairs in order (fixed order: deterministic);
// E = (hi + lo) / 2 in FP64 once
template <typename real>
__global__ void k_energy_final(const real *__restrict__ epart, int nb, double *energy) {
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

__global__ void k_zero_energy(double *energy) { *energy = 0.0; }

template <typename real>
void launch_unsplit(const Geom &g, const Ptrs<real> &P, const WsLayout &W, int n, const float *q,
                    real *potential, double *energy, real *forces, const double *grad_energy,
                    real *grad_q, bool backward, cudaStream_t st, Tracer &tr) {
    tr.begin(FMM_STAGE_UNSPLIT, st);
    if (n == 0) {
        if (energy && !backward) {
            k_zero_energy<<<1, 1, 0, st>>>(energy);
            tr.count();
        }
        tr.end();
        return;
    }
    int nb = (n + UNSPLIT_BS - 1) / UNSPLIT_BS;
    real *ep = (!backward && energy) ? reinterpret_cast<real *>(P.epart) : nullptr;  // [nb][2]
    // unit box -> box of edge L: potentials of 1/r^k scale by L^-k, forces by L^-(k+1)
    const double iL = 1.0 / g.L, sphi = g.power == 2 ? iL * iL : iL;
    k_unsplit<real><<<nb, UNSPLIT_BS, 0, st>>>(
        g, P.hdr, n, q, g.continuous ? P.offset : nullptr, P.count, P.axes,
        g.continuous ? P.e_wd : nullptr, P.out_e,
        (std::is_same<real, float>::value && g.continuous && g.force_mode == FMM_FORCE_ADJOINT) ? P.delta : nullptr,
        potential, forces, ep, grad_energy, grad_q,
        backward ? 1 : 0, (real)sphi, (real)(sphi * iL));
    tr.count();
    if (ep) {
        k_energy_final<real><<<1, 1024, 0, st>>>(ep, nb, energy);
        tr.count();
    }
    tr.end();
}

void launch_split_delta(const Geom &g, const Coef<double> &Cd, const Ptrs<float> &P, const WsLayout &W, int n,
                        const float *pos, cudaStream_t st, Tracer &tr) {
    if (n <= 0) return;
    tr.begin(FMM_STAGE_UNSPLIT, st);
    const int nb = (n + 32 * SD_WARPS - 1) / (32 * SD_WARPS);  // 32 particles per warp
    const float *leaf = reinterpret_cast<const float *>(P.loc) + W.loc_level[g.depth];
    // charges per pass: the charges of a particle split along one axis
    const int ch = g.p <= 4 ? 4 : (g.p <= 6 ? 6 : 8);
#define SD_LAUNCH(POW, CH)                                                                                  \
    k_split_delta<POW, CH><<<nb, 32 * SD_WARPS, 0, st>>>(g, Cd, n, pos, P.count, P.offset, P.leaf_start, P.s_pt, \
                                                        P.s_origin, leaf, P.delta, P.hdr)
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
